// Internal declarations shared by the engine (host) and the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/tucket.h"

#define TK_MAXP TK_MAX_MODES
#define TK_MAXL 40      // tree levels (2^39 leaf blocks)
#define TK_MAXH 64      // hits per stitch job handled by the kernel
#define TK_NT 256       // threads per CTA of the leaf kernel
#define TK_HITREC_BYTES 176  // bytes of one hit record in a stitch job's workspace

// Device view of a tree: dimensions, the implicit dyadic node numbering and
// the pooled HBM arena.  Passed by value to every kernel.
//
// Node (level j, index k) covers leaf blocks [k 2^j, (k+1) 2^j), i.e. slices
// [k 2^j B, min((k+1) 2^j B, T)).  It is complete (a leaf or an intermediate
// node of Section 4.2) iff (k+1) 2^j <= nb, the number of complete blocks; the
// open block (level 0, index nb, when T > nb B) is the tail leaf.  Its slot
// is level_base[j] + k.
struct TkTreeView {
  int p;
  int D[TK_MAXP];          // D[0] unused (time)
  int r[TK_MAXP];          // build ranks (slot capacities)
  int B;
  int theta_num, theta_den;
  int max_iter;
  double tol;
  int eig64;               // FP32 tree: stitch eigenproblems (tridiagonal method) in FP64
  int init;                // Stitch start: TK_INIT_HOSVD or TK_INIT_RANDOM (seeded)
  uint64_t seed;
  int64_t T, nb, nbt;      // slices, complete blocks, blocks incl. the tail
  int height;              // ceil(log2 nbt) + 1, 0 when empty
  int nlevels;
  int64_t level_base[TK_MAXL];
  int64_t T_cap;           // rows per level of the temporal arrays
  void* core_pool;         // slot * core_stride, capacity dims r[0..p-1]
  int64_t core_stride;
  void* fac_pool[TK_MAXP]; // mode n >= 1: slot * fac_stride[n], D_n x r_n rows
  int64_t fac_stride[TK_MAXP];
  void* tfac;              // level * tfac_level_stride + t * r[0]: temporal rows
  int64_t tfac_level_stride;
  int* node_ranks;         // slot * TK_MAXP: logical ranks of the stored node
};

struct TkWorkspace {
  void* base;              // per-worker chunks of `per_cta` elements (a worker is a
                           // CTA in k_stitch and a cluster in k_leaf)
  int64_t per_cta;         // elements per worker (k_leaf: per cluster)
  int nsm;                 // unused by the current kernels
  int warps;               // warps per CTA of k_stitch
  size_t smem_arena;       // k_stitch: bytes of the per-job shared arena
  int* status;             // first device-side error (0 = none)
  unsigned* counter;       // k_stitch job queue, zeroed before each launch
};

enum { TK_JOB_QUERY = 0, TK_JOB_MERGE = 1 };

struct TkQueryBatch {
  int n;
  const int64_t* ranges;   // device, 2n
  const int64_t* offsets;  // device, n+1
  void* out;               // device
  tk_query_info* info;     // device, n (may be null)
  const int* order;        // device, n: processing order (may be null: index order)
  const int* split;        // device (may be null): leading entries of `order` that are heavy
  int rq[TK_MAXP];         // requested ranks
  const int64_t* tq;       // device, n (may be null): the T each query is answered at
                           // (<= the tree's T; a query must not reach into that T's open block
                           // unless it is the tree's current T)
};

#define TK_LEAF_CL 8  // CTAs of the thread-block cluster that decomposes one leaf block

// Workspace of one leaf cluster: element offsets into its chunk, computed on
// the host from the build dimensions and ranks (upper bounds for any block).
struct TkLeafLayout {
  int64_t U[TK_MAXP];      // factor of mode n: D_n x r_n (mode 0: B x r_1)
  int64_t Vs[TK_MAXP];     // saved eigenbasis of mode n (D_n x D_n), the warm start
  int64_t part[TK_MAXP];   // TK_LEAF_CL partial Grams of mode n (D_n x D_n each)
  int64_t norm;            // TK_LEAF_CL partial squared norms
  int64_t flag;            // stop flag of the ALS loop
  int64_t Y;               // mat_n(Y_n), D_n x prod_{m!=n} r_m, row-major
  int64_t G;               // core
  int64_t cta, cta_stride; // per-CTA regions: start and size
  // offsets within a CTA region
  int64_t slab, b0, b1;    // gathered slab of X and the TTM chain buffers
  int64_t T;               // warm-start product of the eigensolver
  int64_t trd;             // vectors of the tridiagonal eigensolver
  int64_t A, V, w, cs, pq; // eigensolver arrays when they do not fit shared memory
  int64_t half;            // entries of each rotation array (order / 2 + 2)
  int nsa;                 // largest order whose eigenproblem matrix A is in shared memory
  int nsv;                 // largest order whose Jacobi arrays (V, rotations) are in shared memory
  int neig;                // largest Gram order of a block
  int rmax;                // largest rank
  int tc;                  // Grams on the tensor cores: 0 no, 1 split TF32 (FP32 accuracy), 2 TF32
  int64_t tc_bytes;        // shared-memory bytes of the tensor-core staging buffers
};

// Launchers (tk_kernels.cu, tk_leaf.cu).  All asynchronous on `stream`.
// k_leaf runs nclusters clusters of TK_LEAF_CL CTAs over njobs blocks.
int tk_launch_leaf(int dtype, const TkTreeView& tv, const void* raw, int64_t block_stride,
                   int64_t first_block, int njobs, int ell, const TkWorkspace& ws,
                   const TkLeafLayout& ly, int nclusters, cudaStream_t stream);
size_t tk_leaf_smem_bytes(int dtype, int nsa, int nsv, int neig, int rmax, int64_t tc_bytes);
size_t tk_leaf_contraction_bytes(int dtype, int neig, int rmax);
int tk_leaf_max_clusters(int dtype, size_t smem);
int tk_launch_merge(int dtype, const TkTreeView& tv, int level, int64_t k0, int njobs,
                    const TkWorkspace& ws, int grid, cudaStream_t stream);
int tk_launch_query(int dtype, const TkTreeView& tv, const TkQueryBatch& qb,
                    const TkWorkspace& ws, int grid, cudaStream_t stream);
// k_batch: one 512-thread CTA per SM for a planned batch (order, split); the
// workspace holds 2 chunks of ws.per_cta elements per CTA, ws.smem_arena is
// the arena of one half.
int tk_launch_batch(int dtype, const TkTreeView& tv, const TkQueryBatch& qb, const TkWorkspace& ws, int grid,
                    cudaStream_t stream);
size_t tk_batch_smem_bytes(int dtype, size_t half_arena);
// order[0..n) longest first; *split = how many queries have >= heavy_hits hits.
int tk_launch_plan(const TkTreeView& tv, int n, const int64_t* ranges, const int64_t* tq, int heavy_hits, int* split,
                   int* order, cudaStream_t stream);
int tk_launch_hitset(const TkTreeView& tv, int n, const int64_t* ranges, tk_hit* out, int cap,
                     int* counts, cudaStream_t stream);

// Shared-memory bytes of a stitch CTA with a job arena of `arena` bytes.
size_t tk_stitch_smem_bytes(int dtype, size_t arena);
int tk_occupancy(int dtype, size_t smem, int threads);  // stitch CTAs per SM

enum { TK_DEV_ERR_WORKSPACE = 1, TK_DEV_ERR_HITS = 2, TK_DEV_ERR_RANGE = 3 };
