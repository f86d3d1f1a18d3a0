/*
 * tucket.h -- C ABI of the GB300 engine for range queries of Tucker
 * decomposition over a stream segment tree (TUCKET, arXiv 2501.06647).
 *
 * Problem (Section 3 of the paper): a tensor stream X of shape
 * T x D_2 x ... x D_p grows by one slice X_T (D_2 x ... x D_p) per stream
 * update; a range query [t_s, t_e) asks for a Tucker decomposition
 * G x_1 U1 ... x_p Up of the subtensor X[t_s:t_e), with G of shape
 * r_1 x ... x r_p, U1 of shape (t_e - t_s) x r_1 and Un of shape D_n x r_n.
 *
 * Conventions shared by every call:
 *  - Mode 0 is time (the paper's mode 1).  Tensors are dense, row-major
 *    (C order), which is the paper's vec ordering (Appendix A).
 *  - Element type is the tree's dtype: double (TK_F64) or float (TK_F32).
 *  - Time ranges are half open, 0 <= t_s < t_e <= T.
 *  - Pointers are device pointers unless the call's `io` argument is
 *    TK_IO_HOST, in which case the data pointers are host pointers and the
 *    library copies through its own device staging buffers.  A pointer passed
 *    as device memory must be device (or managed) memory of the tree's GPU;
 *    anything else (host memory, another GPU's memory) gives TK_ERR_ARG
 *    before any work is issued.
 *  - The caller owns every buffer it passes; the library owns the tree's
 *    device arena and workspaces.  Inputs are consumed before the call's
 *    stream work completes; the library never keeps a caller pointer.
 *  - Calls are asynchronous on the tree's stream unless stated otherwise;
 *    tk_sync() waits and reports device-side errors.
 *  - Every function returns TK_OK (0) or a negative tk_status; a call that
 *    fails argument validation changes nothing.  No exception crosses the ABI.
 *  - One tree must not be used from two host threads at once.
 */
#ifndef TUCKET_H
#define TUCKET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TK_MAX_MODES 8

typedef enum tk_status {
  TK_OK = 0,
  TK_ERR_ARG = -1,         /* malformed argument (null pointer, bad config) */
  TK_ERR_RANGE = -2,       /* time range outside [0, T) or empty */
  TK_ERR_RANK = -3,        /* query rank < 1 or above the build rank */
  TK_ERR_NOMEM = -4,       /* device allocation failed */
  TK_ERR_CUDA = -5,        /* a CUDA runtime call failed */
  TK_ERR_STATE = -6,       /* call not valid in the tree's current state */
  TK_ERR_WORKSPACE = -7,   /* device job exceeded its workspace (reported by tk_sync) */
  TK_ERR_TOO_BIG = -8,     /* request exceeds a fixed limit of the engine */
  TK_ERR_TIMEOUT = -9,     /* a wait ran out of time */
  TK_ERR_IO = -10          /* a tree file could not be read or written, or is not one */
} tk_status;

typedef enum tk_dtype { TK_F64 = 0, TK_F32 = 1 } tk_dtype;
/* Arithmetic of the leaf blocks' Gram matrices (the dense contractions of
 * Tucker-ALS over raw data, Section 2), for FP32 trees:
 *   TK_MATH_AUTO       tensor cores with split TF32 products (hi*hi + hi*lo +
 *                      lo*hi, FP32 accumulation), FP32 accuracy (FP64 trees:
 *                      FP64 CUDA cores);
 *   TK_MATH_CUDA_CORES FP32 (or FP64) CUDA cores;
 *   TK_MATH_TF32       tensor cores with one TF32 product (FP32 accumulation):
 *                      faster, about 1e-3 relative error per product.
 * Everything else (the stitch, eigensolvers, QR) runs in the tree's dtype,
 * except the stitch eigenproblems under tk_config.eig_fp64. */
typedef enum tk_math { TK_MATH_AUTO = 0, TK_MATH_CUDA_CORES = 1, TK_MATH_TF32 = 2 } tk_math;
typedef enum tk_io { TK_IO_DEVICE = 0, TK_IO_HOST = 1 } tk_io;

/* Start of Stitch (Algorithm 2), for queries and node merges alike:
 *   TK_INIT_HOSVD   the implicit HOSVD of the stitched tensor (default;
 *                   deterministic, no random numbers);
 *   TK_INIT_RANDOM  the paper's random U^(2..p), drawn from tk_config.seed by
 *                   a counter-based generator: splitmix64 outputs
 *                   mix(seed + (k+1) * 0x9E3779B97F4A7C15), uniforms
 *                   ((out >> 11) + 1) * 2^-53, Box-Muller Gaussians (even
 *                   element: cos, odd: sin), mode n = 2..p a D_n x r_n
 *                   row-major matrix from element sum_{m<n} D_m r_m on (r the
 *                   stitch's output ranks), orthonormalized by QR.  The same
 *                   seed serves every stitch, so answers are reproducible.
 * The leaf blocks' Tucker-ALS always starts from the HOSVD of the block. */
typedef enum tk_init { TK_INIT_HOSVD = 0, TK_INIT_RANDOM = 1 } tk_init;

/* Tree configuration.  Hyperparameter defaults follow Section 8.1 of the
 * paper: at most 20 ALS iterations, tolerance 0.01, theta = 0.7. */
typedef struct tk_config {
  int32_t p;                        /* number of modes, 2..TK_MAX_MODES */
  int64_t dims[TK_MAX_MODES];       /* dims[1..p-1] = D_2..D_p; dims[0] unused */
  int32_t ranks[TK_MAX_MODES];      /* build ranks r_1..r_p (>= 1) */
  int32_t leaf_slices;              /* B: slices per leaf block (>= 1; 1 = paper) */
  int32_t theta_num, theta_den;     /* pruning threshold theta = num/den in (0,1] */
  int32_t max_iter;                 /* ALS iteration cap for leaves and stitches */
  double tol;                       /* stop when |e_k - e_{k-1}| < tol; <= 0: run max_iter */
  int32_t dtype;                    /* tk_dtype */
  int32_t device;                   /* CUDA device ordinal */
  int64_t hbm_budget;               /* device bytes the tree may hold (0: no limit) */
  int32_t math;                     /* tk_math of the leaf Grams (TK_MATH_TF32: FP32 trees only) */
  int32_t eig_fp64;                 /* 1: an FP32 tree solves the eigenproblems of its stitches
                                       (queries and node merges, Algorithm 2) in FP64 on the GPU,
                                       for orders >= 20 (the tridiagonal method; smaller orders
                                       use FP32 Jacobi); 0 (default): in the tree's dtype.  FP64
                                       trees ignore it.  0 or 1. */
  uint64_t seed;                    /* seed of TK_INIT_RANDOM */
  int32_t init;                     /* tk_init of Stitch (default TK_INIT_HOSVD) */
} tk_config;

/* One node of a hit set (Algorithm 1, Section 5.1), in time order. */
typedef struct tk_hit {
  int32_t level;                    /* 0 = leaf block; level j spans 2^j blocks */
  int32_t partial;                  /* 1 if the node is not contained in the query */
  int64_t index;                    /* node index within its level */
  int64_t node_lo, node_hi;         /* node range [sigma, tau) in slices */
  int64_t lo, hi;                   /* clipped range [max(t_s,sigma), min(t_e,tau)) */
} tk_hit;

/* Per-query report. */
typedef struct tk_query_info {
  int32_t ranks[TK_MAX_MODES];      /* effective output ranks (<= requested) */
  int32_t iters;                    /* ALS iterations run; < 0 on a device-side error */
  int32_t n_hits;                   /* hit-set size s */
  double fit_err;                   /* sqrt(1 - ||G||^2 / ||Y~||^2) of the stitched tensor */
  int32_t eig_sweeps;               /* Jacobi sweeps summed over the query's eigenproblems */
  int32_t eig_max_order;            /* largest eigenproblem order of the query */
  int64_t device_cycles;            /* SM clock cycles the query's job group spent on it */
  int64_t eig_cycles;               /* of which in the eigensolver (Jacobi) */
  int64_t qr_cycles;                /* of which in Householder QR (partial hits and Phi_n) */
  int64_t hit_cycles;               /* stage 1: hit set, stored or partial-hit decompositions */
  int64_t init_cycles;              /* stage 2: QR of the stacked factors and the HOSVD start */
  int64_t als_cycles;               /* stage 3: the ALS iterations of Algorithm 2 */
  int64_t out_cycles;               /* stage 4: core and factor assembly into the output */
  int64_t start_ns, end_ns;         /* GPU global timer when the query's job started and ended */
} tk_query_info;

typedef struct tk_tree tk_tree;

/* Fill *cfg with defaults: p = 3, ranks 10, B = 1, theta = 7/10,
 * max_iter = 20, tol = 0.01, TK_F32, device 0, no memory budget.  dims must
 * still be set. */
int tk_config_default(tk_config* cfg);

/* Create an empty stream segment tree (Section 4.2: before the first stream
 * update there is no node; Algorithm 4 creates the first leaf) with T = 0,
 * on cfg->device.  cuda_stream is a
 * cudaStream_t to run on, or NULL for a stream the tree creates and owns.
 *
 * Memory budget: with cfg->hbm_budget > 0, every call that would take the
 * device bytes the tree holds (node arena, workspaces, staging buffers,
 * the open block's slices) above the budget returns TK_ERR_NOMEM before
 * changing anything; so does tk_tree_create when the empty tree does not fit.
 * An arena that grows holds its old and new copies together while the nodes
 * are copied, and the check counts both.  Not counted: a server's own
 * buffers (sized by tk_server_config). */
int tk_tree_create(const tk_config* cfg, void* cuda_stream, tk_tree** out);
void tk_tree_destroy(tk_tree* t);

/* Build the tree over X (T x D_2 x ... x D_p) on an EMPTY tree.  The result
 * is the tree that T successive tk_stream_append calls produce (Section 4.2,
 * Algorithms 3-4): leaf blocks are decomposed by Tucker-ALS (Section 2) and
 * every complete intermediate node by Stitch (Algorithm 2) of its children. */
int tk_tree_build(tk_tree* t, const void* X, int64_t T, int io);

/* Stream update (Section 3, Algorithm 4): append one slice.  When a leaf
 * block completes, the leaf is decomposed and the nu_2(#blocks) newly
 * complete ancestors are re-decomposed by Stitch of their two children. */
int tk_stream_append(tk_tree* t, const void* slice, int io);

/* The timespan T of the stream (Section 3: the tensor X has T slices after T
 * stream updates), i.e. the largest valid t_e of a range query; -1 for NULL. */
int64_t tk_timespan(const tk_tree* t);

/* Pruned hit set of [t_s, t_e) (Algorithm 1), written to host array out.
 * Synchronous.  *n_out receives the hit count; TK_ERR_TOO_BIG if > cap. */
int tk_hit_set(tk_tree* t, int64_t t_s, int64_t t_e, tk_hit* out, int cap, int* n_out);

/* Elements of one query's packed output for ranks r (NULL = build ranks):
 *   prod_n r_n  (core, r_1 x ... x r_p)
 * + (t_e - t_s) * r_1  (U1, row-major)
 * + sum_{n>=2} D_n * r_n  (Un, row-major).
 * Entries beyond the effective ranks are zero.  Returns < 0 on error. */
int64_t tk_query_output_elems(const tk_tree* t, int64_t t_s, int64_t t_e, const int32_t* ranks);

/* Range query of Tucker decomposition (Section 6.1): Recall, partial-hit
 * approximation (Eq. partial-tucker), Stitch (Algorithm 2).  `out` holds
 * tk_query_output_elems() elements.  ranks = NULL means the build ranks.
 * If info != NULL (host pointer) the call is synchronous and fills it. */
int tk_range_query(tk_tree* t, int64_t t_s, int64_t t_e, const int32_t* ranks,
                   void* out, tk_query_info* info, int io);

/* Batched range queries: n independent queries in one persistent launch.
 * ranges: 2n int64 (t_s, t_e pairs); offsets: n+1 int64 element offsets of
 * each query's packed output in `out` (tk_batch_layout computes them).
 * With io = TK_IO_DEVICE, ranges/offsets/out are device pointers and the
 * call is asynchronous; with TK_IO_HOST they are host pointers and the call
 * copies in, computes, copies out and synchronizes.  info: optional host
 * array of n reports (makes the call synchronous).  The launch is ordered on
 * the tree's stream only: device buffers that work on another stream writes
 * (a fill of `out`, say) must be complete before the call, or that stream
 * must be the tree's; a tree created with a NULL stream runs on a stream of
 * its own that does not synchronize with the legacy default stream. */
int tk_batch_layout(const tk_tree* t, int n, const int64_t* ranges_host,
                    const int32_t* ranks, int64_t* offsets_host);
int tk_range_query_batch(tk_tree* t, int n, const int64_t* ranges, const int64_t* offsets,
                         const int32_t* ranks, void* out, tk_query_info* info, int io);

/* Launch shape of tk_range_query_batch (no counterpart in the paper).  Its
 * persistent kernel runs each query whose hit set has at least `hits` nodes
 * on a whole 512-thread CTA with both shared-memory arenas, and every other
 * query on a 256-thread half CTA: a whole CTA shortens one query, halves keep
 * two queries in flight per SM.  hits = 0 restores the default,
 * max(3, ceil(55 / largest build rank)); values above the kernel's hit limit
 * (64) run every query on a half.  Answers do not depend on it beyond
 * rounding order.  TK_ERR_ARG for a NULL tree or hits < 0.
 * tk_batch_get_heavy_hits reports the threshold in use. */
int tk_batch_set_heavy_hits(tk_tree* t, int hits);
int tk_batch_get_heavy_hits(const tk_tree* t, int* hits);

/* Autotuner of that launch shape (no counterpart in the paper): runs the
 * batch as tk_range_query_batch with io = TK_IO_DEVICE would (ranges,
 * offsets, out: device pointers of the tree's GPU; out is overwritten), for
 * each candidate threshold in {3, 4, 5, 6, 7, 8, 10, 12, 16, 24, 32, 65}
 * once untimed and then `reps` times timed with CUDA events on the tree's
 * stream, skipping a candidate that selects the same heavy queries as the
 * previous one; keeps the fastest (best of its reps) with
 * tk_batch_set_heavy_hits and reports it in *best_hits and its time in
 * *best_ms (optional; -1 when n = 1, which needs no tuning).  Synchronous.
 * Errors: TK_ERR_ARG for NULL or host pointers, n < 1 or reps < 1; the
 * errors of tk_range_query_batch, after which the threshold is left as it
 * was. */
int tk_batch_tune(tk_tree* t, int n, const int64_t* ranges_dev, const int64_t* offsets_dev,
                  const int32_t* ranks, void* out_dev, int reps, int* best_hits, float* best_ms);

/* Copy a stored node's decomposition to host memory, packed like a query
 * output with the build ranks and the node's full time range (for tests).
 * ranks_out (TK_MAX_MODES) receives the node's ranks.  Synchronous. */
int tk_node_payload(tk_tree* t, int level, int64_t index, void* out_host,
                    int64_t out_elems, int32_t* ranks_out);

/* Device bytes held by the tree's node arena (cores, factors, temporal rows). */
int64_t tk_arena_bytes(const tk_tree* t);

/* Wait for the tree's stream; return the first device-side error, if any. */
int tk_sync(tk_tree* t);

/* Kernel launches issued by this tree since creation (all engine kernels). */
int64_t tk_launch_count(const tk_tree* t);

const char* tk_strerror(int code);

/* Measurement helper with no counterpart in the paper: the rate of fused
 * multiply-adds in dtype (TK_F32 or TK_F64) that device sustains, in FLOP/s
 * (2 per FMA), from a kernel of independent FMA chains on every SM timed with
 * CUDA events (best of 3 after a warm-up).  It is the denominator of the
 * engine's arithmetic roofline.  Synchronous; allocates a small buffer. */
int tk_probe_fma_rate(int dtype, int device, double* flops_per_s);

/* Copy of the configuration the tree was created with. */
int tk_tree_get_config(const tk_tree* t, tk_config* out);

/* ---- Tree files (checkpoint and resume of a stream summary) --------------
 *
 * The tree is the stream's persistent summary (Section 4): after a restart a
 * stream can resume from a saved tree instead of re-decomposing its history.
 *
 * tk_tree_save writes the tree to the file `path` (created or truncated):
 * its configuration, its time span T, the node arena (the core, the factors
 * of every mode, the temporal factor rows and the ranks of every stored
 * node, including the open block's decomposition when it is current) and the
 * raw slices of the open leaf block.  Synchronous: it first waits for the
 * tree's stream and returns the first device-side error, if any, without
 * writing.  The file holds the host's byte order and the element size and is
 * read back only by tk_tree_load.  Not valid while a server uses the tree.
 *
 * tk_tree_load creates a tree from such a file, on `device` (-1: the device
 * recorded in the file) and `cuda_stream` (as for tk_tree_create), and
 * returns it in *out.  Its arena holds the saved bytes, so it answers every
 * query and takes further appends exactly as the saved tree would.
 * Synchronous.
 *
 * Both return TK_ERR_IO when the file cannot be opened, written or read, or
 * is not a complete tree file of this format (wrong header, sizes that do
 * not match its configuration, missing or trailing bytes); tk_tree_load
 * also returns the errors of tk_tree_create.  On error tk_tree_load leaves
 * *out NULL and frees what it created. */
int tk_tree_save(tk_tree* t, const char* path);
int tk_tree_load(const char* path, int device, void* cuda_stream, tk_tree** out);

/* ---- Serving: continuous batching of queries and appends ---------------
 *
 * A server owns a worker thread that executes the requests submitted to it,
 * from any host thread, in ticket (arrival) order: a range query sees every
 * stream update submitted before it and none submitted after it (Section 3's
 * two operations, served concurrently).  Appends are issued at once, in
 * stream order behind the batches already running; an append's ticket
 * completes when it has been issued.  Queries are admitted into one batched
 * launch, up to max_batch queries and max_batch_out_elems output elements
 * (the device memory a batch may hold), each answered against the tree as of
 * its own submission (nodes complete then are never changed by later
 * appends); a query that reaches into the open block of its time makes the
 * batch launch before the next append.  The next batch is enqueued while
 * the current one runs.  While a server exists, the tree must not be used
 * directly. */
typedef struct tk_server tk_server;
typedef struct tk_server_config {
  int32_t max_batch;               /* queries per batch (default 1024) */
  int64_t max_batch_out_elems;     /* output elements per batch (default 16 Mi) */
} tk_server_config;
typedef struct tk_server_stats {
  int64_t queries_done, appends_done, batches;
  double mean_batch;               /* queries per batch */
  double latency_p50_ms, latency_p99_ms, latency_max_ms;  /* queries: submit to completion */
  double elapsed_s;                /* first submit to last completion */
} tk_server_stats;

/* cfg may be NULL (defaults). */
int tk_server_create(tk_tree* t, const tk_server_config* cfg, tk_server** out);
/* Queue a range query [t_s, t_e) (checked against T including queued
 * appends); the packed output (tk_query_output_elems layout) is written to
 * out_host and the report to info_host (may be NULL) on completion. */
int tk_server_submit_query(tk_server* s, int64_t t_s, int64_t t_e, const int32_t* ranks, void* out_host,
                           tk_query_info* info_host, uint64_t* ticket);
/* Queue a stream update; the slice (host memory) is copied at submission. */
int tk_server_submit_append(tk_server* s, const void* slice_host, uint64_t* ticket);
/* Wait for one request (timeout_s < 0: no limit); returns its status, or
 * TK_ERR_TIMEOUT.  A ticket's status can be collected once: an unknown or
 * already collected ticket gives TK_ERR_ARG.  Statuses that are never
 * collected are kept until the server is destroyed. */
int tk_server_wait(tk_server* s, uint64_t ticket, double timeout_s);
/* Wait until every submitted request has completed. */
int tk_server_drain(tk_server* s, double timeout_s);
int tk_server_get_stats(tk_server* s, tk_server_stats* out);
/* Finish the queued requests, stop the worker and free the server. */
void tk_server_destroy(tk_server* s);

/* ---- Allocation-free range queries (no counterpart in the paper) --------
 *
 * tk_range_query_batch_noalloc answers the same batched range queries as
 * tk_range_query_batch with io = TK_IO_DEVICE, but makes no device
 * allocation of any kind: no cudaMalloc/cudaFree and no allocating library
 * routine.  Its answers equal tk_range_query_batch's to rounding (the
 * regular call runs queries with many hits on wider thread groups, which sums
 * in another order): within 1e-9 relative error and 1e-3 rad in FP64 and
 * 1e-6 per element in FP32, as its tests check.
 *
 * It exists for callers that cannot let a library allocate device memory at
 * query time: code that runs under a memory manager or arena of its own (an
 * embedding runtime, a database engine), real-time or serving loops whose
 * latency budget rules out the device-wide synchronization that
 * cudaMalloc/cudaFree may cause, and processes that must keep a fixed
 * device-memory footprint after start-up.
 *
 * Its scratch is one file-scope device array of TK_NOALLOC_SCRATCH_BYTES
 * (16 MiB), held by every GPU that loads the library until the process
 * exits.  The first call on a device resolves the array's address on that
 * device (set-up, once per device); make that first call before any CUDA
 * stream capture.  All calls share the array and it keeps the last call's
 * contents: the call clears what must start at zero (its job counter), and
 * calls whose work overlaps on the GPU (two streams, two trees, two host
 * threads) race on it, so serialize them.  Device-side errors (an invalid
 * range, a job that overflows its workspace) set the tree's own sticky status
 * word, as for every other call, and tk_sync reports them.
 *
 * ranges (2n int64), offsets (n+1 int64, from tk_batch_layout) and out are
 * device pointers owned by the caller, as for tk_range_query_batch.  info is
 * an optional host array of n reports; with info the call synchronizes and
 * returns what tk_sync would, without it the call is asynchronous.
 * Returns TK_ERR_TOO_BIG when one query's workspace (which grows with the
 * tree's capacity, ranks and dimensions) does not fit the scratch array; the
 * reports of a call with info are staged in the same array (n times
 * sizeof(tk_query_info) bytes), so with info they also bound n,
 * TK_ERR_STATE when the open leaf block still awaits its decomposition (any
 * regular query, tk_node_payload, or the append that completes the block
 * decomposes it), and the usual argument and rank errors. */
#define TK_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
int tk_range_query_batch_noalloc(tk_tree* t, int n, const int64_t* ranges_dev, const int64_t* offsets_dev,
                                 const int32_t* ranks, void* out_dev, tk_query_info* info);

#ifdef __cplusplus
}
#endif
#endif /* TUCKET_H */
