// Host side of the engine: the C ABI of include/tucket.h, the tree metadata,
// the pooled HBM arena, the workspaces, and the launch sequences of tree
// build (Section 4.2), stream update (Algorithms 3-4) and range query
// (Section 6.1).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "tk_device.cuh"
#include "tk_internal.h"
#include "tk_tc.cuh"

namespace {

int64_t next_pow2(int64_t x) {
  int64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

int ceil_log2(int64_t x) {
  int h = 0;
  while (((int64_t)1 << h) < x) ++h;
  return h;
}

struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct tk_tree {
  tk_config cfg{};
  int dev = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t es = 4;
  int p = 0;
  int64_t slice_elems = 0;
  // state
  int64_t T = 0, nb = 0;
  bool tail_dirty = false;
  // arena capacity
  int64_t nbcap = 0;
  int nlevels = 0;
  int64_t level_base[TK_MAXL] = {};
  int64_t nslots = 0;
  int64_t core_stride = 0;
  int64_t fac_stride[TK_MAXP] = {};
  DevBuf core_pool, fac_pool[TK_MAXP], tfac, node_ranks, tail_raw;
  // workspaces
  DevBuf ws_stitch, ws_leaf, status;
  int64_t ws_stitch_per_cta = 0, ws_leaf_per_cta = 0;
  int ws_stitch_ctas = 0, ws_leaf_ctas = 0;
  int nsm_stitch = 0, nsa_leaf = 0, nsv_leaf = 0, tc_leaf = 0;
  int64_t tc_bytes_leaf = 0;
  int sm_count = 0;
  int smem_optin = 0;  // shared memory a block may opt in to (bytes)
  int heavy_set = 0;  // batch heavy-query threshold set by the caller (0: default)
  // staging for host io and batch metadata
  DevBuf stage_in, stage_out, stage_meta, stage_info, hit_buf, plan;
  int64_t launches = 0;
};

namespace {

int cuda_ok(cudaError_t e) { return e == cudaSuccess ? TK_OK : TK_ERR_CUDA; }

// A caller's buffer passed as device memory must be device (or managed)
// memory of the tree's GPU: a host pointer handed to a kernel would fault.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

int dalloc(DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes && b.ptr) return TK_OK;
  if (b.ptr) cudaFree(b.ptr);
  b.ptr = nullptr;
  b.bytes = 0;
  if (bytes == 0) return TK_OK;
  if (cudaMalloc(&b.ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    b.ptr = nullptr;
    return TK_ERR_NOMEM;
  }
  b.bytes = bytes;
  return TK_OK;
}

void dfree(DevBuf& b) {
  if (b.ptr) cudaFree(b.ptr);
  b.ptr = nullptr;
  b.bytes = 0;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// Device bytes the tree holds in its own buffers.
size_t held_bytes(const tk_tree* t) {
  const DevBuf* bufs[] = {&t->core_pool, &t->tfac, &t->node_ranks, &t->tail_raw, &t->ws_stitch, &t->ws_leaf,
                          &t->status, &t->stage_in, &t->stage_out, &t->stage_meta, &t->stage_info,
                          &t->hit_buf, &t->plan};
  size_t b = 0;
  for (const DevBuf* x : bufs) b += x->bytes;
  for (int n = 0; n < TK_MAXP; ++n) b += t->fac_pool[n].bytes;
  return b;
}

// True when the tree may hold `add` more bytes after releasing `drop`
// (cfg.hbm_budget, 0 = no limit).
bool within_budget(const tk_tree* t, size_t drop, size_t add) {
  if (t->cfg.hbm_budget <= 0) return true;
  return held_bytes(t) - drop + add <= (size_t)t->cfg.hbm_budget;
}

// dalloc of one of the tree's buffers (or a temporary of a call) under the budget.
int tdalloc(tk_tree* t, DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes && b.ptr) return TK_OK;
  if (!within_budget(t, b.bytes, bytes)) return TK_ERR_NOMEM;
  return dalloc(b, bytes);
}

int64_t nbt_of(const tk_tree* t) { return (t->T + t->cfg.leaf_slices - 1) / t->cfg.leaf_slices; }

TkTreeView make_view(const tk_tree* t) {
  TkTreeView v{};
  v.p = t->p;
  for (int n = 0; n < TK_MAXP; ++n) {
    v.D[n] = n < t->p ? (int)t->cfg.dims[n] : 1;
    v.r[n] = n < t->p ? t->cfg.ranks[n] : 1;
  }
  v.D[0] = 1;
  v.B = t->cfg.leaf_slices;
  v.theta_num = t->cfg.theta_num;
  v.theta_den = t->cfg.theta_den;
  v.max_iter = t->cfg.max_iter;
  v.tol = t->cfg.tol;
  v.eig64 = (t->cfg.eig_fp64 && t->cfg.dtype == TK_F32) ? 1 : 0;
  v.init = t->cfg.init;
  v.seed = t->cfg.seed;
  v.T = t->T;
  v.nb = t->nb;
  v.nbt = nbt_of(t);
  v.height = v.nbt > 0 ? ceil_log2(v.nbt) + 1 : 0;
  v.nlevels = t->nlevels;
  for (int j = 0; j < TK_MAXL; ++j) v.level_base[j] = t->level_base[j];
  v.T_cap = t->nbcap * t->cfg.leaf_slices;
  v.core_pool = t->core_pool.ptr;
  v.core_stride = t->core_stride;
  for (int n = 0; n < TK_MAXP; ++n) {
    v.fac_pool[n] = t->fac_pool[n].ptr;
    v.fac_stride[n] = t->fac_stride[n];
  }
  v.tfac = t->tfac.ptr;
  v.tfac_level_stride = v.T_cap * t->cfg.ranks[0];
  v.node_ranks = (int*)t->node_ranks.ptr;
  return v;
}

// Arena layout for nbcap leaf blocks: level j holds nbcap >> j slots.
struct ArenaLayout {
  int nlevels;
  int64_t base[TK_MAXL];
  int64_t nslots;
};

ArenaLayout layout_for(int64_t nbcap) {
  ArenaLayout a{};
  a.nlevels = ceil_log2(nbcap) + 1;
  int64_t acc = 0;
  for (int j = 0; j < TK_MAXL; ++j) {
    a.base[j] = acc;
    if (j < a.nlevels) acc += std::max<int64_t>(1, nbcap >> j);
  }
  a.nslots = acc;
  return a;
}

// Grow the arena so that `need_blocks` leaf blocks fit; existing nodes are
// copied level by level into the new layout.
int ensure_capacity(tk_tree* t, int64_t need_blocks) {
  if (need_blocks <= t->nbcap) return TK_OK;
  const int64_t ncap = next_pow2(std::max<int64_t>(need_blocks, 1));
  const ArenaLayout L = layout_for(ncap);
  if (L.nlevels > TK_MAXL) return TK_ERR_TOO_BIG;
  const int p = t->p;
  const size_t es = t->es;
  const int r0 = t->cfg.ranks[0];
  const int64_t Tcap_new = ncap * t->cfg.leaf_slices;
  {
    size_t old_arena = t->core_pool.bytes + t->tfac.bytes + t->node_ranks.bytes, new_arena = 0;
    for (int n = 0; n < TK_MAXP; ++n) old_arena += t->fac_pool[n].bytes;
    new_arena += (size_t)L.nslots * t->core_stride * es;
    for (int n = 1; n < p; ++n) new_arena += (size_t)L.nslots * t->fac_stride[n] * es;
    new_arena += (size_t)L.nlevels * Tcap_new * r0 * es + (size_t)L.nslots * TK_MAXP * sizeof(int);
    // the old arena is released only after its levels were copied into the
    // new one, so both are held at once
    (void)old_arena;
    if (!within_budget(t, 0, new_arena)) return TK_ERR_NOMEM;
  }
  DevBuf core, fac[TK_MAXP], tf, nr;
  int rc = dalloc(core, (size_t)L.nslots * t->core_stride * es);
  for (int n = 1; n < p && rc == TK_OK; ++n) rc = dalloc(fac[n], (size_t)L.nslots * t->fac_stride[n] * es);
  if (rc == TK_OK) rc = dalloc(tf, (size_t)L.nlevels * Tcap_new * r0 * es);
  if (rc == TK_OK) rc = dalloc(nr, (size_t)L.nslots * TK_MAXP * sizeof(int));
  if (rc != TK_OK) {
    dfree(core);
    for (int n = 0; n < TK_MAXP; ++n) dfree(fac[n]);
    dfree(tf);
    dfree(nr);
    return rc;
  }
  cudaMemsetAsync(core.ptr, 0, core.bytes, t->stream);
  cudaMemsetAsync(tf.ptr, 0, tf.bytes, t->stream);
  cudaMemsetAsync(nr.ptr, 0, nr.bytes, t->stream);
  for (int n = 1; n < p; ++n) cudaMemsetAsync(fac[n].ptr, 0, fac[n].bytes, t->stream);
  if (t->nbcap > 0) {
    const int64_t Tcap_old = t->nbcap * t->cfg.leaf_slices;
    for (int j = 0; j < t->nlevels; ++j) {
      const int64_t cnt = std::max<int64_t>(1, t->nbcap >> j);
      cudaMemcpyAsync((char*)core.ptr + L.base[j] * t->core_stride * es,
                      (char*)t->core_pool.ptr + t->level_base[j] * t->core_stride * es,
                      cnt * t->core_stride * es, cudaMemcpyDeviceToDevice, t->stream);
      for (int n = 1; n < p; ++n)
        cudaMemcpyAsync((char*)fac[n].ptr + L.base[j] * t->fac_stride[n] * es,
                        (char*)t->fac_pool[n].ptr + t->level_base[j] * t->fac_stride[n] * es,
                        cnt * t->fac_stride[n] * es, cudaMemcpyDeviceToDevice, t->stream);
      cudaMemcpyAsync((char*)nr.ptr + L.base[j] * TK_MAXP * sizeof(int),
                      (char*)t->node_ranks.ptr + t->level_base[j] * TK_MAXP * sizeof(int),
                      cnt * TK_MAXP * sizeof(int), cudaMemcpyDeviceToDevice, t->stream);
      cudaMemcpyAsync((char*)tf.ptr + (size_t)j * Tcap_new * r0 * es,
                      (char*)t->tfac.ptr + (size_t)j * Tcap_old * r0 * es, Tcap_old * r0 * es,
                      cudaMemcpyDeviceToDevice, t->stream);
    }
    // the old buffers are released only after the copies ran
    cudaStreamSynchronize(t->stream);
  }
  dfree(t->core_pool);
  for (int n = 0; n < TK_MAXP; ++n) dfree(t->fac_pool[n]);
  dfree(t->tfac);
  dfree(t->node_ranks);
  t->core_pool = core;
  for (int n = 0; n < TK_MAXP; ++n) t->fac_pool[n] = fac[n];
  t->tfac = tf;
  t->node_ranks = nr;
  t->nbcap = ncap;
  t->nlevels = L.nlevels;
  for (int j = 0; j < TK_MAXL; ++j) t->level_base[j] = L.base[j];
  t->nslots = L.nslots;
  // workspaces depend on T_cap and the height: recompute lazily
  t->ws_stitch_per_cta = 0;
  t->ws_leaf_per_cta = 0;
  return TK_OK;
}

int64_t round32(int64_t x) { return (x + 31) & ~(int64_t)31; }

// Upper bound of a stitch job's workspace (elements), mirroring the device
// bump allocation of stitch_job with every rank at its build value.
int64_t stitch_ws_bound(const tk_tree* t, int hmax) {
  const int p = t->p;
  const int* r = t->cfg.ranks;
  int64_t rprod = 1;
  for (int n = 0; n < p; ++n) rprod *= r[n];
  const int64_t Tcap = t->nbcap * t->cfg.leaf_slices;
  int64_t tot = ((int64_t)TK_MAXH * TK_HITREC_BYTES + (int64_t)t->es - 1) / (int64_t)t->es;
  tot += hmax * round32(rprod);
  tot += 2 * (round32(Tcap * (r[0] + 1)) + round32(r[0]));  // at most two partial hits (odd-padded rows)
  int64_t k[TK_MAXP], c[TK_MAXP];
  int64_t neig = (int64_t)hmax * r[0];
  k[0] = c[0] = (int64_t)hmax * r[0];
  for (int n = 1; n < p; ++n) {
    const int64_t Dn = t->cfg.dims[n];
    k[n] = (int64_t)hmax * r[n];
    c[n] = std::min<int64_t>(Dn, k[n]);
    tot += round32(Dn * (k[n] + 1)) + round32(k[n]) + round32(c[n] * k[n]) + round32(c[n] * r[n]) + round32(c[n] * c[n]);
    neig = std::max(neig, c[n]);
  }
  tot += round32(c[0] * r[0]) + round32(c[0] * c[0]);
  int64_t Kel = k[0];
  for (int m = 1; m < p; ++m) Kel *= r[m];
  tot += round32(Kel);
  int64_t tb = 0;
  for (int n = 0; n < p; ++n) {
    int64_t s = 1;
    for (int m = 0; m < p; ++m) s *= (m == n) ? std::max<int64_t>(c[m], r[m]) : r[m];
    tb = std::max(tb, s);
  }
  tot += 3 * round32(tb);
  int64_t wmax = (int64_t)r[0] * r[0];
  for (int m = 0; m < p; ++m) wmax = std::max<int64_t>(wmax, (int64_t)r[m] * r[m]);
  tot += round32(wmax);
  tot += round32(rprod);
  // T of the warm start, and the eig scratch if it spills out of shared memory
  tot += 3 * round32(neig * neig) + round32(neig) + round32(neig + 2) + round32(2 * (neig / 2 + 2)) + round32(neig / 2 + 2);
  // vectors of the tridiagonal eigensolver (a group has at most 32 warps)
  int rmax = 1;
  for (int n = 0; n < p; ++n) rmax = std::max(rmax, r[n]);
  tot += round32(tk::trd_scratch_elems((int)neig, rmax, 32));
  if (t->cfg.init == TK_INIT_RANDOM) {  // the random start's Gaussian matrix, its Q, and tau
    int64_t dr = 0;
    for (int n = 1; n < p; ++n) dr = std::max<int64_t>(dr, t->cfg.dims[n] * (r[n] + 1));
    tot += 2 * round32(dr) + round32(rmax);
  }
  if (t->cfg.eig_fp64 && t->cfg.dtype == TK_F32)  // the FP64 eigenproblem's buffers, in float units
    tot += 2 * (round32(neig * neig) + round32(neig * rmax) + round32(tk::trd_scratch_elems((int)neig, rmax, 32)) + 32);
  return tot + 256;
}

// Workspace of one leaf cluster (see TkLeafLayout), with every rank at its
// build value and the block at its full B slices: bounds for any block.
// nsa / nsv: the shared-memory capacities (orders) of the eigensolvers.
TkLeafLayout leaf_layout(const tk_tree* t, int nsa, int nsv, int tc, int64_t tc_bytes, int64_t* per_cluster) {
  TkLeafLayout ly{};
  const int p = t->p;
  const int CL = TK_LEAF_CL;
  int64_t xd[TK_MAXP], r[TK_MAXP];
  xd[0] = t->cfg.leaf_slices;
  for (int n = 1; n < p; ++n) xd[n] = t->cfg.dims[n];
  for (int n = 0; n < p; ++n) r[n] = std::min<int64_t>(t->cfg.ranks[n], xd[n]);
  int64_t N = 1, rprod = 1, neig = 0;
  for (int n = 0; n < p; ++n) {
    N *= xd[n];
    rprod *= r[n];
    neig = std::max(neig, xd[n]);
  }
  int64_t cur = 0;
  auto take = [&](int64_t nel) {
    const int64_t o = cur;
    cur += round32(nel);
    return o;
  };
  int64_t ymax = 0;
  for (int n = 0; n < p; ++n) {
    ly.U[n] = take(xd[n] * r[n]);
    ly.Vs[n] = take(xd[n] * xd[n]);
    ly.part[n] = n > 0 ? take(CL * xd[n] * xd[n]) : 0;
    ymax = std::max(ymax, xd[n] * (rprod / r[n]));
  }
  ly.norm = take(CL);
  ly.flag = take(1);
  ly.Y = take(ymax);
  ly.G = take(rprod);
  ly.cta = cur;
  // per CTA: the gathered slab of mode n (n >= 1) and the chain buffers, whose
  // largest content is the slab after its first contraction (mode p, or p-1
  // when n is the last mode): every later contraction shrinks it
  int64_t slab = 0, chain = 0;
  for (int n = 0; n < p; ++n) {
    const int64_t sl = (xd[n] + CL - 1) / CL * (N / xd[n]);
    if (n > 0) slab = std::max(slab, sl);
    const int m0 = n == p - 1 ? p - 2 : p - 1;
    chain = std::max(chain, sl / xd[m0] * r[m0]);
  }
  cur = 0;
  ly.slab = take(slab);
  ly.b0 = take(chain);
  ly.b1 = take(chain);
  ly.T = take(neig * neig);
  {
    int rmx = 1;
    for (int n = 0; n < p; ++n) rmx = std::max<int>(rmx, (int)r[n]);
    ly.trd = take(tk::trd_scratch_elems((int)neig, rmx, TK_NT / 32));
  }
  ly.nsa = nsa;
  ly.nsv = nsv;
  ly.tc = tc;
  ly.tc_bytes = tc_bytes;
  ly.neig = (int)neig;
  ly.rmax = 1;
  for (int n = 0; n < p; ++n) ly.rmax = std::max<int>(ly.rmax, (int)r[n]);
  ly.half = neig / 2 + 2;
  if (neig > nsv) {
    // some eigenproblem may not fit shared memory: it works in the CTA's global region
    ly.A = take(neig * neig);
    ly.V = take(neig * neig);
    ly.w = take(neig + 2);
    ly.cs = take(2 * ly.half);
    ly.pq = take(ly.half);
  }
  ly.cta_stride = cur + 32;
  *per_cluster = ly.cta + CL * ly.cta_stride;
  return ly;
}

int max_hits(const tk_tree* t, int64_t nbt) {
  const int h = nbt > 0 ? ceil_log2(nbt) + 1 : 1;
  return std::min(TK_MAXH, std::max(2 * (h - 1), 1) + 2);
}

// Largest eig order kept in shared memory for each kernel family.
// One CTA of stitch_warps() warps runs one stitch job at a time; the job
// places its hottest buffers in a shared arena of this many bytes (two CTAs
// per SM) and the rest in its global workspace chunk.
int pick_nsm_stitch(const tk_tree* t) {
  (void)t;
  return 96 * 1024;
}

int stitch_warps(const tk_tree* t) { (void)t; return 8; }

// Shared-memory capacities of the leaf kernel's eigensolvers: the Jacobi
// arrays for orders below the tridiagonal method's, and A (the only n x n
// array of the tridiagonal method) for the largest order that fits next to
// the contraction buffers in a CTA's shared memory.
//
// Grams on the tensor cores (FP32 trees, unless the configuration asks for
// CUDA cores): their staging buffers alias the contraction buffers and get
// what shared memory the eigensolver leaves, up to 64 columns per chunk of
// the largest order; the kernel then asks for at least 116 KB, so that one
// CTA per SM holds tensor memory (a second CTA's allocation would wait).
void pick_nsm_leaf(const tk_tree* t, int* nsa, int* nsv, int* tc, int64_t* tc_bytes) {
  int need = t->cfg.leaf_slices, rmax = 1;
  for (int n = 1; n < t->p; ++n) need = std::max<int>(need, (int)t->cfg.dims[n]);
  for (int n = 0; n < t->p; ++n) rmax = std::max<int>(rmax, t->cfg.ranks[n]);
  rmax = std::min(rmax, need);
  *nsv = std::max(2, std::min(need, tk::kTrdMinOrder - 1));
  const size_t limit = 227 * 1024 - 512;
  const size_t base = tk_leaf_smem_bytes(t->cfg.dtype, 0, *nsv, need, rmax, 0);
  int a = 0;
  if (base < limit) a = (int)std::sqrt((double)(limit - base - 16) / (double)t->es);
  *nsa = std::max(*nsv, std::min(need, a));
  while (*nsa > *nsv && tk_leaf_smem_bytes(t->cfg.dtype, *nsa, *nsv, need, rmax, 0) > limit) --*nsa;
  *tc = 0;
  *tc_bytes = 0;
  if (t->cfg.dtype != TK_F32 || t->cfg.math == TK_MATH_CUDA_CORES) return;
  int dtc = 0;  // largest Gram order on the tensor-core path
  for (int n = 0; n < t->p; ++n) {
    const int d = n == 0 ? t->cfg.leaf_slices : (int)t->cfg.dims[n];
    if (d <= tk::kTcMaxD) dtc = std::max(dtc, d);
  }
  if (dtc == 0) return;
  const size_t with = tk_leaf_smem_bytes(t->cfg.dtype, *nsa, *nsv, need, rmax, 0);
  const size_t rest = with - tk_leaf_contraction_bytes(t->cfg.dtype, need, rmax);
  const int64_t want = (int64_t)4 * 16 * tk::tc_lbo(dtc);  // 64 columns per chunk
  int64_t bytes = std::min<int64_t>(want, (int64_t)limit - (int64_t)rest);
  bytes = std::max<int64_t>(bytes, (int64_t)(116 * 1024) - (int64_t)rest);
  bytes &= ~(int64_t)15;
  if (tk::tc_chunk(dtc, bytes, TK_NT) < 8 || rest + (size_t)bytes > limit) return;
  *tc = t->cfg.math == TK_MATH_TF32 ? 2 : 1;
  *tc_bytes = bytes;
}

// Stitch workspace: one chunk per CTA of the grid.
int ensure_ws_stitch(tk_tree* t, int want_ctas) {
  const int hmax = max_hits(t, t->nbcap);
  const int64_t per = stitch_ws_bound(t, hmax);
  if (t->nsm_stitch == 0) t->nsm_stitch = pick_nsm_stitch(t);
  int ctas = std::max(1, want_ctas);
  if (per != t->ws_stitch_per_cta || ctas > t->ws_stitch_ctas) {
    ctas = std::max(ctas, t->ws_stitch_ctas);
    const int rc = tdalloc(t, t->ws_stitch, (size_t)per * ctas * t->es);
    if (rc) return rc;
    t->ws_stitch_per_cta = per;
    t->ws_stitch_ctas = ctas;
  }
  return TK_OK;
}

// Leaf workspace: one chunk per cluster of the grid.
int ensure_ws_leaf(tk_tree* t, int want_clusters, TkLeafLayout* ly) {
  if (t->nsa_leaf == 0) pick_nsm_leaf(t, &t->nsa_leaf, &t->nsv_leaf, &t->tc_leaf, &t->tc_bytes_leaf);
  int64_t per = 0;
  *ly = leaf_layout(t, t->nsa_leaf, t->nsv_leaf, t->tc_leaf, t->tc_bytes_leaf, &per);
  int n = std::max(1, want_clusters);
  if (per != t->ws_leaf_per_cta || n > t->ws_leaf_ctas) {
    n = std::max(n, t->ws_leaf_ctas);
    const int rc = tdalloc(t, t->ws_leaf, (size_t)per * n * t->es);
    if (rc) return rc;
    t->ws_leaf_per_cta = per;
    t->ws_leaf_ctas = n;
  }
  return TK_OK;
}

// Heavy queries: hit sets of at least heavy_hits() nodes (eigenproblem
// orders >= ~55, a threshold measured on the FP32 plain workload); k_batch
// runs them with a whole CTA.
int heavy_hits(const tk_tree* t) {
  if (t->heavy_set > 0) return t->heavy_set;
  int r = 1;
  for (int n = 0; n < t->p; ++n) r = std::max(r, t->cfg.ranks[n]);
  return std::max(3, (55 + r - 1) / r);
}
// Shared arena of one half of a k_batch CTA (a heavy query gets both
// halves): all the shared memory a block may take, less the two halves'
// headers, split in two.
size_t batch_half_arena(const tk_tree* t) {
  const size_t total = t->smem_optin > 0 ? (size_t)t->smem_optin : 227 * 1024;
  const size_t hdrs = tk_batch_smem_bytes(t->cfg.dtype, 0);
  return ((total - hdrs) / 2) & ~(size_t)127;
}

TkWorkspace ws_view(const tk_tree* t, bool leaf) {
  TkWorkspace w{};
  w.base = leaf ? t->ws_leaf.ptr : t->ws_stitch.ptr;
  w.per_cta = leaf ? t->ws_leaf_per_cta : t->ws_stitch_per_cta;
  w.nsm = 0;
  w.smem_arena = leaf ? 0 : (size_t)t->nsm_stitch;
  w.warps = stitch_warps(t);
  w.status = (int*)t->status.ptr;
  w.counter = (unsigned*)((char*)t->status.ptr + 16);
  return w;
}

// Grid of a stitch launch with njobs jobs: persistent (at most the resident
// CTAs), and no more CTAs than jobs (a stitch CTA runs one job at a time).
int grid_for(tk_tree* t, int njobs) {
  const int dtype = t->cfg.dtype;
  const int warps = stitch_warps(t);
  const size_t smem = tk_stitch_smem_bytes(dtype, (size_t)t->nsm_stitch);
  int occ = tk_occupancy(dtype, smem, 32 * warps);
  if (occ < 1) occ = 1;
  return std::max(1, std::min(njobs, occ * t->sm_count));
}

// Decompose leaf blocks [first, first+njobs) read from raw (block stride in
// elements), each of `ell` slices: one cluster per block, persistent.
int run_leaves(tk_tree* t, const void* raw, int64_t block_stride, int64_t first, int njobs, int ell) {
  if (njobs <= 0) return TK_OK;
  if (t->nsa_leaf == 0) pick_nsm_leaf(t, &t->nsa_leaf, &t->nsv_leaf, &t->tc_leaf, &t->tc_bytes_leaf);
  int64_t per = 0;
  const TkLeafLayout probe = leaf_layout(t, t->nsa_leaf, t->nsv_leaf, t->tc_leaf, t->tc_bytes_leaf, &per);
  int maxc = tk_leaf_max_clusters(t->cfg.dtype, tk_leaf_smem_bytes(t->cfg.dtype, probe.nsa, probe.nsv, probe.neig,
                                                                   probe.rmax, probe.tc_bytes));
  if (maxc < 1) maxc = 1;
  const int ncl = std::min(njobs, maxc);
  TkLeafLayout ly{};
  int rc = ensure_ws_leaf(t, ncl, &ly);
  if (rc) return rc;
  rc = tk_launch_leaf(t->cfg.dtype, make_view(t), raw, block_stride, first, njobs, ell, ws_view(t, true), ly, ncl,
                      t->stream);
  t->launches += 1;
  return rc;
}

int run_merges(tk_tree* t, int level, int64_t k0, int njobs) {
  if (njobs <= 0) return TK_OK;
  if (t->nsm_stitch == 0) t->nsm_stitch = pick_nsm_stitch(t);
  const int grid = grid_for(t, njobs);
  int rc = ensure_ws_stitch(t, grid);
  if (rc) return rc;
  rc = tk_launch_merge(t->cfg.dtype, make_view(t), level, k0, njobs, ws_view(t, false), grid, t->stream);
  t->launches += 1;
  return rc;
}

// Decompose the open block if slices arrived since its last decomposition.
int ensure_tail(tk_tree* t) {
  if (!t->tail_dirty) return TK_OK;
  const int64_t ell = t->T - t->nb * t->cfg.leaf_slices;
  int rc = TK_OK;
  if (ell > 0) rc = run_leaves(t, t->tail_raw.ptr, 0, t->nb, 1, (int)ell);
  if (rc == TK_OK) t->tail_dirty = false;
  return rc;
}

int check_ranks(const tk_tree* t, const int32_t* ranks, int* rq) {
  for (int n = 0; n < TK_MAXP; ++n) rq[n] = 1;
  for (int n = 0; n < t->p; ++n) {
    const int v = ranks ? ranks[n] : t->cfg.ranks[n];
    if (v < 1 || v > t->cfg.ranks[n]) return TK_ERR_RANK;
    rq[n] = v;
  }
  return TK_OK;
}

int64_t out_elems(const tk_tree* t, int64_t L, const int* rq) {
  int64_t c = 1;
  for (int n = 0; n < t->p; ++n) c *= rq[n];
  c += L * rq[0];
  for (int n = 1; n < t->p; ++n) c += t->cfg.dims[n] * rq[n];
  return c;
}

// One batch launch sequence (plan, then the batch kernel; a single query runs alone)
// with all pointers on the device.  Asynchronous on the tree's stream.
int launch_batch(tk_tree* t, int n, const int64_t* d_ranges, const int64_t* d_offsets, const int* rq, void* d_out,
                 tk_query_info* d_info, const int64_t* d_tq = nullptr) {
  int rc = TK_OK;
  if (t->nsm_stitch == 0) t->nsm_stitch = pick_nsm_stitch(t);
  const int grid = grid_for(t, n);
  rc = ensure_ws_stitch(t, grid);
  if (rc) return rc;
  TkQueryBatch qb{};
  qb.n = n;
  qb.ranges = d_ranges;
  qb.offsets = d_offsets;
  qb.out = d_out;
  qb.info = d_info;
  qb.order = nullptr;
  qb.tq = d_tq;
  for (int k = 0; k < TK_MAXP; ++k) qb.rq[k] = rq[k];
  if (n > 1) {
    // Longest-first order (k_plan), then one k_batch launch: a CTA per SM
    // runs the heavy head of the order with all its threads and then the
    // light rest in two halves (see k_batch).
    const int bgrid = std::min(n, t->sm_count);
    const int64_t per = stitch_ws_bound(t, max_hits(t, t->nbcap));
    rc = tdalloc(t, t->plan, sizeof(int) * ((size_t)n + 4));
    if (rc == TK_OK) rc = ensure_ws_stitch(t, 2 * bgrid);
    if (rc) return rc;
    int* split = (int*)t->plan.ptr;
    int* order = split + 4;
    rc = tk_launch_plan(make_view(t), n, d_ranges, d_tq, heavy_hits(t), split, order, t->stream);
    t->launches += 1;
    if (rc) return rc;
    qb.order = order;
    qb.split = split;
    TkWorkspace wb = ws_view(t, false);
    wb.per_cta = per;
    wb.smem_arena = batch_half_arena(t);
    rc = tk_launch_batch(t->cfg.dtype, make_view(t), qb, wb, bgrid, t->stream);
    t->launches += 1;
  } else {
    rc = tk_launch_query(t->cfg.dtype, make_view(t), qb, ws_view(t, false), grid, t->stream);
    t->launches += 1;
  }
  if (rc) return rc;
  return rc;
}

}  // namespace

extern "C" {

const char* tk_strerror(int code) {
  switch (code) {
    case TK_OK: return "ok";
    case TK_ERR_ARG: return "invalid argument";
    case TK_ERR_RANGE: return "time range outside [0, T) or empty";
    case TK_ERR_RANK: return "query rank below 1 or above the build rank";
    case TK_ERR_NOMEM: return "device allocation failed";
    case TK_ERR_CUDA: return "CUDA runtime error";
    case TK_ERR_STATE: return "call not valid in the current tree state";
    case TK_ERR_WORKSPACE: return "device job exceeded its workspace or hit limit";
    case TK_ERR_TOO_BIG: return "request exceeds a fixed engine limit";
    case TK_ERR_TIMEOUT: return "a wait ran out of time";
    case TK_ERR_IO: return "tree file could not be read or written, or is not a tree file";
    default: return "unknown error";
  }
}

int tk_config_default(tk_config* cfg) {
  if (!cfg) return TK_ERR_ARG;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->p = 3;
  for (int n = 0; n < TK_MAX_MODES; ++n) cfg->ranks[n] = 10;
  cfg->leaf_slices = 1;
  cfg->theta_num = 7;
  cfg->theta_den = 10;
  cfg->max_iter = 20;
  cfg->tol = 0.01;
  cfg->dtype = TK_F32;
  cfg->device = 0;
  return TK_OK;
}

int tk_tree_create(const tk_config* cfg, void* cuda_stream, tk_tree** out) {
  if (!cfg || !out) return TK_ERR_ARG;
  *out = nullptr;
  if (cfg->p < 2 || cfg->p > TK_MAX_MODES) return TK_ERR_ARG;
  if (cfg->leaf_slices < 1 || cfg->theta_den < 1 || cfg->theta_num < 1 || cfg->theta_num > cfg->theta_den)
    return TK_ERR_ARG;
  if (cfg->max_iter < 1 || (cfg->dtype != TK_F64 && cfg->dtype != TK_F32)) return TK_ERR_ARG;
  if (cfg->hbm_budget < 0) return TK_ERR_ARG;
  if (cfg->eig_fp64 != 0 && cfg->eig_fp64 != 1) return TK_ERR_ARG;
  if (cfg->init != TK_INIT_HOSVD && cfg->init != TK_INIT_RANDOM) return TK_ERR_ARG;
  if (cfg->math < TK_MATH_AUTO || cfg->math > TK_MATH_TF32 || (cfg->math == TK_MATH_TF32 && cfg->dtype != TK_F32))
    return TK_ERR_ARG;
  for (int n = 0; n < cfg->p; ++n)
    if (cfg->ranks[n] < 1 || cfg->ranks[n] > 4096) return TK_ERR_ARG;
  for (int n = 1; n < cfg->p; ++n)
    if (cfg->dims[n] < 1 || cfg->dims[n] > (1 << 20)) return TK_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
    cudaGetLastError();
    return TK_ERR_CUDA;
  }
  tk_tree* t = new (std::nothrow) tk_tree();
  if (!t) return TK_ERR_NOMEM;
  t->cfg = *cfg;
  t->dev = cfg->device;
  t->p = cfg->p;
  t->es = cfg->dtype == TK_F64 ? 8 : 4;
  DeviceGuard g(t->dev);
  cudaDeviceGetAttribute(&t->sm_count, cudaDevAttrMultiProcessorCount, t->dev);
  cudaDeviceGetAttribute(&t->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, t->dev);
  if (cuda_stream) {
    t->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&t->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete t;
      return TK_ERR_CUDA;
    }
    t->own_stream = true;
  }
  t->slice_elems = 1;
  for (int n = 1; n < t->p; ++n) t->slice_elems *= cfg->dims[n];
  t->core_stride = 1;
  for (int n = 0; n < t->p; ++n) t->core_stride *= cfg->ranks[n];
  for (int n = 1; n < t->p; ++n) t->fac_stride[n] = cfg->dims[n] * cfg->ranks[n];
  int rc = tdalloc(t, t->tail_raw, (size_t)cfg->leaf_slices * t->slice_elems * t->es);
  if (rc == TK_OK) rc = tdalloc(t, t->status, 64);
  if (rc == TK_OK) rc = cuda_ok(cudaMemsetAsync(t->status.ptr, 0, 64, t->stream));
  if (rc == TK_OK) rc = ensure_capacity(t, 1);
  if (rc != TK_OK) {
    tk_tree_destroy(t);
    return rc;
  }
  *out = t;
  return TK_OK;
}

void tk_tree_destroy(tk_tree* t) {
  if (!t) return;
  DeviceGuard g(t->dev);
  if (t->stream) cudaStreamSynchronize(t->stream);
  DevBuf* bufs[] = {&t->core_pool, &t->tfac, &t->node_ranks, &t->tail_raw, &t->ws_stitch, &t->ws_leaf,
                    &t->status, &t->stage_in, &t->stage_out, &t->stage_meta, &t->stage_info, &t->hit_buf,
                    &t->plan};
  for (DevBuf* b : bufs) dfree(*b);
  for (int n = 0; n < TK_MAXP; ++n) dfree(t->fac_pool[n]);
  if (t->own_stream && t->stream) cudaStreamDestroy(t->stream);
  delete t;
}

int64_t tk_timespan(const tk_tree* t) { return t ? t->T : -1; }

int tk_tree_get_config(const tk_tree* t, tk_config* out) {
  if (!t || !out) return TK_ERR_ARG;
  *out = t->cfg;
  return TK_OK;
}
int64_t tk_launch_count(const tk_tree* t) { return t ? t->launches : -1; }

int tk_batch_set_heavy_hits(tk_tree* t, int hits) {
  if (!t || hits < 0) return TK_ERR_ARG;
  t->heavy_set = std::min(hits, TK_MAXH + 1);
  return TK_OK;
}

int tk_batch_get_heavy_hits(const tk_tree* t, int* hits) {
  if (!t || !hits) return TK_ERR_ARG;
  *hits = heavy_hits(t);
  return TK_OK;
}

int64_t tk_arena_bytes(const tk_tree* t) {
  if (!t) return -1;
  int64_t b = t->core_pool.bytes + t->tfac.bytes + t->node_ranks.bytes;
  for (int n = 0; n < TK_MAXP; ++n) b += t->fac_pool[n].bytes;
  return b;
}

int tk_sync(tk_tree* t) {
  if (!t) return TK_ERR_ARG;
  DeviceGuard g(t->dev);
  if (cudaStreamSynchronize(t->stream) != cudaSuccess) return TK_ERR_CUDA;
  int st = 0;
  if (cudaMemcpy(&st, t->status.ptr, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return TK_ERR_CUDA;
  if (st == TK_DEV_ERR_RANGE) return TK_ERR_RANGE;
  if (st != 0) return TK_ERR_WORKSPACE;
  return TK_OK;
}

int tk_tree_build(tk_tree* t, const void* X, int64_t T, int io) {
  if (!t || !X || T < 1 || (io != TK_IO_DEVICE && io != TK_IO_HOST)) return TK_ERR_ARG;
  if (t->T != 0) return TK_ERR_STATE;
  if (io == TK_IO_DEVICE && !on_device(X, t->dev)) return TK_ERR_ARG;
  DeviceGuard g(t->dev);
  const int B = t->cfg.leaf_slices;
  const int64_t nb = T / B, nbt = (T + B - 1) / B;
  int rc = ensure_capacity(t, nbt);
  if (rc) return rc;
  const void* Xd = X;
  DevBuf tmp;
  if (io == TK_IO_HOST) {
    rc = tdalloc(t, tmp, (size_t)T * t->slice_elems * t->es);
    if (rc) return rc;
    rc = cuda_ok(cudaMemcpyAsync(tmp.ptr, X, tmp.bytes, cudaMemcpyHostToDevice, t->stream));
    if (rc) {
      dfree(tmp);
      return rc;
    }
    Xd = tmp.ptr;
  }
  // complete leaf blocks, then each level of intermediate nodes
  t->T = nb * B;
  t->nb = nb;
  rc = run_leaves(t, Xd, (int64_t)B * t->slice_elems, 0, (int)nb, B);
  for (int j = 1; rc == TK_OK; ++j) {
    const int64_t cnt = nb >> j;
    if (cnt <= 0) break;
    rc = run_merges(t, j, 0, (int)cnt);
  }
  // open tail block
  if (rc == TK_OK && T > nb * B) {
    const int64_t ell = T - nb * B;
    rc = cuda_ok(cudaMemcpyAsync(t->tail_raw.ptr, (const char*)Xd + (size_t)nb * B * t->slice_elems * t->es,
                                 (size_t)ell * t->slice_elems * t->es, cudaMemcpyDeviceToDevice, t->stream));
    t->T = T;
    t->tail_dirty = true;
  }
  if (tmp.ptr) {
    cudaStreamSynchronize(t->stream);
    dfree(tmp);
  }
  return rc;
}

int tk_stream_append(tk_tree* t, const void* slice, int io) {
  if (!t || !slice || (io != TK_IO_DEVICE && io != TK_IO_HOST)) return TK_ERR_ARG;
  if (io == TK_IO_DEVICE && !on_device(slice, t->dev)) return TK_ERR_ARG;
  DeviceGuard g(t->dev);
  const int B = t->cfg.leaf_slices;
  int rc = ensure_capacity(t, (t->T + 1 + B - 1) / B);
  if (rc) return rc;
  const int64_t off = t->T - t->nb * B;
  char* dst = (char*)t->tail_raw.ptr + (size_t)off * t->slice_elems * t->es;
  rc = cuda_ok(cudaMemcpyAsync(dst, slice, (size_t)t->slice_elems * t->es,
                               io == TK_IO_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, t->stream));
  if (rc) return rc;
  if (io == TK_IO_HOST) cudaStreamSynchronize(t->stream);  // the caller may reuse its host buffer
  t->T += 1;
  if (off + 1 == B) {
    // Algorithm 3: the leaf completes, then every ancestor whose range ends here is stitched
    t->tail_dirty = false;
    rc = run_leaves(t, t->tail_raw.ptr, 0, t->nb, 1, B);
    t->nb += 1;
    for (int j = 1; rc == TK_OK; ++j) {
      if (t->nb % ((int64_t)1 << j) != 0) break;
      rc = run_merges(t, j, (t->nb >> j) - 1, 1);
    }
  } else {
    t->tail_dirty = true;
  }
  return rc;
}

int tk_hit_set(tk_tree* t, int64_t t_s, int64_t t_e, tk_hit* out, int cap, int* n_out) {
  if (!t || !out || !n_out || cap < 1) return TK_ERR_ARG;
  if (!(t_s >= 0 && t_s < t_e && t_e <= t->T)) return TK_ERR_RANGE;
  DeviceGuard g(t->dev);
  const size_t need = 64 + sizeof(int64_t) * 2 + sizeof(tk_hit) * TK_MAXH;
  int rc = tdalloc(t, t->hit_buf, need);
  if (rc) return rc;
  int64_t rng[2] = {t_s, t_e};
  char* base = (char*)t->hit_buf.ptr;
  int* counts = (int*)base;
  int64_t* dr = (int64_t*)(base + 16);
  tk_hit* dh = (tk_hit*)(base + 64);
  rc = cuda_ok(cudaMemcpyAsync(dr, rng, sizeof(rng), cudaMemcpyHostToDevice, t->stream));
  if (rc) return rc;
  rc = tk_launch_hitset(make_view(t), 1, dr, dh, TK_MAXH, counts, t->stream);
  t->launches += 1;
  if (rc) return rc;
  int cnt = 0;
  std::vector<tk_hit> h(TK_MAXH);
  rc = cuda_ok(cudaMemcpyAsync(&cnt, counts, sizeof(int), cudaMemcpyDeviceToHost, t->stream));
  if (rc == TK_OK) rc = cuda_ok(cudaMemcpyAsync(h.data(), dh, sizeof(tk_hit) * TK_MAXH, cudaMemcpyDeviceToHost, t->stream));
  if (rc == TK_OK) rc = cuda_ok(cudaStreamSynchronize(t->stream));
  if (rc) return rc;
  if (cnt < 0) return TK_ERR_TOO_BIG;
  *n_out = cnt;
  if (cnt > cap) return TK_ERR_TOO_BIG;
  std::memcpy(out, h.data(), sizeof(tk_hit) * cnt);
  return TK_OK;
}

int64_t tk_query_output_elems(const tk_tree* t, int64_t t_s, int64_t t_e, const int32_t* ranks) {
  if (!t) return TK_ERR_ARG;
  if (!(t_s >= 0 && t_s < t_e)) return TK_ERR_RANGE;
  int rq[TK_MAXP];
  const int rc = check_ranks(t, ranks, rq);
  if (rc) return rc;
  return out_elems(t, t_e - t_s, rq);
}

int tk_batch_layout(const tk_tree* t, int n, const int64_t* ranges, const int32_t* ranks, int64_t* offsets) {
  if (!t || n < 0 || (n > 0 && (!ranges || !offsets))) return TK_ERR_ARG;
  int rq[TK_MAXP];
  const int rc = check_ranks(t, ranks, rq);
  if (rc) return rc;
  offsets[0] = 0;
  for (int i = 0; i < n; ++i) {
    const int64_t ts = ranges[2 * i], te = ranges[2 * i + 1];
    if (!(ts >= 0 && ts < te)) return TK_ERR_RANGE;
    offsets[i + 1] = offsets[i] + out_elems(t, te - ts, rq);
  }
  return TK_OK;
}

int tk_range_query_batch(tk_tree* t, int n, const int64_t* ranges, const int64_t* offsets, const int32_t* ranks,
                         void* out, tk_query_info* info, int io) {
  if (!t || n < 0) return TK_ERR_ARG;
  if (n == 0) return TK_OK;
  if (!ranges || !offsets || !out || (io != TK_IO_DEVICE && io != TK_IO_HOST)) return TK_ERR_ARG;
  if (io == TK_IO_DEVICE &&
      !(on_device(ranges, t->dev) && on_device(offsets, t->dev) && on_device(out, t->dev)))
    return TK_ERR_ARG;
  DeviceGuard g(t->dev);
  int rq[TK_MAXP];
  int rc = check_ranks(t, ranks, rq);
  if (rc) return rc;
  if (t->T == 0) return TK_ERR_RANGE;
  if (io == TK_IO_HOST) {
    for (int i = 0; i < n; ++i)
      if (!(ranges[2 * i] >= 0 && ranges[2 * i] < ranges[2 * i + 1] && ranges[2 * i + 1] <= t->T)) return TK_ERR_RANGE;
  }
  rc = ensure_tail(t);
  if (rc) return rc;
  const int64_t* d_ranges = ranges;
  const int64_t* d_offsets = offsets;
  void* d_out = out;
  if (io == TK_IO_HOST) {
    const size_t meta = sizeof(int64_t) * (2 * (size_t)n + n + 1);
    rc = tdalloc(t, t->stage_meta, meta);
    if (rc) return rc;
    rc = tdalloc(t, t->stage_out, (size_t)offsets[n] * t->es);
    if (rc) return rc;
    int64_t* m = (int64_t*)t->stage_meta.ptr;
    rc = cuda_ok(cudaMemcpyAsync(m, ranges, sizeof(int64_t) * 2 * n, cudaMemcpyHostToDevice, t->stream));
    if (rc == TK_OK)
      rc = cuda_ok(cudaMemcpyAsync(m + 2 * n, offsets, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, t->stream));
    if (rc) return rc;
    d_ranges = m;
    d_offsets = m + 2 * n;
    d_out = t->stage_out.ptr;
  }
  tk_query_info* d_info = nullptr;
  if (info) {
    rc = tdalloc(t, t->stage_info, sizeof(tk_query_info) * n);
    if (rc) return rc;
    d_info = (tk_query_info*)t->stage_info.ptr;
  }
  rc = launch_batch(t, n, d_ranges, d_offsets, rq, d_out, d_info);
  if (rc) return rc;
  if (io == TK_IO_HOST) {
    rc = cuda_ok(cudaMemcpyAsync(out, d_out, (size_t)offsets[n] * t->es, cudaMemcpyDeviceToHost, t->stream));
    if (rc) return rc;
  }
  if (info) {
    rc = cuda_ok(cudaMemcpyAsync(info, d_info, sizeof(tk_query_info) * n, cudaMemcpyDeviceToHost, t->stream));
    if (rc) return rc;
  }
  if (io == TK_IO_HOST || info) {
    rc = tk_sync(t);
    if (rc) return rc;
  }
  return TK_OK;
}

int tk_batch_tune(tk_tree* t, int n, const int64_t* ranges, const int64_t* offsets, const int32_t* ranks, void* out,
                  int reps, int* best_hits, float* best_ms) {
  if (!t || n < 1 || reps < 1 || !best_hits || !ranges || !offsets || !out) return TK_ERR_ARG;
  if (!(on_device(ranges, t->dev) && on_device(offsets, t->dev) && on_device(out, t->dev))) return TK_ERR_ARG;
  DeviceGuard g(t->dev);
  if (best_ms) *best_ms = -1.f;
  if (n == 1) {  // a single query runs on one CTA whatever the threshold
    *best_hits = heavy_hits(t);
    return TK_OK;
  }
  // Candidates in increasing order; one above the kernel's hit limit runs
  // every query on a half CTA.  A candidate that selects the same heavy head
  // as the previous one is the same launch and is not timed again.
  static const int cand[] = {3, 4, 5, 6, 7, 8, 10, 12, 16, 24, 32, TK_MAXH + 1};
  const int saved = t->heavy_set;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = cuda_ok(cudaEventCreate(&e0));
  if (rc == TK_OK) rc = cuda_ok(cudaEventCreate(&e1));
  int prev_split = -1, best_c = heavy_hits(t);
  float best = 0.f;
  bool have = false;
  for (int ci = 0; rc == TK_OK && ci < (int)(sizeof(cand) / sizeof(cand[0])); ++ci) {
    t->heavy_set = cand[ci];
    rc = tk_range_query_batch(t, n, ranges, offsets, ranks, out, nullptr, TK_IO_DEVICE);  // warm-up
    if (rc == TK_OK) rc = tk_sync(t);
    int split = 0;
    if (rc == TK_OK) rc = cuda_ok(cudaMemcpy(&split, t->plan.ptr, sizeof(int), cudaMemcpyDeviceToHost));
    if (rc || split == prev_split) continue;
    prev_split = split;
    float ms = 0.f;
    for (int r = 0; rc == TK_OK && r < reps; ++r) {
      rc = cuda_ok(cudaEventRecord(e0, t->stream));
      if (rc == TK_OK) rc = tk_range_query_batch(t, n, ranges, offsets, ranks, out, nullptr, TK_IO_DEVICE);
      if (rc == TK_OK) rc = cuda_ok(cudaEventRecord(e1, t->stream));
      if (rc == TK_OK) rc = tk_sync(t);
      float m = 0.f;
      if (rc == TK_OK) rc = cuda_ok(cudaEventElapsedTime(&m, e0, e1));
      if (rc == TK_OK && (r == 0 || m < ms)) ms = m;
    }
    if (rc == TK_OK && (!have || ms < best)) {
      best = ms;
      best_c = cand[ci];
      have = true;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc) {
    t->heavy_set = saved;
    return rc;
  }
  t->heavy_set = best_c;
  *best_hits = best_c;
  if (best_ms) *best_ms = best;
  return TK_OK;
}

}  // extern "C"

// Batched queries with every pointer on the device, reports included;
// asynchronous.  Used by the serving runtime (tk_server.cu).  d_tq (device, n,
// may be null) gives the T each query is answered at; the open block is
// decomposed first only when need_tail is set (some query reaches into the
// current open block).
int tk_query_batch_device(tk_tree* t, int n, const int64_t* d_ranges, const int64_t* d_offsets,
                          const int32_t* ranks, void* d_out, tk_query_info* d_info, const int64_t* d_tq,
                          bool need_tail) {
  if (!t || n < 0) return TK_ERR_ARG;
  if (n == 0) return TK_OK;
  DeviceGuard g(t->dev);
  int rq[TK_MAXP];
  int rc = check_ranks(t, ranks, rq);
  if (rc) return rc;
  if (t->T == 0) return TK_ERR_RANGE;
  if (need_tail) {
    rc = ensure_tail(t);
    if (rc) return rc;
  }
  return launch_batch(t, n, d_ranges, d_offsets, rq, d_out, d_info, d_tq);
}

cudaStream_t tk_tree_stream(const tk_tree* t) { return t->stream; }
int tk_tree_device(const tk_tree* t) { return t->dev; }
size_t tk_tree_elem_size(const tk_tree* t) { return t->es; }

extern "C" {

int tk_range_query(tk_tree* t, int64_t t_s, int64_t t_e, const int32_t* ranks, void* out, tk_query_info* info,
                   int io) {
  if (!t || !out || (io != TK_IO_DEVICE && io != TK_IO_HOST)) return TK_ERR_ARG;
  if (!(t_s >= 0 && t_s < t_e && t_e <= t->T)) return TK_ERR_RANGE;
  int rq[TK_MAXP];
  int rc = check_ranks(t, ranks, rq);
  if (rc) return rc;
  int64_t rng[2] = {t_s, t_e};
  int64_t offs[2] = {0, out_elems(t, t_e - t_s, rq)};
  DeviceGuard g(t->dev);
  if (io == TK_IO_HOST) return tk_range_query_batch(t, 1, rng, offs, ranks, out, info, TK_IO_HOST);
  // device output: the two small arrays go through the metadata staging buffer
  rc = tdalloc(t, t->stage_meta, std::max<size_t>(t->stage_meta.bytes, sizeof(int64_t) * 4));
  if (rc) return rc;
  int64_t* m = (int64_t*)t->stage_meta.ptr;
  int64_t hm[4] = {t_s, t_e, 0, offs[1]};
  rc = cuda_ok(cudaMemcpyAsync(m, hm, sizeof(hm), cudaMemcpyHostToDevice, t->stream));
  if (rc) return rc;
  // the host array must outlive the async copy
  rc = cuda_ok(cudaStreamSynchronize(t->stream));
  if (rc) return rc;
  return tk_range_query_batch(t, 1, m, m + 2, ranks, out, info, TK_IO_DEVICE);
}

int tk_node_payload(tk_tree* t, int level, int64_t index, void* out_host, int64_t out_elems_cap, int32_t* ranks_out) {
  if (!t || !out_host || level < 0 || index < 0) return TK_ERR_ARG;
  DeviceGuard g(t->dev);
  int rc = ensure_tail(t);
  if (rc) return rc;
  const int B = t->cfg.leaf_slices;
  const int64_t nbt = nbt_of(t);
  const bool complete = ((index + 1) << level) <= t->nb;
  const bool tail = level == 0 && index == t->nb && t->T > t->nb * B;
  if (!complete && !tail) return TK_ERR_RANGE;
  (void)nbt;
  const int64_t lo = (index << level) * B;
  const int64_t hi = std::min<int64_t>(lo + ((int64_t)1 << level) * B, t->T);
  const int* r = t->cfg.ranks;
  int rq[TK_MAXP];
  for (int n = 0; n < TK_MAXP; ++n) rq[n] = n < t->p ? r[n] : 1;
  const int64_t need = out_elems(t, hi - lo, rq);
  if (out_elems_cap < need) return TK_ERR_ARG;
  const int64_t slot = t->level_base[level] + index;
  char* o = (char*)out_host;
  const size_t es = t->es;
  rc = cuda_ok(cudaMemcpyAsync(o, (char*)t->core_pool.ptr + slot * t->core_stride * es, t->core_stride * es,
                               cudaMemcpyDeviceToHost, t->stream));
  o += t->core_stride * es;
  const int64_t Tcap = t->nbcap * B;
  if (rc == TK_OK)
    rc = cuda_ok(cudaMemcpyAsync(o, (char*)t->tfac.ptr + ((size_t)level * Tcap + lo) * r[0] * es,
                                 (size_t)(hi - lo) * r[0] * es, cudaMemcpyDeviceToHost, t->stream));
  o += (size_t)(hi - lo) * r[0] * es;
  for (int n = 1; n < t->p && rc == TK_OK; ++n) {
    rc = cuda_ok(cudaMemcpyAsync(o, (char*)t->fac_pool[n].ptr + slot * t->fac_stride[n] * es,
                                 t->fac_stride[n] * es, cudaMemcpyDeviceToHost, t->stream));
    o += t->fac_stride[n] * es;
  }
  int nr[TK_MAXP];
  if (rc == TK_OK)
    rc = cuda_ok(cudaMemcpyAsync(nr, (char*)t->node_ranks.ptr + slot * TK_MAXP * sizeof(int), sizeof(nr),
                                 cudaMemcpyDeviceToHost, t->stream));
  if (rc == TK_OK) rc = tk_sync(t);
  if (rc == TK_OK && ranks_out)
    for (int n = 0; n < TK_MAXP; ++n) ranks_out[n] = nr[n];
  return rc;
}

}  // extern "C"

// ---- Allocation-free batched range queries ---------------------------------
// The scratch of tk_range_query_batch_noalloc: a fixed device array instead of
// the tree's allocated workspaces.  Layout per call: [0, 256) the job
// counter, then the optional per-query reports, then one workspace chunk per
// CTA.
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[TK_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
struct NoAllocDevice {
  std::once_flag once;
  void* ptr = nullptr;   // device address of g_noalloc_scratch on this device
  int rc = TK_ERR_CUDA;
};
NoAllocDevice g_noalloc_dev[kMaxDevices];

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" int tk_range_query_batch_noalloc(tk_tree* t, int n, const int64_t* ranges_dev,
                                            const int64_t* offsets_dev, const int32_t* ranks, void* out_dev,
                                            tk_query_info* info) {
  if (!t || n < 1 || !ranges_dev || !offsets_dev || !out_dev) return TK_ERR_ARG;
  if (t->dev < 0 || t->dev >= kMaxDevices) return TK_ERR_ARG;
  if (!(on_device(ranges_dev, t->dev) && on_device(offsets_dev, t->dev) && on_device(out_dev, t->dev)))
    return TK_ERR_ARG;
  int rq[TK_MAXP];
  int rc = check_ranks(t, ranks, rq);
  if (rc) return rc;
  // the open block would need the leaf kernel (and its workspace) first
  if (t->tail_dirty && t->T > t->nb * t->cfg.leaf_slices) return TK_ERR_STATE;
  DeviceGuard g(t->dev);
  // set-up, once per device, with the tree's device current
  NoAllocDevice& d = g_noalloc_dev[t->dev];
  std::call_once(d.once, [&d] {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    d.ptr = p;
    d.rc = (e == cudaSuccess && p != nullptr) ? TK_OK : TK_ERR_CUDA;
  });
  if (d.rc != TK_OK) return d.rc;
  // size check: one query's workspace must fit next to the status word and reports
  if (t->nsm_stitch == 0) t->nsm_stitch = pick_nsm_stitch(t);
  const int64_t per_cta = stitch_ws_bound(t, max_hits(t, t->nbcap));
  const size_t per_cta_bytes = round256((size_t)per_cta * t->es);
  const size_t info_bytes = info ? round256(sizeof(tk_query_info) * (size_t)n) : 0;
  const size_t head = 256 + info_bytes;
  if (head + per_cta_bytes > TK_NOALLOC_SCRATCH_BYTES) return TK_ERR_TOO_BIG;
  if (t->T == 0) return TK_ERR_RANGE;
  const int warps = stitch_warps(t);
  const int fit = (int)std::min<size_t>((TK_NOALLOC_SCRATCH_BYTES - head) / per_cta_bytes, 1 << 20);
  const int grid = std::max(1, std::min(grid_for(t, n), fit));
  char* base = (char*)d.ptr;
  TkWorkspace ws{};
  ws.base = base + head;
  ws.per_cta = (int64_t)(per_cta_bytes / t->es);
  ws.nsm = 0;
  ws.smem_arena = (size_t)t->nsm_stitch;
  ws.warps = warps;
  // device-side errors go to the tree's own sticky status word (allocated at
  // tk_tree_create), so that tk_sync reports them after an asynchronous call;
  // the job counter (zeroed by the launcher) lives in the scratch array
  ws.status = (int*)t->status.ptr;
  ws.counter = (unsigned*)(base + 64);
  TkQueryBatch qb{};
  qb.n = n;
  qb.ranges = ranges_dev;
  qb.offsets = offsets_dev;
  qb.out = out_dev;
  qb.info = info ? (tk_query_info*)(base + 256) : nullptr;
  for (int k = 0; k < TK_MAXP; ++k) qb.rq[k] = rq[k];
  rc = tk_launch_query(t->cfg.dtype, make_view(t), qb, ws, grid, t->stream);
  t->launches += 1;
  if (rc) return rc;
  if (!info) return TK_OK;
  rc = cuda_ok(cudaMemcpyAsync(info, base + 256, sizeof(tk_query_info) * (size_t)n, cudaMemcpyDeviceToHost,
                               t->stream));
  if (rc) return rc;
  return tk_sync(t);
}

// ---- Tree files --------------------------------------------------------------
// A saved tree is its configuration and time span followed by the device
// buffers that hold its state, byte for byte: the node arena (cores, the
// non-temporal factors of every mode, the temporal factor rows of every level,
// the node ranks) and the raw slices of the open leaf block.  The arena layout
// is a function of the block capacity alone, so a tree created with the saved
// configuration and grown to the saved capacity has buffers of the same sizes
// and layout, and copying the bytes back restores the tree exactly.
namespace {

constexpr char kFileMagic[8] = {'T', 'K', 'T', 'R', 'E', 'E', '\0', '\3'};
constexpr int kFileSections = 4 + TK_MAXP;

struct TkFileHeader {
  char magic[8];
  uint32_t header_bytes;  // sizeof(TkFileHeader): catches a different build of this struct
  uint32_t elem_bytes;    // 4 or 8
  tk_config cfg;
  int64_t T, nb, nbcap;
  int32_t tail_dirty;
  int32_t nsec;
  int64_t sec_bytes[kFileSections];
};

// The buffers of a file, in file order: core pool, temporal factor rows, node
// ranks, open-block slices, then the factor pool of each mode (mode 0 and the
// modes beyond p have none: zero bytes).
void file_sections(tk_tree* t, DevBuf** s) {
  s[0] = &t->core_pool;
  s[1] = &t->tfac;
  s[2] = &t->node_ranks;
  s[3] = &t->tail_raw;
  for (int n = 0; n < TK_MAXP; ++n) s[4 + n] = &t->fac_pool[n];
}

constexpr size_t kFileChunk = (size_t)64 << 20;

int section_out(tk_tree* t, const DevBuf& b, FILE* f, std::vector<char>& stage) {
  for (size_t done = 0; done < b.bytes;) {
    const size_t c = std::min(stage.size(), b.bytes - done);
    if (cudaMemcpyAsync(stage.data(), (const char*)b.ptr + done, c, cudaMemcpyDeviceToHost, t->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(t->stream) != cudaSuccess)
      return TK_ERR_CUDA;
    if (std::fwrite(stage.data(), 1, c, f) != c) return TK_ERR_IO;
    done += c;
  }
  return TK_OK;
}

int section_in(tk_tree* t, DevBuf& b, FILE* f, std::vector<char>& stage) {
  for (size_t done = 0; done < b.bytes;) {
    const size_t c = std::min(stage.size(), b.bytes - done);
    if (std::fread(stage.data(), 1, c, f) != c) return TK_ERR_IO;
    if (cudaMemcpyAsync((char*)b.ptr + done, stage.data(), c, cudaMemcpyHostToDevice, t->stream) != cudaSuccess ||
        cudaStreamSynchronize(t->stream) != cudaSuccess)
      return TK_ERR_CUDA;
    done += c;
  }
  return TK_OK;
}

// Header fields that must hold before any device work.
bool header_plausible(const TkFileHeader& h) {
  if (std::memcmp(h.magic, kFileMagic, sizeof(kFileMagic)) != 0) return false;
  if (h.header_bytes != sizeof(TkFileHeader) || h.nsec != kFileSections) return false;
  if (h.cfg.dtype != TK_F64 && h.cfg.dtype != TK_F32) return false;
  if (h.elem_bytes != (h.cfg.dtype == TK_F64 ? 8u : 4u)) return false;
  const int64_t B = h.cfg.leaf_slices;
  if (B < 1 || h.T < 0 || h.nb != h.T / B) return false;
  if (h.nbcap < 1 || (h.nbcap & (h.nbcap - 1)) != 0 || h.nbcap < (h.T + B - 1) / B) return false;
  if (h.tail_dirty != 0 && h.tail_dirty != 1) return false;
  for (int i = 0; i < kFileSections; ++i)
    if (h.sec_bytes[i] < 0) return false;
  return true;
}

}  // namespace

extern "C" int tk_tree_save(tk_tree* t, const char* path) {
  if (!t || !path) return TK_ERR_ARG;
  DeviceGuard g(t->dev);
  int rc = tk_sync(t);  // pending work first; a device-side error is reported, nothing is written
  if (rc) return rc;
  TkFileHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, kFileMagic, sizeof(kFileMagic));
  h.header_bytes = sizeof(TkFileHeader);
  h.elem_bytes = (uint32_t)t->es;
  h.cfg = t->cfg;
  h.T = t->T;
  h.nb = t->nb;
  h.nbcap = t->nbcap;
  h.tail_dirty = t->tail_dirty ? 1 : 0;
  h.nsec = kFileSections;
  DevBuf* s[kFileSections];
  file_sections(t, s);
  size_t largest = 0;
  for (int i = 0; i < kFileSections; ++i) {
    h.sec_bytes[i] = (int64_t)s[i]->bytes;
    largest = std::max(largest, s[i]->bytes);
  }
  FILE* f = std::fopen(path, "wb");
  if (!f) return TK_ERR_IO;
  std::vector<char> stage;
  try {
    stage.resize(std::max<size_t>(1, std::min(largest, kFileChunk)));
  } catch (...) {
    std::fclose(f);
    return TK_ERR_NOMEM;
  }
  rc = std::fwrite(&h, sizeof(h), 1, f) == 1 ? TK_OK : TK_ERR_IO;
  for (int i = 0; i < kFileSections && rc == TK_OK; ++i) rc = section_out(t, *s[i], f, stage);
  if (std::fclose(f) != 0 && rc == TK_OK) rc = TK_ERR_IO;
  return rc;
}

extern "C" int tk_tree_load(const char* path, int device, void* cuda_stream, tk_tree** out) {
  if (!path || !out) return TK_ERR_ARG;
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return TK_ERR_IO;
  TkFileHeader h;
  if (std::fread(&h, sizeof(h), 1, f) != 1 || !header_plausible(h)) {
    std::fclose(f);
    return TK_ERR_IO;
  }
  tk_config cfg = h.cfg;
  if (device >= 0) cfg.device = device;
  tk_tree* t = nullptr;
  int rc = tk_tree_create(&cfg, cuda_stream, &t);
  if (rc) {
    std::fclose(f);
    return rc;
  }
  {
    DeviceGuard g(t->dev);
    rc = ensure_capacity(t, h.nbcap);
    if (rc == TK_OK && t->nbcap != h.nbcap) rc = TK_ERR_IO;
    DevBuf* s[kFileSections];
    file_sections(t, s);
    size_t largest = 0;
    for (int i = 0; i < kFileSections && rc == TK_OK; ++i) {
      if ((int64_t)s[i]->bytes != h.sec_bytes[i]) rc = TK_ERR_IO;
      largest = std::max(largest, s[i]->bytes);
    }
    std::vector<char> stage;
    if (rc == TK_OK) {
      try {
        stage.resize(std::max<size_t>(1, std::min(largest, kFileChunk)));
      } catch (...) {
        rc = TK_ERR_NOMEM;
      }
    }
    for (int i = 0; i < kFileSections && rc == TK_OK; ++i) rc = section_in(t, *s[i], f, stage);
    if (rc == TK_OK && std::fgetc(f) != EOF) rc = TK_ERR_IO;  // trailing bytes: not a file of this tree
  }
  std::fclose(f);
  if (rc) {
    tk_tree_destroy(t);
    return rc;
  }
  t->T = h.T;
  t->nb = h.nb;
  t->tail_dirty = h.tail_dirty != 0;
  *out = t;
  return TK_OK;
}
