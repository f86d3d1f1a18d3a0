// Leaf-block kernel: Tucker-ALS (Section 2: Eq. (tuckerals), Eq. (als-mat))
// of the raw B x D_2 x ... x D_p block of a leaf (Algorithm 3 decomposes a
// new leaf from its raw slices), and of the open tail block.
//
// One thread-block cluster of TK_LEAF_CL CTAs decomposes one block.  The
// expensive steps are contractions over the raw block:
//   * the HOSVD start's Grams mat_n(X) mat_n(X)^T, n >= 2, split by columns
//     over the CTAs (each CTA writes a partial Gram, the partials are summed
//     in CTA order);
//   * per ALS iteration and mode, Y_n = X x_{m != n} U_m^T, split by the
//     mode-n index: each CTA contracts its slab of X and owns whole rows of
//     mat_n(Y_n).
// The small steps -- the Gram of mat_n(Y_n) (D_n x prod_{m!=n} r_m), its
// eigendecomposition, the core G = Y_p x_p U_p^T and the stop test -- run on
// the cluster's first CTA; the p-1 eigendecompositions of the HOSVD start run
// on p-1 CTAs at once.  Hardware cluster barriers separate the steps.
//
// The arithmetic of every stored value depends on the cluster size only, not
// on how many blocks a launch decomposes, so tree build and appends store the
// same bits.
#include <algorithm>
#include <type_traits>

#include "tk_device.cuh"
#include "tk_internal.h"
#include "tk_tc.cuh"

namespace tk {

namespace {

constexpr int kHdr = 1024;  // bytes of the shared header
constexpr int kKC = 32;    // Gram columns staged in shared memory at a time
constexpr int kStage = 16 * TK_NT;  // elements of the staging buffer of a contraction

template <class S> struct LeafSm {
  S red[40];
  S sc[4];
  int flag;
  int nsw;
  S thr;
  S xn2;
  int cl[64];
};

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_id() {
  unsigned r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned num_clusters() {
  unsigned r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}

// Barrier of all threads of the cluster.  Global-memory writes made before it
// by any CTA of the cluster are visible to every CTA after it (the arrive has
// release and the wait acquire semantics at cluster scope; the fence extends
// the release to the global writes of every thread).
__device__ __forceinline__ void cluster_barrier() {
  __threadfence();
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void ld4(const float* p, float* o) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x;
  o[1] = v.y;
  o[2] = v.z;
  o[3] = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double* o) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  const double2 w = *reinterpret_cast<const double2*>(p + 2);
  o[0] = v.x;
  o[1] = v.y;
  o[2] = w.x;
  o[3] = w.y;
}

__device__ __forceinline__ int64_t prod64(const int* d, int a, int b) {
  int64_t p = 1;
  for (int m = a; m < b; ++m) p *= d[m];
  return p;
}

// A (D x D, leading dimension lda) <- sum over the columns c in [c0, c1) of
// x_c x_c^T, where the columns are those of the mode-n matricization of a
// C-order tensor seen as (outer, D, inner): x_c[a] = X[(o D + a) inner + i],
// c = o inner + i.  One CTA: kKC columns at a time are staged in shared
// memory (`tile`, kKC * (round4(D) + 4) elements, 16-byte aligned) and every thread
// accumulates 4x4 blocks of the upper triangle, mirrored on output.  The
// loads of the next kKC columns are issued into registers before the current
// ones are used, so their latency overlaps the arithmetic.  Every entry sums
// its columns in increasing order.
template <class S>
__device__ void gram_cols(const S* X, int D, int64_t inner, int64_t c0, int64_t c1, S* A, int lda, S* tile) {
  constexpr int MT = 2;
  // staged elements per thread and tile (the register prefetch is used for
  // float only: in double it would spill, and the double path is not hot)
  constexpr int PF = sizeof(S) == 4 ? 20 : 1;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  // tile row length: D rounded to 4 for the float4 reads, plus 4 so that the
  // column-per-lane stores of the inner > 1 path spread over 8 banks, not 1
  const int ld = ((D + 3) & ~3) + 4;
  const int nb4 = ((D + 3) & ~3) / 4;
  const int ntile = nb4 * (nb4 + 1) / 2;
  const int per = (kKC * ld + nt - 1) / nt;  // staged elements per thread
  const bool fits = sizeof(S) == 4 && per <= PF;
  // staging map (fixed for every tile): element u of this thread is (kk[u], a[u])
  int skk[PF], sa[PF];
#pragma unroll
  for (int u = 0; u < PF; ++u) {
    if (inner == 1) {
      const int e = tid + u * nt;
      skk[u] = e / ld;
      sa[u] = e - skk[u] * ld;
    } else {
      skk[u] = lane;
      sa[u] = warp + u * nw;
    }
  }
  auto fetch = [&](int64_t c, int kc, S* v) {
    if (inner == 1) {
#pragma unroll
      for (int u = 0; u < PF; ++u)
        v[u] = (u < per && skk[u] < kc && sa[u] < D) ? X[(c + skk[u]) * D + sa[u]] : S(0);
    } else {
      const int64_t col = c + lane;
      const int64_t o = col / inner, i = col - o * inner;
      const S* xp = X + o * D * inner + i;
#pragma unroll
      for (int u = 0; u < PF; ++u) v[u] = (u < per && lane < kc && sa[u] < D) ? xp[(int64_t)sa[u] * inner] : S(0);
    }
  };
  for (int pass0 = 0; pass0 < ntile; pass0 += nt * MT) {
    int I[MT], J[MT];
    bool act[MT];
#pragma unroll
    for (int u = 0; u < MT; ++u) {
      int q = pass0 + u * nt + tid;
      act[u] = q < ntile;
      int a = 0;
      if (act[u])
        while (q >= nb4 - a) {
          q -= nb4 - a;
          ++a;
        }
      I[u] = a;
      J[u] = act[u] ? a + q : a;
    }
    S acc[MT][4][4];
#pragma unroll
    for (int u = 0; u < MT; ++u)
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[u][x][y] = S(0);
    S v[PF];
    if (fits && c0 < c1) fetch(c0, (int)((c1 - c0) < kKC ? (c1 - c0) : kKC), v);
    for (int64_t c = c0; c < c1; c += kKC) {
      const int kc = (int)((c1 - c) < kKC ? (c1 - c) : kKC);
      __syncthreads();  // the previous tile has been consumed
      if (fits) {
#pragma unroll
        for (int u = 0; u < PF; ++u)
          if (u < per && skk[u] < kKC && sa[u] < ld) tile[skk[u] * ld + sa[u]] = v[u];
      } else if (inner == 1) {  // a column is D contiguous elements
        for (int kk = warp; kk < kc; kk += nw) {
          const S* xp = X + (c + kk) * D;
          for (int a = lane; a < ld; a += 32) tile[kk * ld + a] = a < D ? xp[a] : S(0);
        }
      } else {  // lane = column: consecutive columns are consecutive addresses within a row
        if (lane < kc) {
          const int64_t col = c + lane;
          const int64_t o = col / inner, i = col - o * inner;
          const S* xp = X + o * D * inner + i;
          for (int a = warp; a < ld; a += nw) tile[lane * ld + a] = a < D ? xp[a * inner] : S(0);
        }
      }
      __syncthreads();
      if (fits && c + kKC < c1) fetch(c + kKC, (int)((c1 - c - kKC) < kKC ? (c1 - c - kKC) : kKC), v);
      for (int kk = 0; kk < kc; ++kk) {
        const S* row = tile + kk * ld;
#pragma unroll
        for (int u = 0; u < MT; ++u) {
          if (!act[u]) continue;
          S av[4], bv[4];
          ld4(row + 4 * I[u], av);
          ld4(row + 4 * J[u], bv);
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[u][x][y] += av[x] * bv[y];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < MT; ++u) {
      if (!act[u]) continue;
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          const int a = 4 * I[u] + x, b = 4 * J[u] + y;
          if (a < D && b < D) {
            A[a * lda + b] = acc[u][x][y];
            A[b * lda + a] = acc[u][x][y];
          }
        }
    }
  }
  __syncthreads();
}

// Y = X x_m M^T... for a C-order tensor X seen as (outer, dm, inner) whose
// blocks X_o (dm x inner) are contiguous and hold at most kStage elements:
// Y_o (a x inner) = U^T X_o with U (dm x a, row-major) the factor, i.e. the
// mode-m product with U^T.  U is copied to shared memory (`us`, dm x round4(a))
// and X streams through `stage` (kStage elements) in chunks of whole blocks;
// the next chunk's loads are issued into registers before the current chunk
// is used.  Each output sums over j = 0..dm-1 in order.
template <class S>
__device__ void ttm_staged(const S* X, int64_t outer, int dm, int inner, const S* U, int a, S* Y, S* stage, S* us) {
  constexpr int PF = kStage / TK_NT;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int a4 = (a + 3) & ~3;
  for (int e = tid; e < dm * a4; e += nt) {
    const int j = e / a4, al = e - j * a4;
    us[e] = al < a ? U[j * a + al] : S(0);
  }
  const int blk = dm * inner;
  // staged stride of a block: one word more when a block is a single row
  // (inner == 1), so that threads reading different rows at the same column
  // hit different banks
  const int bst = inner == 1 ? blk + 1 : blk;
  const int ob = kStage / bst;  // blocks per chunk
  const int64_t nchunk = (outer + ob - 1) / ob;
  const int nch = a4 / 4;
  // this thread's staging slots: element e = tid + u * nt of a chunk is
  // (block e / blk, offset e % blk), walked with carries
  const int db = nt / blk, doff = nt - db * blk;
  auto fetch = [&](int64_t ch, S* v) {
    const int64_t o0 = ch * ob;
    const int64_t cnt = ((outer - o0) < ob ? (outer - o0) : ob) * blk;
    const S* xp = X + o0 * blk;
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int e = tid + u * nt;
      v[u] = e < cnt ? xp[e] : S(0);
    }
  };
  S v[PF];
  if (nchunk > 0) fetch(0, v);
  for (int64_t ch = 0; ch < nchunk; ++ch) {
    const int64_t o0 = ch * ob;
    const int nob = (int)((outer - o0) < ob ? (outer - o0) : ob);
    __syncthreads();  // the stage (and, first time, us) is free / ready
    {
      int b = tid / blk, off = tid - (tid / blk) * blk;
#pragma unroll
      for (int u = 0; u < PF; ++u) {
        if (b < ob) stage[b * bst + off] = v[u];
        off += doff;
        b += db;
        if (off >= blk) {
          off -= blk;
          ++b;
        }
      }
    }
    __syncthreads();
    if (ch + 1 < nchunk) fetch(ch + 1, v);
    // items (ob, c4, i), i fastest
    const int items = nob * nch * inner;
    for (int it = tid; it < items; it += nt) {
      const int i = it % inner;
      const int t = it / inner;
      const int c4 = t % nch, b = t / nch;
      const S* xs = stage + b * bst + i;
      const S* ms = us + 4 * c4;
      S acc[4] = {S(0), S(0), S(0), S(0)};
      for (int j = 0; j < dm; ++j) {
        const S x = xs[j * inner];
        S mv[4];
        ld4(ms + j * a4, mv);
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] += mv[c] * x;
      }
      S* yp = Y + ((o0 + b) * a + 4 * c4) * inner + i;
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (4 * c4 + c < a) yp[c * inner] = acc[c];
    }
  }
  __syncthreads();
}

// Rows [s0, s1) of mat_n(Y_n), Y_n = X x_{m != n} U_m^T (modes contracted
// from the last to the first), written to Y (D_n x Rn, row-major).  The slab
// X[..., s0:s1, ...] is first gathered into a contiguous buffer (mode 0's slab
// is contiguous already), then contracted with the block's TTM routine.
template <class S>
__device__ void slab_rows(const S* X, const int* xd, const int* rl, int p, int n, int s0, int s1, const S* const* U,
                          S* slab, S* b0, S* b1, S* Y, int64_t Rn, S* stage, S* us) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ds = s1 - s0;
  int dims[TK_MAXP];
  for (int m = 0; m < p; ++m) dims[m] = xd[m];
  dims[n] = ds;
  const int64_t outer = prod64(xd, 0, n), inner = prod64(xd, n + 1, p);
  const S* src;
  if (n == 0) {
    src = X + (int64_t)s0 * inner;
  } else {
    // for each outer index o the slab's rows are ds * inner contiguous elements
    // of X; element e = o * len + off is walked with carries (no division),
    // kGather elements per thread at a time so that their loads overlap
    constexpr int kGather = 16;
    const int64_t len = (int64_t)ds * inner, tot = outer * len;
    const int64_t dO = nt / len, dOff = nt - dO * len;
    int64_t o = tid / len, off = tid - (tid / len) * len;
    for (int64_t e0 = tid; e0 < tot; e0 += (int64_t)kGather * nt) {
      S v[kGather];
      int64_t oo = o, of = off;
#pragma unroll
      for (int u = 0; u < kGather; ++u) {
        v[u] = (e0 + (int64_t)u * nt < tot) ? X[(oo * xd[n] + s0) * inner + of] : S(0);
        of += dOff;
        oo += dO;
        if (of >= len) {
          of -= len;
          ++oo;
        }
      }
#pragma unroll
      for (int u = 0; u < kGather; ++u)
        if (e0 + (int64_t)u * nt < tot) slab[e0 + (int64_t)u * nt] = v[u];
      o = oo;
      off = of;
    }
    __syncthreads();
    src = slab;
  }
  S* dst = b0;
  for (int m = p - 1; m >= 0; --m) {
    if (m == n) continue;
    const int64_t in = prod64(dims, m + 1, p);
    if ((int64_t)dims[m] * in + 1 <= kStage)
      ttm_staged<S>(src, prod64(dims, 0, m), dims[m], (int)in, U[m], rl[m], dst, stage, us);
    else
      ttm<BlockGroup, S>(src, dims, p, m, U[m], 1, rl[m], rl[m], dst, false);
    dims[m] = rl[m];
    src = dst;
    dst = (dst == b0) ? b1 : b0;
  }
  // (o', d, i') of the contracted slab -> row s0 + d, column o' * inr + i'
  const int64_t inr = prod64(rl, n + 1, p);
  const int64_t tot = prod64(rl, 0, n) * ds * inr;
  for (int64_t e = tid; e < tot; e += nt) {
    const int64_t i = e % inr, t = e / inr;
    const int64_t d = t % ds, o = t / ds;
    Y[(s0 + d) * Rn + o * inr + i] = src[e];
  }
  __syncthreads();
}

}  // namespace

template <class S>
__global__ void __cluster_dims__(TK_LEAF_CL, 1, 1) __launch_bounds__(TK_NT)
    k_leaf(TkTreeView tv, const S* raw, int64_t block_stride, int64_t first_block, int njobs, int ell,
           TkWorkspace wsd, TkLeafLayout ly) {
  using BG = BlockGroup;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  static_assert(sizeof(LeafSm<S>) <= kHdr, "leaf shared header");
  LeafSm<S>& sm = *reinterpret_cast<LeafSm<S>*>(smem_raw);
  const int crank = (int)cluster_rank();
  const int cid = (int)cluster_id(), ncl = (int)num_clusters();
  // shared memory: the header, the Jacobi arrays for orders <= nsv, A for
  // orders <= nsa (the tridiagonal method needs A only; Jacobi also V),
  // then the contraction buffers
  const int nsa = ly.nsa, nsv = ly.nsv;
  const int half_cap = nsv / 2 + 2;
  size_t off = kHdr;
  int* js_pq = reinterpret_cast<int*>(smem_raw + off);
  off += align16(half_cap * sizeof(int));
  S* js_c = reinterpret_cast<S*>(smem_raw + off);
  S* js_s = js_c + half_cap;
  S* js_w = js_s + half_cap;
  off += align16(sizeof(S) * (2 * half_cap + nsv + 2));
  S* sA = reinterpret_cast<S*>(smem_raw + off);
  off += align16(sizeof(S) * (size_t)nsa * nsa);
  S* sV = reinterpret_cast<S*>(smem_raw + off);
  off += align16(sizeof(S) * (size_t)nsv * nsv);
  S* tile = reinterpret_cast<S*>(smem_raw + off);
  // the tensor-core Gram's staging buffers alias tile, stage and us: the Gram
  // phases and the contractions that use those never overlap
  unsigned char* tc_stage = smem_raw + off;
  off += align16(sizeof(S) * (size_t)kKC * (((ly.neig + 3) & ~3) + 4));
  S* stage = reinterpret_cast<S*>(smem_raw + off);
  off += align16(sizeof(S) * (size_t)kStage);
  S* us = reinterpret_cast<S*>(smem_raw + off);

  // tensor memory and the mbarriers of the tensor-core Grams (FP32 trees)
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_mbar[2];
  constexpr bool kF32 = std::is_same<S, float>::value;
  const bool tc_on = kF32 && ly.tc != 0;
  TcState st;
  st.tmem = 0;
  st.mbar = s_mbar;
  st.phase[0] = st.phase[1] = 0;
  st.pending[0] = st.pending[1] = 0;
  st.failed = 0;
  if (tc_on) {
    if (threadIdx.x == 0) {
      mbar_init(&s_mbar[0], 1);
      mbar_init(&s_mbar[1], 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((threadIdx.x >> 5) == 0) tmem_alloc(&s_tmem, kTcTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    st.tmem = s_tmem;
  }
  // Gram of the columns [c0, c1) of a matricization on the tensor cores when
  // that path is on and the order fits it, else on the CUDA cores
  auto gram = [&](const S* Xg, int D, int64_t inner, int64_t c0, int64_t c1, S* Ag, int lda) {
    bool done = false;
    if constexpr (kF32) {
      // (orders below 32 stay on the CUDA cores: too little work per chunk)
      const int kc = tc_on && D >= 32 && D <= kTcMaxD ? tc_chunk(D, ly.tc_bytes, blockDim.x) : 0;
      if (kc > 0)
        done = gram_tc(reinterpret_cast<const float*>(Xg), D, inner, c0, c1, reinterpret_cast<float*>(Ag), lda,
                       tc_stage, kc, st, ly.tc == 1, wsd.status);
    }
    if (!done) gram_cols<S>(Xg, D, inner, c0, c1, Ag, lda, tile);
  };

  S* wc = reinterpret_cast<S*>(wsd.base) + (int64_t)cid * wsd.per_cta;  // the cluster's chunk
  S* wt = wc + ly.cta + (int64_t)crank * ly.cta_stride;                 // this CTA's part
  // eigenproblem buffers for order dn: shared memory when they fit, else
  // this CTA's global region (ly.A etc. exist whenever some order exceeds nsv)
  auto uses_trd = [&](int dn, int rk) { return dn >= kTrdMinOrder && rk <= kTrdMaxRank; };
  auto eig_A = [&](int dn, int rk) -> S* { return (uses_trd(dn, rk) ? dn <= nsa : dn <= nsv) ? sA : wt + ly.A; };
  auto jac = [&](int dn, S** V, S** w) -> JacobiScratch<S> {
    const bool sm_ok = dn <= nsv;
    JacobiScratch<S> js;
    js.pq = sm_ok ? js_pq : reinterpret_cast<int*>(wt + ly.pq);
    js.c = sm_ok ? js_c : wt + ly.cs;
    js.s = sm_ok ? js_s : wt + ly.cs + ly.half;
    js.flag = &sm.flag;
    js.red = sm.red;
    js.nsw = &sm.nsw;
    js.thr = &sm.thr;
    *V = sm_ok ? sV : wt + ly.V;
    *w = sm_ok ? js_w : wt + ly.w;
    return js;
  };
  S* T = wt + ly.T;
  const S* U[TK_MAXP];
  for (int n = 0; n < TK_MAXP; ++n) U[n] = wc + ly.U[n];
  const int p = tv.p;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int maxsw = sizeof(S) == 8 ? 24 : 16;
  const int maxit = tv.max_iter > 0 ? tv.max_iter : 1;

  for (int job = cid; job < njobs; job += ncl) {
    const int64_t b = first_block + job;
    const S* X = raw + (int64_t)job * block_stride;
    const int64_t slot = tv.level_base[0] + b;
    int xd[TK_MAXP], rl[TK_MAXP];
    xd[0] = ell;
    for (int n = 1; n < p; ++n) xd[n] = tv.D[n];
    // rank clamp: min(r_n, extent_n), then r_n <= prod_{m!=n} r_m
    for (int n = 0; n < p; ++n) rl[n] = tv.r[n] < xd[n] ? tv.r[n] : xd[n];
    for (bool ch = true; ch;) {
      ch = false;
      for (int n = 0; n < p; ++n) {
        int64_t pr = 1;
        for (int m = 0; m < p; ++m)
          if (m != n) pr *= rl[m];
        if (rl[n] > pr) {
          rl[n] = (int)pr;
          ch = true;
        }
      }
    }
    const int64_t N = prod64(xd, 0, p);

    // ---- HOSVD start: ||X||^2 and the Grams of mat_n(X), n >= 2, by parts --
    {
      const int64_t e0 = N * crank / TK_LEAF_CL, e1 = N * (crank + 1) / TK_LEAF_CL;
      S a = 0;
      for (int64_t i = e0 + tid; i < e1; i += nt) a += X[i] * X[i];
      a = BG::sum<S>(a, sm.red);
      if (tid == 0) wc[ly.norm + crank] = a;
    }
    for (int n = 1; n < p; ++n) {
      const int64_t ncols = N / xd[n];
      const int64_t DD = (int64_t)xd[n] * xd[n];
      gram(X, xd[n], prod64(xd, n + 1, p), ncols * crank / TK_LEAF_CL, ncols * (crank + 1) / TK_LEAF_CL,
           wc + ly.part[n] + crank * DD, xd[n]);
    }
    cluster_barrier();
    for (int n = 1; n < p; ++n) {
      if ((n - 1) % TK_LEAF_CL != crank) continue;
      const int D = xd[n];
      const int DD = D * D;
      const S* part = wc + ly.part[n];
      S* A = eig_A(D, rl[n]);
      for (int i = tid; i < DD; i += nt) {
        S a = 0;
        for (int c = 0; c < TK_LEAF_CL; ++c) a += part[(int64_t)c * DD + i];
        A[i] = a;
      }
      __syncthreads();
      if (uses_trd(D, rl[n])) {
        trd_eig<BG, S>(D, rl[n], A, D, wc + ly.U[n], rl[n], wt + ly.trd, sm.sc, sm.cl);
      } else {
        S *V, *ew;
        JacobiScratch<S> js = jac(D, &V, &ew);
        jacobi_eig<BG, S>(D, rl[n], A, V, T, false, ew, js, maxsw);
        select_top<BG, S>(D, ew, V, rl[n], wc + ly.U[n], rl[n]);
        for (int i = tid; i < DD; i += nt) wc[ly.Vs[n] + i] = V[i];
        __syncthreads();
      }
    }
    if (crank == 0 && tid == 0) {
      S a = 0;
      for (int c = 0; c < TK_LEAF_CL; ++c) a += wc[ly.norm + c];
      sm.xn2 = a;
    }
    cluster_barrier();

    // ---- ALS iterations (Gauss-Seidel over the modes, then the core) -------
    S e_prev = S(-1), e = S(0);
    int it;
    for (it = 1; it <= maxit; ++it) {
      for (int n = 0; n < p; ++n) {
        const int dn = xd[n];
        int64_t Rn = 1;
        for (int m = 0; m < p; ++m)
          if (m != n) Rn *= rl[m];
        const int s0 = (int)((int64_t)dn * crank / TK_LEAF_CL);
        const int s1 = (int)((int64_t)dn * (crank + 1) / TK_LEAF_CL);
        if (s1 > s0)
          slab_rows<S>(X, xd, rl, p, n, s0, s1, U, wt + ly.slab, wt + ly.b0, wt + ly.b1, wc + ly.Y, Rn, stage, us);
        cluster_barrier();
        if (crank == 0) {
          const S* Y = wc + ly.Y;
          S* A = eig_A(dn, rl[n]);
          gram(Y, dn, Rn, 0, Rn, A, dn);
          if (uses_trd(dn, rl[n])) {
            trd_eig<BG, S>(dn, rl[n], A, dn, wc + ly.U[n], rl[n], wt + ly.trd, sm.sc, sm.cl);
          } else {
            // Jacobi, warm-started from the mode's previous basis (the HOSVD
            // start's for n >= 2 in the first iteration)
            S *V, *ew;
            JacobiScratch<S> js = jac(dn, &V, &ew);
            const bool warm = n > 0 || it > 1;
            if (warm) {
              for (int i = tid; i < dn * dn; i += nt) V[i] = wc[ly.Vs[n] + i];
              __syncthreads();
            }
            jacobi_eig<BG, S>(dn, rl[n], A, V, T, warm, ew, js, maxsw);
            select_top<BG, S>(dn, ew, V, rl[n], wc + ly.U[n], rl[n]);
            for (int i = tid; i < dn * dn; i += nt) wc[ly.Vs[n] + i] = V[i];
          }
          if (n == p - 1) {
            // core: G = fold_p(U_p^T mat_p(Y_p)), G[o * r_p + a] = sum_d U_p[d, a] Y[d, o]
            __syncthreads();
            S* Gc = wc + ly.G;
            gemm<BG, S>((int)Rn, rl[n], dn, Y, 1, (int)Rn, wc + ly.U[n], rl[n], 1, Gc, rl[n], 1, false);
            const S gn2 = sum_squares<BG, S>(Gc, Rn * rl[n], sm.red);
            e = sm.xn2 > S(0) ? sqrt(fmax(S(0), S(1) - gn2 / sm.xn2)) : S(0);
            const bool stop = tv.tol > 0 && it > 1 && fabs(e - e_prev) < (S)tv.tol;
            e_prev = e;
            if (tid == 0) wc[ly.flag] = stop ? S(1) : S(0);
          }
          __syncthreads();
        }
        cluster_barrier();
      }
      if (wc[ly.flag] != S(0)) break;
    }

    // ---- store: core (capacity dims r), temporal rows (ld r0), factors ------
    if (crank == 0) {
      S* core = reinterpret_cast<S*>(tv.core_pool) + slot * tv.core_stride;
      int ctot = 1;
      for (int m = 0; m < p; ++m) ctot *= tv.r[m];
      const S* Gc = wc + ly.G;
      for (int idx = tid; idx < ctot; idx += nt) {
        int rem = idx, src = 0, strd = 1;
        bool inside = true;
        for (int n = p - 1; n >= 0; --n) {
          const int in = rem % tv.r[n];
          rem /= tv.r[n];
          if (in >= rl[n]) inside = false;
          src += in * strd;
          strd *= rl[n];
        }
        core[idx] = inside ? Gc[src] : S(0);
      }
      S* tf = reinterpret_cast<S*>(tv.tfac) + b * (int64_t)tv.B * tv.r[0];
      const S* U0 = wc + ly.U[0];
      for (int idx = tid; idx < ell * tv.r[0]; idx += nt) {
        const int t = idx / tv.r[0], c = idx % tv.r[0];
        tf[idx] = c < rl[0] ? U0[t * rl[0] + c] : S(0);
      }
      for (int n = 1; n < p; ++n) {
        S* F = reinterpret_cast<S*>(tv.fac_pool[n]) + slot * tv.fac_stride[n];
        const S* Un = wc + ly.U[n];
        for (int idx = tid; idx < tv.D[n] * tv.r[n]; idx += nt) {
          const int d = idx / tv.r[n], c = idx % tv.r[n];
          F[idx] = c < rl[n] ? Un[d * rl[n] + c] : S(0);
        }
      }
      if (tid < TK_MAXP) tv.node_ranks[slot * TK_MAXP + tid] = tid < p ? rl[tid] : 0;
    }
    cluster_barrier();  // the cluster's workspace is reused by the next job
  }
  if (tc_on) {
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if ((threadIdx.x >> 5) == 0) tmem_free(st.tmem, kTcTmemCols);
  }
}

}  // namespace tk

using namespace tk;

size_t tk_leaf_smem_bytes(int dtype, int nsa, int nsv, int neig, int rmax, int64_t tc_bytes) {
  const size_t es = dtype == TK_F64 ? 8 : 4;
  const int half_cap = nsv / 2 + 2;
  size_t b = kHdr + align16(half_cap * sizeof(int));
  b += align16(es * (2 * half_cap + nsv + 2));
  b += align16(es * (size_t)nsa * nsa) + align16(es * (size_t)nsv * nsv);
  size_t c = align16(es * (size_t)kKC * (((neig + 3) & ~3) + 4));
  c += align16(es * (size_t)kStage);
  c += es * (size_t)neig * ((rmax + 3) & ~3);
  return b + std::max<size_t>(c, (size_t)tc_bytes);
}

// Bytes of the contraction buffers (tile, stage, us) of the leaf kernel.
size_t tk_leaf_contraction_bytes(int dtype, int neig, int rmax) {
  const size_t es = dtype == TK_F64 ? 8 : 4;
  return align16(es * (size_t)kKC * (((neig + 3) & ~3) + 4)) + align16(es * (size_t)kStage) +
         es * (size_t)neig * ((rmax + 3) & ~3);
}

template <class S> static const void* leaf_fn() { return (const void*)k_leaf<S>; }

int tk_leaf_max_clusters(int dtype, size_t smem) {
  const void* fn = dtype == TK_F64 ? leaf_fn<double>() : leaf_fn<float>();
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(TK_LEAF_CL, 1, 1);
  cfg.blockDim = dim3(TK_NT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

int tk_launch_leaf(int dtype, const TkTreeView& tv, const void* raw, int64_t block_stride, int64_t first_block,
                   int njobs, int ell, const TkWorkspace& ws, const TkLeafLayout& ly, int nclusters,
                   cudaStream_t stream) {
  if (njobs <= 0) return TK_OK;
  const size_t smem = tk_leaf_smem_bytes(dtype, ly.nsa, ly.nsv, ly.neig, ly.rmax, ly.tc_bytes);
  const dim3 grid(TK_LEAF_CL * nclusters);
  if (dtype == TK_F64) {
    if (cudaFuncSetAttribute(leaf_fn<double>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return TK_ERR_CUDA;
    k_leaf<double><<<grid, TK_NT, smem, stream>>>(tv, (const double*)raw, block_stride, first_block, njobs, ell, ws,
                                                  ly);
  } else {
    if (cudaFuncSetAttribute(leaf_fn<float>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return TK_ERR_CUDA;
    k_leaf<float><<<grid, TK_NT, smem, stream>>>(tv, (const float*)raw, block_stride, first_block, njobs, ell, ws,
                                                 ly);
  }
  return cudaGetLastError() == cudaSuccess ? TK_OK : TK_ERR_CUDA;
}
