// Device code of the stitch kernels (k_stitch, k_batch): included by the
// translation units that instantiate them, one kernel and precision each,
// so that the large job function is compiled in parallel.
//
//  k_hitset  Algorithm 1 (Recall) over the implicit dyadic stream segment tree.
//  k_plan    longest-first processing order of a query batch.
//  k_stitch  one CTA per job, jobs taken from a dynamic queue; a job is a
//            range query (Section 6.1: Recall, Eq. (partial-tucker),
//            Algorithm 2) or the re-decomposition of a newly complete node
//            from its two children (Algorithm 3, Stitch).
//  (k_leaf, the leaf blocks' Tucker-ALS, is in tk_leaf.cu.)
//
// Stitch runs in coefficient space.  Every V~_i^(1) has orthonormal columns
// and the hits occupy disjoint time rows, so Z^(1) of Eq. (stitch-temp-2)
// equals blockdiag(V~_i^(1)) K with K = [mat_1(H~_i x_{m>=2} W_im)]_i,
// W_im = U^(m)T V~_i^(m), and the leading left singular vectors of Z^(1) are
// blockdiag(V~_i^(1)) times the leading eigenvectors C of K K^T.  Hence
// U^(1)T_[t_{i-1},t_i) V~_i^(1) = C_i^T (the block rows of C).  For a
// non-temporal mode n, Phi_n = [V~_1^(n) ... V~_s^(n)] = Q_n R_n (Householder,
// once per job) turns Z^(n) of Eq. (stitch-nontemp-3) into Q_n N_n with
// N_n = sum_i mat_n(H~_i x_1 C_i^T x_{m!=1,n} W_im x_n R_n[:,blk i]); then
// U^(n) = Q_n E_n with E_n the leading eigenvectors of N_n N_n^T and
// W_im = E_m^T R_m[:,blk i].  The core is N_p x_p E_p^T (Algorithm 2's last
// step).  The loop never touches D or L: they enter only through the QR of
// Phi_n and the final factor assembly.  This is an exact rewrite: the result
// is Algorithm 2's iterate, up to rounding order.
//
// A job's problems are small (eig orders ~ sum_i r_i, tensors of r^p
// elements): one CTA owns a job, its hottest buffers in a shared-memory
// arena.  Eigenproblems of order >= kTrdMinOrder use the tridiagonal top-r
// method; smaller ones use Jacobi, warm-started from the same mode's
// eigenvectors of the previous iteration (or of the initialization).
#pragma once
#include <cstdio>

#include "tk_device.cuh"
#include "tk_internal.h"

namespace tk {

// Leading dimension of the matrices that the Householder steps walk by
// column (Phi_n, a partial hit's temporal slice, the staged output block):
// the next odd number, so that the 32 lanes of a warp, reading one column on
// consecutive rows, fall on 32 different shared-memory banks.  (Ranks are
// often multiples of 16, which puts a whole column on one or two banks.)
__device__ __forceinline__ int odd_ld(int k) { return k | 1; }

struct HitRec {
  int level, partial;
  int64_t index, node_lo, node_hi, lo, hi, slot;
  int64_t toff;       // row offset t_{i-1} of the hit in U^(1)
  void* core;         // H~_i (dims q)
  void* slice;        // partial slice (reflectors), if partial
  void* stau;         // its tau
  int q[TK_MAXP];     // ranks of H~_i
  int nr0;            // stored temporal rank of the node
  int chol;           // partial hit factored by Cholesky QR (R in the slice buffer), else Householder
  int koff[TK_MAXP];  // column offset of the hit's block in mode n's coefficient space
};
static_assert(sizeof(HitRec) <= TK_HITREC_BYTES, "HitRec grew: update TK_HITREC_BYTES");

template <class S> struct StitchCtx {
  int nh, err;
  int64_t L;
  int ro[TK_MAXP];
  int k[TK_MAXP];     // sum_i q_i[n]
  int c[TK_MAXP];     // coefficient dimension: k[0] for time, min(D_n, k_n) otherwise
  int qmax[TK_MAXP];
  HitRec* hits;       // the job's hit records (shared-memory copy when it fits)
  S *phi[TK_MAXP], *tau[TK_MAXP], *R[TK_MAXP], *E[TK_MAXP], *Vs[TK_MAXP];
  S *K, *b0, *b1, *N, *W, *G, *T, *A, *V, *w, *cs, *trdv;
  double *Ad, *Ed, *trdd, *scd;  // FP64 eigenproblem of an FP32 tree (eig64)
  S *Ug, *Uq, *Ut;               // seeded start: Gaussian matrix (its QR), its Q, tau
  int* pq;
  int neig;           // largest eig order of the job
  int smem_used;      // bytes of the shared arena in use
  int stage_end;      // arena offset of the first buffer after the staging region (E and later)
};

// Shared memory of one job group (a warp or a CTA): this header, then the
// Jacobi arrays for orders up to nsm (pq, c, s, w, A, V).
template <class S> struct WarpSm {
  StitchCtx<S> ctx;
  S red[40];
  S sc[4];
  int cl[64];
  S wbuf[16 * 33];  // reflector dot products (reflect_cols), up to 32 warps
  int flag;
  int job;
  int nsw;
  S thr;
};


// Shared bytes of one job group: the header, then `arena` bytes into which
// the job places its hottest buffers (the rest goes to its global chunk).
template <class S> __host__ __device__ inline size_t group_smem_bytes(size_t arena) {
  return align16(sizeof(WarpSm<S>)) + align16(arena);
}


__device__ __forceinline__ int64_t node_lo_of(const TkTreeView& tv, int j, int64_t k) {
  return (k << j) * (int64_t)tv.B;
}

// The tree as of T slices: complete blocks, blocks including the tail, and
// the height of Section 4.2.  Nodes complete at T stay unchanged by later
// appends, so a query can be answered against an earlier T as long as it
// does not reach into that T's open block.
struct TkEpoch {
  int64_t T, nb, nbt;
  int height;
};

__device__ __forceinline__ TkEpoch epoch_at(const TkTreeView& tv, int64_t T) {
  TkEpoch e;
  e.T = T;
  e.nb = T / tv.B;
  e.nbt = (T + tv.B - 1) / tv.B;
  e.height = e.nbt > 0 ? (e.nbt > 1 ? 64 - __clzll((unsigned long long)(e.nbt - 1)) : 0) + 1 : 0;
  return e;
}

__device__ __forceinline__ TkEpoch epoch_now(const TkTreeView& tv) {
  TkEpoch e;
  e.T = tv.T;
  e.nb = tv.nb;
  e.nbt = tv.nbt;
  e.height = tv.height;
  return e;
}

// Algorithm 1 (Recall) on the implicit tree as of epoch ep; with REC, writes
// up to cap hits in time order.  theta test in integers: theta_den * overlap
// >= theta_num * |v|.  Leaves are terminal: an overlapping leaf (complete or
// tail) is a hit.  Returns the hit count, or -1 if more than cap hits were
// found (REC only).
template <bool REC>
__device__ int recall_walk(const TkTreeView& tv, const TkEpoch& ep, int64_t ts, int64_t te, HitRec* hits, int cap) {
  if (ep.height <= 0) return 0;
  int sj[2 * TK_MAXL + 4];
  int64_t sk[2 * TK_MAXL + 4];
  int sp = 1, nh = 0;
  sj[0] = ep.height - 1;
  sk[0] = 0;
  while (sp > 0) {
    --sp;
    const int j = sj[sp];
    const int64_t k = sk[sp];
    const int64_t w = ((int64_t)1 << j) * tv.B;
    const int64_t lo = k * w;
    int64_t hi = lo + w;
    if (hi > ep.T) hi = ep.T;
    const int64_t a = ts > lo ? ts : lo, b = te < hi ? te : hi;
    const int64_t ov = b > a ? b - a : 0;
    const bool complete = ((k + 1) << j) <= ep.nb;
    bool hit = false;
    if (j == 0) hit = (k < ep.nbt) && ov > 0;
    else if (complete) hit = (int64_t)tv.theta_den * ov >= (int64_t)tv.theta_num * (hi - lo);
    if (hit) {
      if (REC) {
        if (nh >= cap) return -1;
        HitRec& h = hits[nh];
        h.level = j;
        h.index = k;
        h.node_lo = lo;
        h.node_hi = hi;
        h.lo = a;
        h.hi = b;
        h.partial = (a != lo || b != hi) ? 1 : 0;
      }
      ++nh;
      continue;
    }
    if (j == 0) continue;
    const int64_t mu = (2 * k + 1) * (w / 2);
    if (te <= mu) {
      sj[sp] = j - 1; sk[sp] = 2 * k; ++sp;
    } else if (ts >= mu) {
      sj[sp] = j - 1; sk[sp] = 2 * k + 1; ++sp;
    } else {
      sj[sp] = j - 1; sk[sp] = 2 * k + 1; ++sp;
      sj[sp] = j - 1; sk[sp] = 2 * k; ++sp;
    }
  }
  return nh;
}

__device__ inline int recall_dev(const TkTreeView& tv, const TkEpoch& ep, int64_t ts, int64_t te, HitRec* hits, int cap) {
  return recall_walk<true>(tv, ep, ts, te, hits, cap);
}

// Size of Algorithm 1's hit set; 0 for an invalid range.
__device__ inline int recall_count(const TkTreeView& tv, const TkEpoch& ep, int64_t ts, int64_t te) {
  if (!(ts >= 0 && ts < te && te <= ep.T)) return 0;
  return recall_walk<false>(tv, ep, ts, te, nullptr, 0);
}

__device__ inline void set_err(int* status, int code) { atomicCAS(status, 0, code); }

// The GPU's global nanosecond timer (the same clock on every SM).
__device__ __forceinline__ int64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return (int64_t)t;
}

// Output-rank clamp of a stitch: r_n' = min(r_n, extent_n, sum_i min(q_in,
// prod_{m!=n} q_im)), then r_n' <= prod_{m!=n} r_m' to a fixpoint.
__device__ inline void stitch_ranks(int p, const int* rq, const int64_t* ext, const HitRec* hits, int nh, int* ro) {
  for (int n = 0; n < p; ++n) {
    int64_t cap = 0;
    for (int i = 0; i < nh; ++i) {
      int64_t prod = 1;
      for (int m = 0; m < p; ++m)
        if (m != n) prod *= hits[i].q[m];
      cap += hits[i].q[n] < prod ? hits[i].q[n] : prod;
    }
    int64_t v = rq[n];
    if (ext[n] < v) v = ext[n];
    if (cap < v) v = cap;
    ro[n] = (int)v;
  }
  bool changed = true;
  while (changed) {
    changed = false;
    for (int n = 0; n < p; ++n) {
      int64_t prod = 1;
      for (int m = 0; m < p; ++m)
        if (m != n) prod *= ro[m];
      if (ro[n] > prod) {
        ro[n] = (int)prod;
        changed = true;
      }
    }
  }
}

// W (ro_m x q) = E_m^T R_m[:, koff .. koff+q): both row-major in the workspace.
template <class G, class S>
__device__ void proj_coef(const S* E, int cm, int rom, const S* R, int km, int koff, int q, S* W) {
  gemm<G, S>(rom, q, cm, E, 1, rom, R + koff, km, 1, W, q, 1, false);
}

// One stitch job, executed by one group G (a warp or a CTA).  ws is the
// group's workspace chunk (ws_cap elements); the hit records occupy its
// first TK_MAXH entries.
template <class G, class S>
__device__ void stitch_job(const TkTreeView& tv, const TkEpoch& ep, int mode, int64_t ts, int64_t te, int mlevel,
                           int64_t mindex,
                           const int* rq, S* ws, int64_t ws_cap, size_t arena_bytes, S* core_dst, S* u0_dst,
                           int64_t ld0,
                           S* const* un_dst, const int64_t* ldn, int* ranks_dst, tk_query_info* info,
                           int* status, unsigned char* wsm_raw, unsigned char* arena) {
  WarpSm<S>& sm = *reinterpret_cast<WarpSm<S>*>(wsm_raw);
  StitchCtx<S>& cx = sm.ctx;
  const long long t_start = clock64();
  const int64_t ns_start = global_ns();
  HitRec* hits = reinterpret_cast<HitRec*>(ws);  // Recall writes here; copied to the arena below
  const int hits_elems = (int)((TK_MAXH * (int64_t)TK_HITREC_BYTES + sizeof(S) - 1) / sizeof(S));
  const int p = tv.p;
  const int lane = G::rank();
  const int nt = G::size();

  if (lane == 0) {
    cx.err = 0;
    int nh = 0;
    if (mode == TK_JOB_QUERY) {
      nh = recall_dev(tv, ep, ts, te, hits, TK_MAXH);
      if (nh < 0) cx.err = TK_DEV_ERR_HITS;
    } else {
      nh = 2;
      for (int c = 0; c < 2; ++c) {
        HitRec& h = hits[c];
        h.level = mlevel - 1;
        h.index = 2 * mindex + c;
        h.node_lo = node_lo_of(tv, h.level, h.index);
        h.node_hi = h.node_lo + ((int64_t)1 << h.level) * tv.B;
        h.lo = h.node_lo;
        h.hi = h.node_hi;
        h.partial = 0;
      }
    }
    if (nh <= 0 && cx.err == 0) cx.err = TK_DEV_ERR_RANGE;
    cx.nh = nh > 0 ? nh : 0;
    int64_t L = 0;
    for (int i = 0; i < cx.nh; ++i) {
      HitRec& h = hits[i];
      h.slot = tv.level_base[h.level] + h.index;
      const int* nr = tv.node_ranks + h.slot * TK_MAXP;
      const int64_t ell = h.hi - h.lo;
      h.nr0 = nr[0];
      h.q[0] = h.partial ? (int)(ell < nr[0] ? ell : nr[0]) : nr[0];
      for (int n = 1; n < p; ++n) h.q[n] = nr[n];
      h.toff = L;
      L += ell;
    }
    cx.L = L;
    int64_t ext[TK_MAXP];
    ext[0] = L;
    for (int n = 1; n < p; ++n) ext[n] = tv.D[n];
    stitch_ranks(p, rq, ext, hits, cx.nh, cx.ro);
    for (int n = 0; n < p; ++n) {
      int kk = 0, qm = 0;
      for (int i = 0; i < cx.nh; ++i) {
        hits[i].koff[n] = kk;
        kk += hits[i].q[n];
        if (hits[i].q[n] > qm) qm = hits[i].q[n];
      }
      cx.k[n] = kk;
      cx.qmax[n] = qm;
      cx.c[n] = (n == 0) ? kk : (tv.D[n] < kk ? tv.D[n] : kk);
    }
    // Workspace layout: bump allocation in the group's shared arena first, in
    // order of how often the buffer is touched, then in the global chunk
    // (after the hit records).  Shared memory avoids the L2 round trip that
    // every read-after-write of the global chunk costs.
    size_t scur = 0;
    int64_t cur = hits_elems;
    auto take_bytes = [&](size_t bytes) -> void* {
      bytes = (bytes + 127) & ~(size_t)127;
      if (scur + bytes <= arena_bytes) {
        void* q = arena + scur;
        scur += bytes;
        return q;
      }
      void* q = ws + cur;
      cur += (int64_t)((bytes + sizeof(S) - 1) / sizeof(S));
      return q;
    };
    auto take = [&](int64_t nel) -> S* { return reinterpret_cast<S*>(take_bytes((size_t)nel * sizeof(S))); };
    {
      HitRec* hcopy = reinterpret_cast<HitRec*>(take_bytes(sizeof(HitRec) * (size_t)(cx.nh > 0 ? cx.nh : 1)));
      for (int i = 0; i < cx.nh; ++i) hcopy[i] = hits[i];
      cx.hits = hcopy;
    }
    int neig = cx.c[0];
    for (int n = 1; n < p; ++n)
      if (cx.c[n] > neig) neig = cx.c[n];
    cx.neig = neig;
    // the Jacobi method's eigenvector matrix, warm-start product and saved
    // bases exist only for the modes whose order is below the tridiagonal
    // method's (which keeps its reflectors in A)
    int njac = 0;
    for (int n = 0; n < p; ++n) {
      const bool trd = cx.c[n] >= kTrdMinOrder && cx.ro[n] <= kTrdMaxRank;
      if (!trd && cx.c[n] > njac) njac = cx.c[n];
    }
    cx.A = take((int64_t)neig * neig);
    cx.V = njac > 0 ? take((int64_t)njac * njac) : nullptr;
    cx.w = take(neig + 2);
    cx.cs = take(2 * (neig / 2 + 2));
    cx.pq = reinterpret_cast<int*>(take_bytes(sizeof(int) * (size_t)(neig / 2 + 2)));
    cx.T = njac > 0 ? take((int64_t)njac * njac) : nullptr;
    {
      int rmx = 1;
      for (int n = 0; n < p; ++n) rmx = cx.ro[n] > rmx ? cx.ro[n] : rmx;
      cx.trdv = take(trd_scratch_elems(neig, rmx, G::nwarps()));
      cx.Ad = cx.Ed = cx.trdd = cx.scd = nullptr;
      if (sizeof(S) == 4 && tv.eig64) {  // take() counts floats: two per double
        cx.Ad = reinterpret_cast<double*>(take(2 * (int64_t)neig * neig));
        cx.Ed = reinterpret_cast<double*>(take(2 * (int64_t)neig * rmx));
        cx.trdd = reinterpret_cast<double*>(take(2 * (int64_t)trd_scratch_elems(neig, rmx, G::nwarps())));
        cx.scd = reinterpret_cast<double*>(take(16));
      }
    }
    // chain buffers b0, b1: every intermediate of a hit's chain has, per mode,
    // at most max(q_max, ro) entries (and the stored temporal rank of a
    // partial hit in time); the core G (ro_1 x ... x ro_p) lives in b1 between
    // an iteration's last step and the next iteration's chains
    int64_t tb = 1;
    for (int m = 0; m < p; ++m) {
      int e = cx.qmax[m] > cx.ro[m] ? cx.qmax[m] : cx.ro[m];
      if (m == 0 && tv.r[0] > e) e = tv.r[0];
      tb *= e;
    }
    for (int n = 0; n < p; ++n) {  // the init's per-hit Gram and its product with R_n's block
      const int64_t g = (int64_t)cx.qmax[n] * cx.qmax[n], rm = (int64_t)cx.c[n] * cx.qmax[n];
      tb = g > tb ? g : tb;
      tb = rm > tb ? rm : tb;
    }
    cx.b0 = take(tb);
    cx.b1 = take(tb);
    cx.G = cx.b1;
    // K (k_1 rows of prod_{m>=2} ro_m) is dead once the temporal eigenvectors
    // C are formed, before any N_n (c_n in mode n, ro elsewhere) is written:
    // one buffer holds both
    int64_t Kel = cx.k[0];
    for (int m = 1; m < p; ++m) Kel *= cx.ro[m];
    for (int n = 1; n < p; ++n) {
      int64_t s = cx.c[n];
      for (int m = 0; m < p; ++m)
        if (m != n) s *= cx.ro[m];
      Kel = s > Kel ? s : Kel;
    }
    cx.K = take(Kel);
    cx.N = cx.K;
    int wmax = tv.r[0] * tv.r[0];
    for (int m = 0; m < p; ++m) {
      const int v = cx.ro[m] * (cx.qmax[m] > 1 ? cx.qmax[m] : 1);
      if (v > wmax) wmax = v;
    }
    cx.W = take(wmax);
    cx.stage_end = (int)scur;  // everything from here on may be live while Phi_n is staged
    for (int n = 0; n < p; ++n) cx.E[n] = take((int64_t)cx.c[n] * cx.ro[n]);
    for (int n = 1; n < p; ++n) cx.R[n] = take((int64_t)cx.c[n] * cx.k[n]);
    for (int i = 0; i < cx.nh; ++i) {
      HitRec& h = cx.hits[i];
      int64_t cs = 1;
      for (int n = 0; n < p; ++n) cs *= (n == 0 ? (h.q[0] > h.nr0 ? h.q[0] : h.nr0) : h.q[n]);
      h.core = take(cs);
    }
    for (int n = 0; n < p; ++n) {
      const bool trd = cx.c[n] >= kTrdMinOrder && cx.ro[n] <= kTrdMaxRank;
      cx.Vs[n] = trd ? nullptr : take((int64_t)cx.c[n] * cx.c[n]);
    }
    for (int n = 1; n < p; ++n) {
      cx.phi[n] = take((int64_t)tv.D[n] * odd_ld(cx.k[n]));
      cx.tau[n] = take(cx.k[n]);
    }
    for (int i = 0; i < cx.nh; ++i) {
      HitRec& h = cx.hits[i];
      if (h.partial) {
        h.slice = take((h.hi - h.lo) * (int64_t)odd_ld(h.nr0));
        h.stau = take(h.nr0);
      } else {
        h.slice = h.stau = nullptr;
      }
    }
    cx.Ug = cx.Uq = cx.Ut = nullptr;
    if (tv.init == TK_INIT_RANDOM) {
      int64_t dr = 0;
      int rmx = 1;
      for (int n = 1; n < p; ++n) {
        const int64_t v = (int64_t)tv.D[n] * odd_ld(cx.ro[n]);
        dr = v > dr ? v : dr;
        rmx = cx.ro[n] > rmx ? cx.ro[n] : rmx;
      }
      cx.Ug = take(dr);
      cx.Uq = take(dr);
      cx.Ut = take(rmx);
    }
    cx.smem_used = (int)scur;
    if (cur > ws_cap && cx.err == 0) cx.err = TK_DEV_ERR_WORKSPACE;
  }
  G::sync();
  if (cx.err) {
    if (lane == 0) {
      set_err(status, cx.err);
      if (info) {
        info->iters = -cx.err;
        info->n_hits = cx.nh;
      }
    }
    G::sync();
    return;
  }
  const int nh = cx.nh;
  hits = cx.hits;
  S* A = cx.A;
  S* V = cx.V;
  S* wv = cx.w;
  JacobiScratch<S> js;
  js.pq = cx.pq;
  js.c = cx.cs;
  js.s = cx.cs + (cx.neig / 2 + 2);
  js.flag = &sm.flag;
  js.red = sm.red;
  js.nsw = &sm.nsw;
  js.thr = &sm.thr;
  S* T = cx.T;
  const int maxsw = sizeof(S) == 8 ? 24 : 16;
  bool have_v[TK_MAXP];
  for (int n = 0; n < TK_MAXP; ++n) have_v[n] = false;
  int sweeps = 0;
  long long eig_cyc = 0, qr_cyc = 0;
  // leading ro[mode_n] eigenvectors of the order-nsz matrix in A, written to
  // Edst (leading dimension lde): the tridiagonal method from order
  // kTrdMinOrder on, else Jacobi warm-started from the mode's previous basis
  auto eig = [&](int mode_n, int nsz, S* Edst, int lde) {
    const long long c0 = clock64();
    const int rkeep = cx.ro[mode_n];
    if (nsz >= kTrdMinOrder && rkeep <= kTrdMaxRank && cx.Ad) {
      // FP64 under an FP32 stitch: the matrix widened, the eigenproblem
      // solved in FP64, the eigenvectors rounded to FP32
      for (int i = lane; i < nsz * nsz; i += nt) cx.Ad[i] = (double)A[i];
      G::sync();
      trd_eig<G, double>(nsz, rkeep, cx.Ad, nsz, cx.Ed, rkeep, cx.trdd, cx.scd, sm.cl);
      for (int i = lane; i < nsz * rkeep; i += nt) Edst[(i / rkeep) * lde + i % rkeep] = (S)cx.Ed[i];
      G::sync();
    } else if (nsz >= kTrdMinOrder && rkeep <= kTrdMaxRank) {
      trd_eig<G, S>(nsz, rkeep, A, nsz, Edst, lde, cx.trdv, sm.sc, sm.cl);
    } else {
      S* Vs = cx.Vs[mode_n];
      const bool warm = have_v[mode_n];
      if (warm) {
        for (int i = lane; i < nsz * nsz; i += nt) V[i] = Vs[i];
        G::sync();
      }
      sweeps += jacobi_eig<G, S>(nsz, rkeep, A, V, T, warm, wv, js, maxsw);
      for (int i = lane; i < nsz * nsz; i += nt) Vs[i] = V[i];
      G::sync();
      have_v[mode_n] = true;
      select_top<G, S>(nsz, wv, V, rkeep, Edst, lde);
    }
    eig_cyc += clock64() - c0;
  };
  int dims[TK_MAXP];

  // Cholesky QR of the ell x m slice S (rows ld apart; ell >= 2m): the Gram
  // S^T S, summed over chunks of rows staged in b0, then its Cholesky factor
  // R (upper triangular, positive diagonal) by warp 0, so that S = Q R with
  // Q = S R^{-1}.  Accepted when the diagonal of R spans at most a factor of
  // 10 (condition number of S near 10 or below: Q is then orthonormal to
  // about 100 ulps); R goes to Rout (leading dimension ldr, zeros below the
  // diagonal).  Returns false, on every thread, otherwise: the caller falls
  // back to Householder.
  auto cholesky_qr = [&](const S* Sg, int ld, int ell, int m, S* Rout, int ldr) -> bool {
    const int npair = m * (m + 1) / 2;
    if (npair > nt) return false;  // one pair of columns per thread
    S* Gm = cx.b1;  // m x m Gram, then R in its upper triangle
    S* st = cx.b0;  // staged rows
    int ch = 0;
    {
      int64_t cap = 1;
      for (int n = 0; n < p; ++n) cap *= (cx.qmax[n] > cx.ro[n] ? cx.qmax[n] : cx.ro[n]);
      ch = (int)(cap / m);
      if (ch < 1) ch = 1;
    }
    int pa = 0, pb = 0;  // this thread's pair (a <= b) of the packed upper triangle
    if (lane < npair) {
      int rem = lane;
      while (rem >= m - pa) {
        rem -= m - pa;
        ++pa;
      }
      pb = pa + rem;
    }
    S acc0 = 0, acc1 = 0;
    for (int t0 = 0; t0 < ell; t0 += ch) {
      const int cn = ell - t0 < ch ? ell - t0 : ch;
      for (int idx = lane; idx < cn * m; idx += nt) {
        const int t = idx / m, c = idx - (idx / m) * m;
        st[idx] = Sg[(int64_t)(t0 + t) * ld + c];
      }
      G::sync();
      if (lane < npair) {
        int t = 0;
        for (; t + 1 < cn; t += 2) {
          acc0 += st[t * m + pa] * st[t * m + pb];
          acc1 += st[(t + 1) * m + pa] * st[(t + 1) * m + pb];
        }
        if (t < cn) acc0 += st[t * m + pa] * st[t * m + pb];
      }
      G::sync();
    }
    if (lane < npair) Gm[pa * m + pb] = acc0 + acc1;
    G::sync();
    if (lane < 32) {
      int ok = 1;
      S dmin = 0, dmax = 0;
      for (int k = 0; k < m; ++k) {
        S d = Gm[k * m + k];
        for (int i = 0; i < k; ++i) d -= Gm[i * m + k] * Gm[i * m + k];
        if (!(d > S(0))) ok = 0;
        const S rkk = ok ? sqrt(d) : S(1);
        dmin = k == 0 ? rkk : fmin(dmin, rkk);
        dmax = k == 0 ? rkk : fmax(dmax, rkk);
        for (int j = k + 1 + lane; j < m; j += 32) {
          S v = Gm[k * m + j];
          for (int i = 0; i < k; ++i) v -= Gm[i * m + k] * Gm[i * m + j];
          Gm[k * m + j] = v / rkk;
        }
        __syncwarp();
        if (lane == 0) Gm[k * m + k] = rkk;
        __syncwarp();
      }
      if (lane == 0) sm.flag = (ok && dmin * S(10) >= dmax) ? 1 : 0;
    }
    G::sync();
    const bool good = sm.flag != 0;
    if (good) {
      for (int idx = lane; idx < m * m; idx += nt) {
        const int a = idx / m, b = idx - (idx / m) * m;
        Rout[a * ldr + b] = b >= a ? Gm[a * m + b] : S(0);
      }
    }
    G::sync();
    return good;
  };

  // ---- hit decompositions: stored payloads or Eq. (partial-tucker) -------
  S hn2 = 0;
  for (int i = 0; i < nh; ++i) {
    const HitRec& h = hits[i];
    const S* core = reinterpret_cast<const S*>(tv.core_pool) + h.slot * tv.core_stride;
    const int* nr = tv.node_ranks + h.slot * TK_MAXP;
    S* Hc = reinterpret_cast<S*>(h.core);
    int qd[TK_MAXP];
    for (int n = 0; n < p; ++n) qd[n] = h.q[n];
    if (!h.partial) {
      int tot = 1;
      for (int n = 0; n < p; ++n) tot *= qd[n];
      for (int idx = lane; idx < tot; idx += nt) {
        int rem = idx, src = 0, strd = 1;
        for (int n = p - 1; n >= 0; --n) {
          const int in = rem % qd[n];
          rem /= qd[n];
          src += in * strd;
          strd *= tv.r[n];
        }
        Hc[idx] = core[src];
      }
      G::sync();
    } else {
      // slice S (ell x nr0) of the node's temporal factor, S = Q R~, then H x_1 R~
      const int ell = (int)(h.hi - h.lo);
      const S* tf = reinterpret_cast<const S*>(tv.tfac) + h.level * tv.tfac_level_stride;
      const S* Sg = tf + h.lo * tv.r[0];  // S[t][c] = Sg[t * r_1 + c]
      S* sl = reinterpret_cast<S*>(h.slice);
      const int nr0 = h.nr0, lds = odd_ld(nr0);
      const long long c0 = clock64();
      const bool chol = ell >= 2 * nr0 && cholesky_qr(Sg, tv.r[0], ell, nr0, sl, lds);
      if (!chol) {  // Householder: S copied to the slice buffer, reflectors below R
        for (int idx = lane; idx < ell * nr0; idx += nt) {
          const int t = idx / nr0, c = idx % nr0;
          sl[t * lds + c] = Sg[t * tv.r[0] + c];
        }
        G::sync();
        householder_qr<G, S>(sl, ell, nr0, lds, reinterpret_cast<S*>(h.stau), sm.sc, sm.red, sm.wbuf);
      }
      if (lane == 0) const_cast<HitRec&>(h).chol = chol ? 1 : 0;
      qr_cyc += clock64() - c0;
      int tot = 1;
      for (int n = 0; n < p; ++n) {
        dims[n] = nr[n];
        tot *= nr[n];
      }
      S* b0 = cx.b0;
      for (int idx = lane; idx < tot; idx += nt) {
        int rem = idx, src = 0, strd = 1;
        for (int n = p - 1; n >= 0; --n) {
          const int in = rem % dims[n];
          rem /= dims[n];
          src += in * strd;
          strd *= tv.r[n];
        }
        b0[idx] = core[src];
      }
      S* Rt = cx.W;
      const int q0 = h.q[0];
      for (int idx = lane; idx < q0 * nr0; idx += nt) {
        const int a = idx / nr0, b = idx % nr0;
        Rt[idx] = (b >= a) ? sl[a * lds + b] : S(0);
      }
      G::sync();
      ttm<G, S>(b0, dims, p, 0, Rt, nr0, 1, q0, Hc, false);
    }
    int tot = 1;
    for (int n = 0; n < p; ++n) tot *= qd[n];
    hn2 += sum_squares<G, S>(Hc, tot, sm.red);
  }

  // Shared-memory staging for the Householder work on Phi_n: while Phi_n is
  // factored (and again while Q_n is applied to the output), the arena from
  // the eigensolver's matrices up to the factor blocks E holds nothing live,
  // so Phi_n, when it lives in global memory, is worked on there.
  auto staging = [&](int64_t nel) -> S* {
    if (!__isShared(cx.A) || __isShared(cx.phi[1])) return nullptr;
    // up to where E was carved: buffers taken after it (tau, R, the cores)
    // may sit in the arena's tail even when E itself went to global memory
    const char* lim = reinterpret_cast<const char*>(arena + cx.stage_end);
    return (lim - reinterpret_cast<const char*>(cx.A)) >= (int64_t)(nel * sizeof(S)) ? cx.A : nullptr;
  };

  const long long t_hits = clock64();
  // ---- non-temporal bases Phi_n = Q_n R_n, and the implicit HOSVD start ---
  for (int n = 1; n < p; ++n) {
    const int Dn = tv.D[n], kn = cx.k[n], cn = cx.c[n], ldp = odd_ld(kn);
    S* stg = staging((int64_t)Dn * ldp);
    S* Phi = stg ? stg : cx.phi[n];
    for (int i = 0; i < nh; ++i) {
      const HitRec& h = hits[i];
      const S* F = reinterpret_cast<const S*>(tv.fac_pool[n]) + h.slot * tv.fac_stride[n];
      const int qn = h.q[n], ko = h.koff[n];
      for (int idx = lane; idx < Dn * qn; idx += nt) {
        const int d = idx / qn, c = idx % qn;
        Phi[d * ldp + ko + c] = F[d * tv.r[n] + c];
      }
    }
    G::sync();
    const long long c0 = clock64();
    householder_qr<G, S>(Phi, Dn, kn, ldp, cx.tau[n], sm.sc, sm.red, sm.wbuf);
    qr_cyc += clock64() - c0;
    S* R = cx.R[n];
    for (int idx = lane; idx < cn * kn; idx += nt) {
      const int a = idx / kn, b = idx % kn;
      R[idx] = (b >= a) ? Phi[a * ldp + b] : S(0);
    }
    if (stg) {  // the reflectors are needed again for the output
      for (int idx = lane; idx < Dn * ldp; idx += nt) cx.phi[n][idx] = stg[idx];
      G::sync();
    }
    if (tv.init == TK_INIT_RANDOM) {
      // Algorithm 2's random start: U^(n) = Q of a seeded D_n x r_n Gaussian
      // matrix (elements from sum_{m<n} D_m r_m on), entering the coefficient
      // space as E_n = Q_n^T U^(n) (first c_n rows of H_{c-1}..H_0 U^(n)):
      // W_im = U^(m)T V~_i^(m) = E_m^T R_m[:, blk i] holds for any U^(m)
      const int rn = cx.ro[n], ldu = odd_ld(rn);
      int64_t off = 0;
      for (int m = 1; m < n; ++m) off += (int64_t)tv.D[m] * cx.ro[m];
      for (int idx = lane; idx < Dn * rn; idx += nt) {
        const int d = idx / rn, c = idx - (idx / rn) * rn;
        cx.Ug[d * ldu + c] = (S)gaussian_at(tv.seed, (uint64_t)(off + idx));
        cx.Uq[d * ldu + c] = d == c ? S(1) : S(0);
      }
      G::sync();
      householder_qr<G, S>(cx.Ug, Dn, rn, ldu, cx.Ut, sm.sc, sm.red, sm.wbuf);
      householder_apply_q<G, S>(cx.Ug, Dn, rn < Dn ? rn : Dn, ldu, cx.Ut, cx.Uq, rn, ldu, sm.wbuf);
      householder_apply_qt<G, S>(cx.phi[n], Dn, cn, ldp, cx.tau[n], cx.Uq, rn, ldu, sm.wbuf);
      for (int idx = lane; idx < cn * rn; idx += nt) {
        const int a = idx / rn, b = idx - (idx / rn) * rn;
        cx.E[n][idx] = cx.Uq[a * ldu + b];
      }
      G::sync();
      continue;
    }
    for (int idx = lane; idx < cn * cn; idx += nt) A[idx] = 0;
    G::sync();
    // init: Q_n^T mat_n(Y~) mat_n(Y~)^T Q_n = sum_i R_i M_i R_i^T, with
    // R_i = R_n[:, blk i] (c_n x q_in) and M_i = mat_n(H~_i) mat_n(H~_i)^T
    // (q_in x q_in): the Gram of mat_n(H~_i x_n R_i) without forming it
    for (int i = 0; i < nh; ++i) {
      const HitRec& h = hits[i];
      for (int m = 0; m < p; ++m) dims[m] = h.q[m];
      const int qn = h.q[n];
      S* Mi = cx.b0;
      S* RM = cx.b1;
      mode_gram<G, S>(reinterpret_cast<S*>(h.core), dims, p, n, Mi, qn, false);
      gemm<G, S>(cn, qn, qn, R + h.koff[n], kn, 1, Mi, qn, 1, RM, qn, 1, false);
      sym_accum<G, S>(cn, qn, RM, qn, R + h.koff[n], kn, A, cn);
    }
    eig(n, cn, cx.E[n], cx.ro[n]);
  }

  const long long t_init = clock64();
  // ---- Algorithm 2 iterations --------------------------------------------
  S e_prev = S(-1);
  S e = 0;
  int it = 0;
  const int maxit = tv.max_iter > 0 ? tv.max_iter : 1;
  const int* ro = cx.ro;
  S* K = cx.K;
  S* C = cx.E[0];
  S* N = cx.N;
  S* Wb = cx.W;
  S* b0 = cx.b0;
  S* b1 = cx.b1;
  for (it = 1; it <= maxit; ++it) {
    // temporal mode, Eq. (stitch-temp-2) in coefficient space
    int krow = 1;
    for (int m = 1; m < p; ++m) krow *= ro[m];
    for (int i = 0; i < nh; ++i) {
      const HitRec& h = hits[i];
      for (int m = 0; m < p; ++m) dims[m] = h.q[m];
      const S* src = reinterpret_cast<S*>(h.core);
      for (int m = 1; m < p; ++m) {
        proj_coef<G, S>(cx.E[m], cx.c[m], ro[m], cx.R[m], cx.k[m], h.koff[m], h.q[m], Wb);
        S* dst = (m == p - 1) ? K + h.koff[0] * krow : ((m & 1) ? b0 : b1);
        ttm<G, S>(src, dims, p, m, Wb, h.q[m], 1, ro[m], dst, false);
        dims[m] = ro[m];
        src = dst;
      }
    }
    {
      const int c0 = cx.c[0];
      dims[0] = c0;
      for (int m = 1; m < p; ++m) dims[m] = ro[m];
      mode_gram<G, S>(K, dims, p, 0, A, c0, false);
      eig(0, c0, C, ro[0]);
    }
    // non-temporal modes, Eq. (stitch-nontemp-3) in coefficient space
    for (int n = 1; n < p; ++n) {
      const int cn = cx.c[n], kn = cx.k[n];
      for (int i = 0; i < nh; ++i) {
        const HitRec& h = hits[i];
        for (int m = 0; m < p; ++m) dims[m] = h.q[m];
        // x_1 C_i^T : M(alpha, j) = C[(koff0 + j) * ro0 + alpha]
        ttm<G, S>(reinterpret_cast<S*>(h.core), dims, p, 0, C + h.koff[0] * ro[0], 1, ro[0], ro[0], b0, false);
        dims[0] = ro[0];
        S* src = b0;
        S* other = b1;
        for (int m = 1; m < p; ++m) {
          if (m == n) continue;
          proj_coef<G, S>(cx.E[m], cx.c[m], ro[m], cx.R[m], cx.k[m], h.koff[m], h.q[m], Wb);
          ttm<G, S>(src, dims, p, m, Wb, h.q[m], 1, ro[m], other, false);
          dims[m] = ro[m];
          S* t = src;
          src = other;
          other = t;
        }
        ttm<G, S>(src, dims, p, n, cx.R[n] + h.koff[n], kn, 1, cn, N, i > 0);
      }
      for (int m = 0; m < p; ++m) dims[m] = ro[m];
      dims[n] = cn;
      mode_gram<G, S>(N, dims, p, n, A, cn, false);
      eig(n, cn, cx.E[n], ro[n]);
    }
    // core: G = N_p x_p E_p^T (Algorithm 2's last step) and the stop test
    {
      const int n = p - 1;
      for (int m = 0; m < p; ++m) dims[m] = ro[m];
      dims[n] = cx.c[n];
      ttm<G, S>(N, dims, p, n, cx.E[n], 1, ro[n], ro[n], cx.G, false);
    }
    int gel = 1;
    for (int m = 0; m < p; ++m) gel *= ro[m];
    const S gn2 = sum_squares<G, S>(cx.G, gel, sm.red);
    e = hn2 > S(0) ? sqrt(fmax(S(0), S(1) - gn2 / hn2)) : S(0);
    if (tv.tol > 0 && it > 1 && fabs(e - e_prev) < (S)tv.tol) break;
    e_prev = e;
  }
  if (it > maxit) it = maxit;
  const long long t_als = clock64();

  // ---- outputs: core, U^(1) = blockdiag(V~_i^(1)) C, U^(n) = Q_n E_n --------
  {
    int ctot = 1;
    for (int m = 0; m < p; ++m) ctot *= rq[m];
    const S* Gc = cx.G;
    for (int idx = lane; idx < ctot; idx += nt) {
      int rem = idx, src = 0, strd = 1;
      bool inside = true;
      for (int n = p - 1; n >= 0; --n) {
        const int in = rem % rq[n];
        rem /= rq[n];
        if (in >= ro[n]) inside = false;
        src += in * strd;
        strd *= ro[n];
      }
      core_dst[idx] = inside ? Gc[src] : S(0);
    }
    G::sync();  // G lives in b1, which the staging below may overwrite
  }
  for (int i = 0; i < nh; ++i) {
    const HitRec& h = hits[i];
    const int ell = (int)(h.hi - h.lo);
    S* Y = u0_dst + h.toff * ld0;
    const S* Ci = C + h.koff[0] * ro[0];
    if (!h.partial) {
      const S* tf = reinterpret_cast<const S*>(tv.tfac) + h.level * tv.tfac_level_stride + h.lo * tv.r[0];
      gemm<G, S>(ell, ro[0], h.q[0], tf, tv.r[0], 1, Ci, ro[0], 1, Y, ld0, 1, false);
    } else if (h.chol) {
      // Q [C_i; 0] = S R^{-1}[:, :q] C_i = S[:, :q] M with M = R[:q, :q]^{-1} C_i
      // (R upper triangular): back substitution, one column of C_i per thread
      const int q0 = h.q[0], lds = odd_ld(h.nr0);
      const S* R = reinterpret_cast<const S*>(h.slice);
      S* M = cx.W;
      for (int c = lane; c < ro[0]; c += nt) {
        for (int a = q0 - 1; a >= 0; --a) {
          S v = Ci[a * ro[0] + c];
          for (int b = a + 1; b < q0; ++b) v -= R[a * lds + b] * M[b * ro[0] + c];
          M[a * ro[0] + c] = v / R[a * lds + a];
        }
      }
      G::sync();
      const S* Sg = reinterpret_cast<const S*>(tv.tfac) + h.level * tv.tfac_level_stride + h.lo * tv.r[0];
      gemm<G, S>(ell, ro[0], q0, Sg, tv.r[0], 1, M, ro[0], 1, Y, ld0, 1, false);
    } else {
      for (int idx = lane; idx < ell * ro[0]; idx += nt) {
        const int t = idx / ro[0], a = idx % ro[0];
        Y[t * ld0 + a] = (t < h.q[0]) ? Ci[t * ro[0] + a] : S(0);
      }
      G::sync();
      householder_apply_q<G, S>(reinterpret_cast<S*>(h.slice), ell, h.q[0], odd_ld(h.nr0), reinterpret_cast<S*>(h.stau), Y, ro[0],
                                ld0, sm.wbuf);
    }
    if (ro[0] < rq[0]) {
      const int padc = rq[0] - ro[0];
      for (int idx = lane; idx < ell * padc; idx += nt) Y[(idx / padc) * ld0 + ro[0] + idx % padc] = 0;
    }
    G::sync();
  }
  for (int n = 1; n < p; ++n) {
    const int Dn = tv.D[n], cn = cx.c[n];
    S* Yout = un_dst[n];
    const int64_t ldo = ldn[n];
    const S* E = cx.E[n];
    const int kn = cx.k[n], ldp = odd_ld(kn);
    // Q_n [E_n; 0], with Phi_n and the block staged in shared memory when possible
    S* stg = staging((int64_t)Dn * ldp + (int64_t)Dn * odd_ld(ro[n]));
    const S* Ph = cx.phi[n];
    S* Y = Yout;
    int64_t ld = ldo;
    if (stg) {
      for (int idx = lane; idx < Dn * ldp; idx += nt) stg[idx] = cx.phi[n][idx];
      Ph = stg;
      Y = stg + (int64_t)Dn * ldp;
      ld = odd_ld(ro[n]);
    }
    for (int idx = lane; idx < Dn * ro[n]; idx += nt) {
      const int d = idx / ro[n], a = idx % ro[n];
      Y[d * ld + a] = d < cn ? E[d * ro[n] + a] : S(0);
    }
    G::sync();
    householder_apply_q<G, S>(Ph, Dn, cn, ldp, cx.tau[n], Y, ro[n], ld, sm.wbuf);
    if (stg || ro[n] < rq[n]) {
      for (int idx = lane; idx < Dn * rq[n]; idx += nt) {
        const int d = idx / rq[n], a = idx % rq[n];
        Yout[d * ldo + a] = a < ro[n] ? Y[d * ld + a] : S(0);
      }
      G::sync();
    }
  }
  if (lane == 0) {
    if (ranks_dst)
      for (int n = 0; n < TK_MAXP; ++n) ranks_dst[n] = n < p ? ro[n] : 0;
    if (info) {
      for (int n = 0; n < TK_MAXP; ++n) info->ranks[n] = n < p ? ro[n] : 0;
      info->iters = it;
      info->n_hits = nh;
      info->fit_err = (double)e;
      info->eig_sweeps = sweeps;
      info->eig_max_order = cx.neig;
      info->device_cycles = (int64_t)(clock64() - t_start);
      info->eig_cycles = (int64_t)eig_cyc;
      info->qr_cycles = (int64_t)qr_cyc;
      info->hit_cycles = (int64_t)(t_hits - t_start);
      info->init_cycles = (int64_t)(t_init - t_hits);
      info->als_cycles = (int64_t)(t_als - t_init);
      info->out_cycles = (int64_t)(clock64() - t_als);
      info->start_ns = ns_start;
      info->end_ns = global_ns();
    }
  }
  G::sync();
}

// One range query of a batch (index q) by group G: validation against the
// query's epoch, output pointers into the packed output, then the stitch.
template <class G, class S>
__device__ void query_job(const TkTreeView& tv, const TkQueryBatch& qb, int q, S* ws, int64_t ws_cap,
                          size_t arena_bytes, int* status, unsigned char* wsm, unsigned char* arena) {
  const int64_t ts = qb.ranges[2 * q], te = qb.ranges[2 * q + 1];
  S* out = reinterpret_cast<S*>(qb.out) + qb.offsets[q];
  tk_query_info* info = qb.info ? qb.info + q : nullptr;
  const TkEpoch ep = (qb.tq && qb.tq[q] <= tv.T) ? epoch_at(tv, qb.tq[q]) : epoch_now(tv);
  if (!(ts >= 0 && ts < te && te <= ep.T)) {
    if (G::rank() == 0) {
      set_err(status, TK_DEV_ERR_RANGE);
      if (info) info->iters = -TK_DEV_ERR_RANGE;
    }
    G::sync();
    return;
  }
  int64_t ctot = 1;
  for (int n = 0; n < tv.p; ++n) ctot *= qb.rq[n];
  S* u0 = out + ctot;
  S* un[TK_MAXP];
  int64_t ldn[TK_MAXP];
  S* cur = u0 + (te - ts) * qb.rq[0];
  for (int n = 1; n < tv.p; ++n) {
    un[n] = cur;
    ldn[n] = qb.rq[n];
    cur += (int64_t)tv.D[n] * qb.rq[n];
  }
  stitch_job<G, S>(tv, ep, TK_JOB_QUERY, ts, te, 0, 0, qb.rq, ws, ws_cap, arena_bytes, out, u0, qb.rq[0], un, ldn,
                   nullptr, info, status, wsm, arena);
}

// Stitch kernel: each CTA repeatedly takes the next job index from the
// launch's queue counter (zeroed by the host before the launch) and runs it.
template <class S, class G>
__global__ void __launch_bounds__(2 * TK_NT) k_stitch(TkTreeView tv, int mode, int level, int64_t k0,
                                                      int njobs, TkQueryBatch qb, TkWorkspace wsd) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = G::rank();
  unsigned char* gsm = smem_raw;
  unsigned char* arena = smem_raw + align16(sizeof(WarpSm<S>));
  WarpSm<S>& sm = *reinterpret_cast<WarpSm<S>*>(gsm);
  S* ws = reinterpret_cast<S*>(wsd.base) + (int64_t)blockIdx.x * wsd.per_cta;
  while (true) {
    if (tid == 0) sm.job = (int)atomicAdd(wsd.counter, 1u);
    G::sync();
    const int job = sm.job;
    G::sync();
    if (job >= njobs) break;
    if (mode == TK_JOB_QUERY) {
      query_job<G, S>(tv, qb, qb.order ? qb.order[job] : job, ws, wsd.per_cta, wsd.smem_arena, wsd.status, gsm,
                      arena);
    } else {
      const int64_t k = k0 + job;
      const int64_t slot = tv.level_base[level] + k;
      S* core = reinterpret_cast<S*>(tv.core_pool) + slot * tv.core_stride;
      S* u0 = reinterpret_cast<S*>(tv.tfac) + level * tv.tfac_level_stride + node_lo_of(tv, level, k) * tv.r[0];
      S* un[TK_MAXP];
      int64_t ldn[TK_MAXP];
      for (int n = 1; n < tv.p; ++n) {
        un[n] = reinterpret_cast<S*>(tv.fac_pool[n]) + slot * tv.fac_stride[n];
        ldn[n] = tv.r[n];
      }
      stitch_job<G, S>(tv, epoch_now(tv), mode, 0, 0, level, k, tv.r, ws, wsd.per_cta, wsd.smem_arena, core, u0,
                       tv.r[0], un, ldn, tv.node_ranks + slot * TK_MAXP, nullptr, wsd.status, gsm, arena);
    }
  }
}

// Batch kernel: one 512-thread CTA per SM, jobs taken longest first from one
// queue (the planned order).  While the queue still holds heavy queries (the
// first *qb.split of the order), a CTA runs each with all 16 warps and a
// shared arena of 2 * smem_arena bytes.  The first light job a CTA draws
// switches it to two independent 256-thread halves (named barriers), each
// with its own header, arena of smem_arena bytes and workspace chunk, each
// drawing light jobs until the queue is empty.  Heavy and light queries thus
// share every SM in the order planned, whatever order the hardware starts
// CTAs in.  Shared memory: [header 0][header 1][arena 2 * smem_arena].
template <class S>
__global__ void __launch_bounds__(2 * TK_NT, 1) k_batch(TkTreeView tv, int njobs, TkQueryBatch qb, TkWorkspace wsd) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const size_t hdr = align16(sizeof(WarpSm<S>));
  unsigned char* arena = smem_raw + 2 * hdr;
  S* ws = reinterpret_cast<S*>(wsd.base) + (int64_t)blockIdx.x * 2 * wsd.per_cta;
  WarpSm<S>& sm0 = *reinterpret_cast<WarpSm<S>*>(smem_raw);
  const int split = qb.split ? *qb.split : 0;
  int light = -1;
  while (true) {
    if (threadIdx.x == 0) sm0.job = (int)atomicAdd(wsd.counter, 1u);
    __syncthreads();
    const int job = sm0.job;
    __syncthreads();
    if (job >= njobs) return;
    if (job >= split) {
      light = job;
      break;
    }
    query_job<BlockGroup, S>(tv, qb, qb.order ? qb.order[job] : job, ws, wsd.per_cta, 2 * wsd.smem_arena,
                             wsd.status, smem_raw, arena);
  }
  // two halves from here on; half 0 starts with the light job already drawn
  const int h = HalfGroup::half();
  unsigned char* hsm = smem_raw + h * hdr;
  WarpSm<S>& sm = *reinterpret_cast<WarpSm<S>*>(hsm);
  unsigned char* harena = arena + h * wsd.smem_arena;
  S* hws = ws + h * wsd.per_cta;
  int job = h == 0 ? light : -1;
  while (true) {
    if (job < 0) {
      if (HalfGroup::rank() == 0) sm.job = (int)atomicAdd(wsd.counter, 1u);
      HalfGroup::sync();
      job = sm.job;
      HalfGroup::sync();
    }
    if (job >= njobs) break;
    query_job<HalfGroup, S>(tv, qb, qb.order ? qb.order[job] : job, hws, wsd.per_cta, wsd.smem_arena, wsd.status,
                            hsm, harena);
    job = -1;
  }
}

}  // namespace tk
