// Cooperative building blocks for the small dense linear algebra of a stitch
// or leaf job.  Every routine is executed by all threads of a *group* -- a
// whole CTA (BlockGroup: leaf CTAs, merge and single-query CTAs, heavy
// queries of a batch) or one 256-thread half of a 512-thread CTA (HalfGroup:
// light queries of a batch) -- works on plain pointers (shared or global
// memory), uses a fixed reduction order (so repeated runs are bit-identical)
// and ends with a group barrier.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tk {

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

template <class S> struct Eps;
template <> struct Eps<double> { static __device__ __forceinline__ double v() { return 2.220446049250313e-16; } };
template <> struct Eps<float> { static __device__ __forceinline__ float v() { return 1.1920929e-7f; } };

template <class S> __device__ __forceinline__ S warp_sum(S v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One CTA.  sum() needs >= 33 elements of shared scratch.
struct BlockGroup {
  static __device__ __forceinline__ int rank() { return threadIdx.x; }
  static __device__ __forceinline__ int size() { return blockDim.x; }
  static __device__ __forceinline__ int nwarps() { return blockDim.x >> 5; }
  static __device__ __forceinline__ void sync() { __syncthreads(); }
  template <class S> static __device__ S sum(S v, S* red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
      S x = lane < nw ? red[lane] : S(0);
      x = warp_sum(x);
      if (lane == 0) red[32] = x;
    }
    __syncthreads();
    const S r = red[32];
    __syncthreads();
    return r;
  }
};

// Half of a 512-thread CTA (256 threads) with its own named barrier (ids 1
// and 2; 0 is __syncthreads), so that the two halves run independent jobs.
struct HalfGroup {
  static __device__ __forceinline__ int half() { return threadIdx.x >> 8; }
  static __device__ __forceinline__ int rank() { return threadIdx.x & 255; }
  static __device__ __forceinline__ int size() { return 256; }
  static __device__ __forceinline__ int nwarps() { return 8; }
  static __device__ __forceinline__ void sync() { asm volatile("bar.sync %0, 256;" ::"r"(1 + half()) : "memory"); }
  template <class S> static __device__ S sum(S v, S* red) {
    v = warp_sum(v);
    const int lane = rank() & 31, warp = rank() >> 5;
    sync();
    if (lane == 0) red[warp] = v;
    sync();
    if (warp == 0) {
      S x = lane < 8 ? red[lane] : S(0);
      x = warp_sum(x);
      if (lane == 0) red[32] = x;
    }
    sync();
    const S r = red[32];
    sync();
    return r;
  }
};

template <class G, class S> __device__ S sum_squares(const S* x, int64_t n, S* red) {
  S a = 0;
  for (int64_t i = G::rank(); i < n; i += G::size()) a += x[i] * x[i];
  return G::template sum<S>(a, red);
}

__device__ __forceinline__ int prod_range(const int* d, int a, int b) {
  int p = 1;
  for (int m = a; m < b; ++m) p *= d[m];
  return p;
}

// Mode-n product of a C-order tensor X (dims d[0..p-1]) with a matrix M of
// shape a x d[n], M(alpha, j) = M[alpha*mrs + j*mcs]:
//   Y[o, alpha, i] = sum_j M(alpha, j) X[o, j, i]   (Appendix A: mat_n(Y) = M mat_n(X)).
// Y has dims d with d[n] replaced by a.  accumulate: Y += result.  Each
// thread computes 4 consecutive alpha for one (o, i), so every X element it
// loads feeds 4 FMAs; consecutive threads take consecutive i (coalesced).
template <class G, class S>
__device__ void ttm(const S* X, const int* d, int p, int n, const S* M, int mrs, int mcs, int a, S* Y,
                    bool accumulate) {
  constexpr int CH = 4;
  const int outer = prod_range(d, 0, n), inner = prod_range(d, n + 1, p), dn = d[n];
  const int pairs = outer * inner;
  const int nch = (a + CH - 1) / CH;
  const int total = pairs * nch;
  // element t = ch * pairs + o * inner + i, walked with a stride of G::size()
  // by carries instead of per-element division
  const int nt = G::size();
  const int dch = nt / pairs, dpi = nt - dch * pairs, dout = dpi / inner, din = dpi - dout * inner;
  int t = G::rank();
  int ch = t / pairs, o = (t - ch * pairs) / inner, i = t - ch * pairs - o * inner;
  for (; t < total; t += nt) {
    const int a0 = ch * CH;
    const S* xp = X + (o * dn) * inner + i;
    const S* mp = M + a0 * mrs;
    S acc[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = 0;
    if (a0 + CH <= a) {
      // eight loads of X issued before their FMAs, so that operands in
      // global memory overlap their latency
      int j = 0;
      for (; j + 8 <= dn; j += 8) {
        S x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = xp[(j + u) * inner];
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int c = 0; c < CH; ++c) acc[c] += mp[c * mrs + (j + u) * mcs] * x[u];
      }
      for (; j < dn; ++j) {
        const S x = xp[j * inner];
#pragma unroll
        for (int c = 0; c < CH; ++c) acc[c] += mp[c * mrs + j * mcs] * x;
      }
    } else {
      for (int j = 0; j < dn; ++j) {
        const S x = xp[j * inner];
#pragma unroll
        for (int c = 0; c < CH; ++c)
          if (a0 + c < a) acc[c] += mp[c * mrs + j * mcs] * x;
      }
    }
    S* yp = Y + (o * a + a0) * inner + i;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      if (a0 + c < a) {
        if (accumulate) yp[c * inner] += acc[c];
        else yp[c * inner] = acc[c];
      }
    }
    i += din;
    o += dout;
    ch += dch;
    if (i >= inner) {
      i -= inner;
      ++o;
    }
    if (o >= outer) {
      o -= outer;
      ++ch;
    }
  }
  G::sync();
}

// Mode-n Gram mat_n(X) mat_n(X)^T (d[n] x d[n], leading dimension lda); each
// thread takes one (a, b) with a <= b of the packed upper triangle.
template <class G, class S>
__device__ void mode_gram(const S* X, const int* d, int p, int n, S* A, int lda, bool accumulate) {
  const int outer = prod_range(d, 0, n), inner = prod_range(d, n + 1, p), dn = d[n];
  const int npairs = dn * (dn + 1) / 2;
  const int nt = G::size();
  int idx = G::rank();
  if (idx < npairs) {  // no early return: every thread must reach the one barrier below
    // row a of the packed upper triangle: idx in [a(2dn-a+1)/2, (a+1)(2dn-a)/2)
    int a = (int)((2.f * dn + 1.f - sqrtf((2.f * dn + 1.f) * (2.f * dn + 1.f) - 8.f * idx)) * 0.5f);
    if (a < 0) a = 0;
    while (a > 0 && a * (2 * dn - a + 1) / 2 > idx) --a;
    while ((a + 1) * (2 * dn - a) / 2 <= idx) ++a;
    int b = idx - a * (2 * dn - a + 1) / 2 + a;
    for (; idx < npairs; idx += nt) {
      S acc = 0;
      for (int o = 0; o < outer; ++o) {
        const S* pa = X + (o * dn + a) * inner;
        const S* pb = X + (o * dn + b) * inner;
        int i = 0;
        for (; i + 4 <= inner; i += 4) {
          S xa[4], xb[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            xa[u] = pa[i + u];
            xb[u] = pb[i + u];
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) acc += xa[u] * xb[u];
        }
        for (; i < inner; ++i) acc += pa[i] * pb[i];
      }
      if (accumulate) {
        A[a * lda + b] += acc;
        if (a != b) A[b * lda + a] += acc;
      } else {
        A[a * lda + b] = acc;
        A[b * lda + a] = acc;
      }
      // advance nt positions along the packed rows (row a holds columns a..dn-1)
      b += nt;
      while (b >= dn && a < dn - 1) {
        b -= dn - (a + 1);
        ++a;
      }
    }
  }
  G::sync();
}

// A (n x n, lda) += P Q^T for P, Q of n x k (row-major, leading dimensions
// ldp, ldq) whose product is symmetric in exact arithmetic: each entry a <= b
// is computed once and written to (a, b) and (b, a), so A stays exactly
// symmetric.  One thread per entry of the packed upper triangle.
template <class G, class S>
__device__ void sym_accum(int n, int k, const S* P, int ldp, const S* Q, int ldq, S* A, int lda) {
  const int npairs = n * (n + 1) / 2;
  for (int idx = G::rank(); idx < npairs; idx += G::size()) {
    int a = (int)((2.f * n + 1.f - sqrtf((2.f * n + 1.f) * (2.f * n + 1.f) - 8.f * idx)) * 0.5f);
    if (a < 0) a = 0;
    while (a > 0 && a * (2 * n - a + 1) / 2 > idx) --a;
    while ((a + 1) * (2 * n - a) / 2 <= idx) ++a;
    const int b = idx - a * (2 * n - a + 1) / 2 + a;
    S acc = 0;
    for (int t = 0; t < k; ++t) acc += P[a * ldp + t] * Q[b * ldq + t];
    A[a * lda + b] += acc;
    if (a != b) A[b * lda + a] += acc;
  }
  G::sync();
}

// C (M x N) = A (M x K) * B (K x N) with general strides; accumulate: C +=.
template <class G, class S>
__device__ void gemm(int M, int N, int K, const S* A, int ars, int acs, const S* B, int brs, int bcs, S* C,
                     int64_t crs, int ccs, bool accumulate) {
  const int nt = G::size();
  const int di = nt / N, dj = nt - di * N;
  int idx = G::rank();
  int i = idx / N, j = idx - (idx / N) * N;
  for (; idx < M * N; idx += nt) {
    S acc = 0;
    int k = 0;
    for (; k + 4 <= K; k += 4) {
      S xa[4], xb[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        xa[u] = A[i * ars + (k + u) * acs];
        xb[u] = B[(k + u) * brs + j * bcs];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) acc += xa[u] * xb[u];
    }
    for (; k < K; ++k) acc += A[i * ars + k * acs] * B[k * brs + j * bcs];
    if (accumulate) C[i * crs + j * ccs] += acc;
    else C[i * crs + j * ccs] = acc;
    j += dj;
    i += di;
    if (j >= N) {
      j -= N;
      ++i;
    }
  }
  G::sync();
}

// Applies the reflector H = I - tau v v^T, v = (1, A[r0+1..m-1][j]) (column
// j of A below row r0), to columns [0, nc) of B (rows r0..m-1, leading
// dimension ldb): w_c = tau (B[r0][c] + sum_{i>r0} v_i B[i][c]), then
// B[r0][c] -= w_c and B[i][c] -= w_c v_i.  Every thread of the group takes a
// share of the rows and accumulates the dot products of up to 16 columns at
// once; one reduction then serves all of them.  For tall matrices (m much
// larger than the CTA), where one warp per column would walk the rows alone.
// wbuf: >= 16 * (nwarps + 1) elements of shared scratch.
template <class G, class S>
__device__ void reflect_cols(const S* A, int lda, int j, int r0, int m, S tau, S* B, int64_t ldb, int nc, S* wbuf) {
  const int tid = G::rank(), nt = G::size(), lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  S* wfin = wbuf + 16 * nw;
  for (int c0 = 0; c0 < nc; c0 += 16) {
    const int cw = nc - c0 < 16 ? nc - c0 : 16;
    S acc[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = S(0);
    for (int i = r0 + 1 + tid; i < m; i += nt) {
      const S vi = A[(int64_t)i * lda + j];
      const S* bp = B + i * ldb + c0;
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (c < cw) acc[c] += vi * bp[c];
    }
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = warp_sum(acc[c]);
    if (lane == 0)
      for (int c = 0; c < cw; ++c) wbuf[warp * 16 + c] = acc[c];
    G::sync();
    if (tid < cw) {
      S w = B[r0 * ldb + c0 + tid];
      for (int q = 0; q < nw; ++q) w += wbuf[q * 16 + tid];
      w *= tau;
      wfin[tid] = w;
      B[r0 * ldb + c0 + tid] -= w;
    }
    G::sync();
    for (int i = r0 + 1 + tid; i < m; i += nt) {
      const S vi = A[(int64_t)i * lda + j];
      S* bp = B + i * ldb + c0;
      for (int c = 0; c < cw; ++c) bp[c] -= wfin[c] * vi;
    }
    G::sync();
  }
}

// Householder QR of the row-major m x n matrix A (leading dimension lda), in
// place (Golub & Van Loan, Algorithm 5.2.1, with LAPACK's dlarfg convention):
// on return the upper triangle holds R (min(m,n) x n) and the part below the
// diagonal holds the reflector vectors v_j (v_j[j] = 1 implicit), with
// H_j = I - tau_j v_j v_j^T and A_in = H_0 H_1 ... H_{k-1} R.  tau: min(m,n).
// sc: >= 3 S of group-private shared scratch.
template <class G, class S>
__device__ void householder_qr(S* A, int m, int n, int lda, S* tau, S* sc, S* red = nullptr, S* wbuf = nullptr) {
  const int kmax = m < n ? m : n;
  const int lane = G::rank() & 31, warp = G::rank() >> 5, nw = G::nwarps();
  if (wbuf && G::nwarps() > 1 && m >= 2 * G::size()) {
    // tall: every thread takes part in every reduction (reflect_cols)
    for (int j = 0; j < kmax; ++j) {
      S s = 0;
      for (int i = j + 1 + G::rank(); i < m; i += G::size()) {
        const S v = A[(int64_t)i * lda + j];
        s += v * v;
      }
      s = G::template sum<S>(s, red);
      if (G::rank() == 0) {
        const S x0 = A[(int64_t)j * lda + j];
        S t = 0, beta = x0, scale = 0;
        if (s != S(0)) {
          const S nrm = sqrt(x0 * x0 + s);
          beta = x0 >= S(0) ? -nrm : nrm;
          t = (beta - x0) / beta;
          scale = S(1) / (x0 - beta);
        }
        sc[0] = t;
        sc[1] = scale;
        sc[2] = beta;
        tau[j] = t;
      }
      G::sync();
      const S t = sc[0], scale = sc[1], beta = sc[2];
      if (t != S(0)) {
        for (int i = j + 1 + G::rank(); i < m; i += G::size()) A[(int64_t)i * lda + j] *= scale;
        G::sync();
        reflect_cols<G, S>(A, lda, j, j, m, t, A + j + 1, lda, n - j - 1, wbuf);
      }
      if (G::rank() == 0) A[(int64_t)j * lda + j] = beta;
      G::sync();
    }
    return;
  }
  for (int j = 0; j < kmax; ++j) {
    if (warp == 0) {
      S s = 0;
      for (int i = j + 1 + lane; i < m; i += 32) {
        const S v = A[i * lda + j];
        s += v * v;
      }
      s = warp_sum(s);
      if (lane == 0) {
        const S x0 = A[j * lda + j];
        S t = 0, beta = x0, scale = 0;
        if (s != S(0)) {
          const S nrm = sqrt(x0 * x0 + s);
          beta = x0 >= S(0) ? -nrm : nrm;
          t = (beta - x0) / beta;
          scale = S(1) / (x0 - beta);
        }
        sc[0] = t;
        sc[1] = scale;
        sc[2] = beta;
        tau[j] = t;
      }
    }
    G::sync();
    const S t = sc[0], scale = sc[1], beta = sc[2];
    if (t != S(0)) {
      for (int i = j + 1 + G::rank(); i < m; i += G::size()) A[i * lda + j] *= scale;
      G::sync();
      for (int k = j + 1 + warp; k < n; k += nw) {
        S w = 0;
        for (int i = j + 1 + lane; i < m; i += 32) w += A[i * lda + j] * A[i * lda + k];
        w = warp_sum(w);
        w = (w + A[j * lda + k]) * t;
        __syncwarp();
        if (lane == 0) A[j * lda + k] -= w;
        for (int i = j + 1 + lane; i < m; i += 32) A[i * lda + k] -= w * A[i * lda + j];
      }
    }
    G::sync();
    if (G::rank() == 0) A[j * lda + j] = beta;
    G::sync();
  }
}

// Y (m x ncols, leading dimension ldy) <- H_0 H_1 ... H_{k-1} Y, the Q factor
// of householder_qr applied to Y.  To form Q [E; 0], fill Y with E on its
// first rows and zeros below before the call.
template <class G, class S>
__device__ void householder_apply_q(const S* A, int m, int kmax, int lda, const S* tau, S* Y, int ncols,
                                    int64_t ldy, S* wbuf = nullptr) {
  const int lane = G::rank() & 31, warp = G::rank() >> 5, nw = G::nwarps();
  if (wbuf && G::nwarps() > 1 && m >= 2 * G::size()) {
    for (int j = kmax - 1; j >= 0; --j)
      if (tau[j] != S(0)) reflect_cols<G, S>(A, lda, j, j, m, tau[j], Y, ldy, ncols, wbuf);
    return;
  }
  for (int j = kmax - 1; j >= 0; --j) {
    const S t = tau[j];
    if (t == S(0)) continue;
    for (int c = warp; c < ncols; c += nw) {
      S w = 0;
      for (int i = j + 1 + lane; i < m; i += 32) w += A[i * lda + j] * Y[i * ldy + c];
      w = warp_sum(w);
      w = (w + Y[j * ldy + c]) * t;
      __syncwarp();
      if (lane == 0) Y[j * ldy + c] -= w;
      for (int i = j + 1 + lane; i < m; i += 32) Y[i * ldy + c] -= w * A[i * lda + j];
    }
    G::sync();
  }
}

// Scratch of jacobi_eig for order n: the round-robin schedule and rotations.
// Y (m x ncols, leading dimension ldy) <- H_{k-1} ... H_1 H_0 Y: the transpose
// of householder_apply_q's product (Q^T Y for the Q of householder_qr).
template <class G, class S>
__device__ void householder_apply_qt(const S* A, int m, int kmax, int lda, const S* tau, S* Y, int ncols,
                                     int64_t ldy, S* wbuf = nullptr) {
  const int lane = G::rank() & 31, warp = G::rank() >> 5, nw = G::nwarps();
  if (wbuf && G::nwarps() > 1 && m >= 2 * G::size()) {
    for (int j = 0; j < kmax; ++j)
      if (tau[j] != S(0)) reflect_cols<G, S>(A, lda, j, j, m, tau[j], Y, ldy, ncols, wbuf);
    return;
  }
  for (int j = 0; j < kmax; ++j) {
    const S t = tau[j];
    if (t == S(0)) continue;
    for (int c = warp; c < ncols; c += nw) {
      S w = 0;
      for (int i = j + 1 + lane; i < m; i += 32) w += A[i * lda + j] * Y[i * ldy + c];
      w = warp_sum(w);
      w = (w + Y[j * ldy + c]) * t;
      __syncwarp();
      if (lane == 0) Y[j * ldy + c] -= w;
      for (int i = j + 1 + lane; i < m; i += 32) Y[i * ldy + c] -= w * A[i * lda + j];
    }
    G::sync();
  }
}

// Counter-based Gaussians for the seeded start of Stitch.  splitmix64
// (Steele, Lea and Flood, OOPSLA 2014; the finalizer constants of Vigna's
// public-domain reference): output k of the stream seeded with s is
// mix(s + (k + 1) * 0x9E3779B97F4A7C15).  Uniform k = ((output k >> 11) + 1)
// * 2^-53 in (0, 1].  Gaussian e by Box-Muller (1958) on uniforms 2(e/2) and
// 2(e/2) + 1: sqrt(-2 ln u1) cos(2 pi u2) for even e, sin for odd e.  Every
// value depends only on (s, e), so any thread computes any element.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t s, uint64_t k) {
  uint64_t z = s + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double uniform_at(uint64_t s, uint64_t k) {
  return (double)((splitmix64_at(s, k) >> 11) + 1) * 0x1.0p-53;
}
__device__ __forceinline__ double gaussian_at(uint64_t s, uint64_t e) {
  const uint64_t j = e >> 1;
  const double u1 = uniform_at(s, 2 * j), u2 = uniform_at(s, 2 * j + 1);
  const double rad = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);  // sin and cos of 2 pi u2, the argument reduced exactly
  return rad * ((e & 1) ? sn : cs);
}

template <class S> struct JacobiScratch {
  int* pq;    // >= n/2 + 1
  S* c;       // >= n/2 + 1
  S* s;       // >= n/2 + 1
  int* flag;  // 1
  S* red;     // group reduction scratch
  int* nsw;   // 1: sweeps of the last call
  S* thr;     // 1: bottom-block threshold of the current sweep
};

// Symmetric eigendecomposition of the n x n matrix A (leading dimension n)
// by the cyclic two-sided Jacobi method with the round-robin parallel
// ordering (Golub & Van Loan, Sections 8.5.2-8.5.5: every round applies n/2
// disjoint rotations J(p,q) given by the Rutishauser formula of Algorithm
// 8.5.1, A <- J^T A J, V <- V J).
//
// warm: V already holds an orthogonal matrix (the eigenvectors of a nearby
// matrix, e.g. the previous ALS iteration's); A is first replaced by V^T A V
// (through T, n x n scratch) and the sweeps then start from a nearly diagonal
// matrix.  Otherwise V starts as the identity.  Either way, on return V holds
// orthonormal eigenvectors of the input A as columns and w the eigenvalues.
// A rotation is skipped when |a_pq| <= eps sqrt(|a_pp a_qq|) or
// |a_pq| <= eps ||A||_F (an entry at the rounding level of A moves no
// eigenvector by more than rounding).  Cyclic Jacobi converges quadratically,
// so after a sweep in which every rotation had |a_pq| < 0.1 sqrt(eps)
// sqrt(|a_pp a_qq|) the off-diagonal part left is below the rounding level:
// the sweeps stop after such a sweep (its small rotations are applied), or
// after max_sweeps.
//
// Only the r leading eigenvectors are wanted.  A is positive semidefinite
// (a Gram matrix), so |a_pq| <= sqrt(a_pp a_qq) and the block of indices
// whose diagonal lies below thr = sqrt(eps) * (r-th largest diagonal) has all
// its eigenvalues below (n - r) thr: rotations of two such indices move no
// vector of the leading-r invariant subspace, and are skipped (the threshold
// is re-evaluated at the start of every sweep).  Pairs involving any other
// index are still driven to the rounding level.
//
// jacobi_prepare does the warm transform (or V = I) and returns the absolute
// skip floor; jacobi_sweeps runs the sweeps.  Both are executed by group G.
template <class G, class S>
__device__ S jacobi_prepare(int n, S* A, S* V, S* T, bool warm, JacobiScratch<S> js) {
  const int tid = G::rank(), nt = G::size();
  const int nn = n * n;
  if (warm) {
    for (int idx = tid; idx < nn; idx += nt) {  // T = A V
      const int i = idx / n, j = idx % n;
      S acc = 0;
      for (int k = 0; k < n; ++k) acc += A[i * n + k] * V[k * n + j];
      T[idx] = acc;
    }
    G::sync();
    for (int idx = tid; idx < nn; idx += nt) {  // A = V^T T, symmetrized
      const int i = idx / n, j = idx % n;
      if (i > j) continue;
      S acc = 0;
      for (int k = 0; k < n; ++k) acc += V[k * n + i] * T[k * n + j];
      A[i * n + j] = acc;
      A[j * n + i] = acc;
    }
  } else {
    for (int idx = tid; idx < nn; idx += nt) V[idx] = ((idx / n) == (idx % n)) ? S(1) : S(0);
  }
  G::sync();
  S a2 = 0;
  for (int idx = tid; idx < nn; idx += nt) a2 += A[idx] * A[idx];
  return Eps<S>::v() * sqrt(G::template sum<S>(a2, js.red));
}

// Pair k of round rd of the round-robin ordering on m indices (m even):
// pair 0 is (rd, m-1), pair k > 0 is (rd + k, rd - k) modulo m - 1.
__device__ __forceinline__ void rr_pair(int rd, int k, int m, int& pp, int& qq) {
  int a, b;
  if (k == 0) {
    a = rd;
    b = m - 1;
  } else {
    a = rd + k;
    if (a >= m - 1) a -= m - 1;
    b = rd - k;
    if (b < 0) b += m - 1;
  }
  pp = a < b ? a : b;
  qq = a < b ? b : a;
}

// One round applies the n/2 disjoint rotations of its pairs at once: for
// every 2x2 block (pair k's rows, pair l's columns) the new block is
// R_k^T B R_l with R = [c s; -s c] (the row update J^T A followed by the
// column update A J of each rotation), written together with its transpose;
// V's rows are updated by the column rotations.  Each element of A is read
// and written once per round and a round needs two barriers.
template <class G, class S>
__device__ int jacobi_sweeps(int n, int r, S* A, S* V, S floor_abs, S* w, JacobiScratch<S> js, int max_sweeps) {
  const int tid = G::rank(), nt = G::size();
  const S eps = Eps<S>::v();
  const int m = n + (n & 1), half = m / 2;
  const int nblk = half * (half + 1) / 2;
  const S floor2 = floor_abs * floor_abs, eps2 = eps * eps;
  // packed upper triangle of blocks (k <= l): walk start for this thread
  int bk0 = 0, bl0 = 0;
  if (tid < nblk) {
    int a = (int)((2.f * half + 1.f - sqrtf((2.f * half + 1.f) * (2.f * half + 1.f) - 8.f * tid)) * 0.5f);
    if (a < 0) a = 0;
    while (a > 0 && a * (2 * half - a + 1) / 2 > tid) --a;
    while ((a + 1) * (2 * half - a) / 2 <= tid) ++a;
    bk0 = a;
    bl0 = tid - a * (2 * half - a + 1) / 2 + a;
  }
  // (row i, pair l) of V: walk start and stride
  const int vdl = nt / half, vdj = nt - vdl * half;  // element e = i * half + l
  const int vi0 = tid / half, vl0 = tid - (tid / half) * half;
  int sweep = 0;
  const S sqeps = sqrt(eps);
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) {
      *js.flag = 0;
      *js.thr = S(-1);
    }
    G::sync();
    if (r > 0 && r < n) {  // thr = sqrt(eps) * (r-th largest diagonal)
      for (int i = tid; i < n; i += nt) {
        const S di = A[i * n + i];
        int rank = 0;
        for (int j = 0; j < n; ++j) {
          const S dj = A[j * n + j];
          if (dj > di || (dj == di && j < i)) ++rank;
        }
        if (rank == r - 1) *js.thr = sqeps * fabs(di);
      }
      G::sync();
    }
    const S thr = *js.thr;
    for (int rd = 0; rd < m - 1; ++rd) {
      for (int k = tid; k < half; k += nt) {
        int pp, qq;
        rr_pair(rd, k, m, pp, qq);
        S c = 1, s = 0;
        int rot = 0;
        if (qq < n) {
          const S apq = A[pp * n + qq];
          const S app = A[pp * n + pp], aqq = A[qq * n + qq];
          const S apq2 = apq * apq;
          const bool bottom = app < thr && aqq < thr && fabs(apq) < thr;
          if (!bottom && apq2 > floor2 && apq2 > eps2 * fabs(app * aqq)) {
            const S theta = (aqq - app) / (S(2) * apq);
            S t;
            if (fabs(theta) > S(1e15)) t = S(0.5) / theta;
            else t = (theta >= S(0) ? S(1) : S(-1)) / (fabs(theta) + sqrt(S(1) + theta * theta));
            c = S(1) / sqrt(S(1) + t * t);
            s = t * c;
            rot = 1;
            if (apq2 > S(0.01) * eps * fabs(app * aqq)) *js.flag = 1;
          }
        }
        js.pq[k] = pp | (qq << 12) | (rot << 24);
        js.c[k] = c;
        js.s[k] = s;
      }
      G::sync();
      for (int b = tid, k = bk0, l = bl0; b < nblk; b += nt) {
        const int ck = js.pq[k], cl = js.pq[l];
        if ((ck | cl) >> 24) {
          const int pk = ck & 0xfff, qk = (ck >> 12) & 0xfff, pl = cl & 0xfff, ql = (cl >> 12) & 0xfff;
          const S c1 = js.c[k], s1 = js.s[k], c2 = js.c[l], s2 = js.s[l];
          const bool vq = qk < n, vr = ql < n;
          const S b00 = A[pk * n + pl];
          const S b01 = vr ? A[pk * n + ql] : S(0);
          const S b10 = vq ? A[qk * n + pl] : S(0);
          const S b11 = (vq && vr) ? A[qk * n + ql] : S(0);
          // rows: R_k^T B
          const S r00 = c1 * b00 - s1 * b10, r01 = c1 * b01 - s1 * b11;
          const S r10 = s1 * b00 + c1 * b10, r11 = s1 * b01 + c1 * b11;
          // columns: (R_k^T B) R_l
          S n00 = c2 * r00 - s2 * r01, n01 = s2 * r00 + c2 * r01;
          S n10 = c2 * r10 - s2 * r11, n11 = s2 * r10 + c2 * r11;
          if (k == l) {  // the annihilated pair
            if (ck >> 24) n01 = n10 = S(0);
            A[pk * n + pk] = n00;
            if (vq) {
              A[pk * n + qk] = n01;
              A[qk * n + pk] = n10;
              A[qk * n + qk] = n11;
            }
          } else {
            A[pk * n + pl] = n00;
            A[pl * n + pk] = n00;
            if (vr) {
              A[pk * n + ql] = n01;
              A[ql * n + pk] = n01;
            }
            if (vq) {
              A[qk * n + pl] = n10;
              A[pl * n + qk] = n10;
            }
            if (vq && vr) {
              A[qk * n + ql] = n11;
              A[ql * n + qk] = n11;
            }
          }
        }
        l += nt;
        while (l >= half && k < half - 1) {
          l -= half - (k + 1);
          ++k;
        }
      }
      for (int e = tid, i = vi0, l = vl0; e < n * half; e += nt) {
        const int cl = js.pq[l];
        if (cl >> 24) {
          const int pl = cl & 0xfff, ql = (cl >> 12) & 0xfff;
          const S c2 = js.c[l], s2 = js.s[l];
          const S vp = V[i * n + pl], vq = V[i * n + ql];
          V[i * n + pl] = c2 * vp - s2 * vq;
          V[i * n + ql] = s2 * vp + c2 * vq;
        }
        l += vdj;
        i += vdl;
        if (l >= half) {
          l -= half;
          ++i;
        }
      }
      G::sync();
    }
    const int any = *js.flag;
    G::sync();
    if (!any) break;
  }
  for (int i = tid; i < n; i += nt) w[i] = A[i * n + i];
  G::sync();
  return sweep;
}

// The whole eigendecomposition by group G.  Returns the sweeps run.
// r: number of leading eigenvectors the caller keeps (r >= n: all of them).
template <class G, class S>
__device__ int jacobi_eig(int n, int r, S* A, S* V, S* T, bool warm, S* w, JacobiScratch<S> js, int max_sweeps) {
  const S floor_abs = jacobi_prepare<G, S>(n, A, V, T, warm, js);
  return jacobi_sweeps<G, S>(n, r, A, V, floor_abs, w, js, max_sweeps);
}

template <class S> struct Tiny;
template <> struct Tiny<float> { static __device__ __forceinline__ float v() { return 1.1754944e-38f; } };
template <> struct Tiny<double> { static __device__ __forceinline__ double v() { return 2.2250738585072014e-308; } };

// Division in the Sturm recurrence: the count only needs the sign pattern,
// so FP32 uses the fast approximate quotient; FP64 divides exactly.
__device__ __forceinline__ float qdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double qdiv(double a, double b) { return a / b; }

// Orders from which trd_eig replaces the Jacobi method, and its largest r.
constexpr int kTrdMinOrder = 20;
constexpr int kTrdMaxRank = 62;

// Elements of the vector scratch of trd_eig for order n, r vectors and nw
// warps in the group.
__host__ __device__ inline int trd_scratch_elems(int n, int r, int nw) {
  const int wv = nw < r ? nw : r;
  return 7 * n + 2 * r + 8 + r * n + 6 * n * (wv > 0 ? wv : 1);
}

// The r leading eigenpairs of a symmetric n x n matrix A (lda), r <= n,
// r <= kTrdMaxRank, executed by group G:
//   1. Householder tridiagonalization Q^T A Q = T (Golub & Van Loan,
//      Algorithm 8.3.1).  Q = H_0 H_1 ... H_{n-3} is not formed: reflector
//      H_k = I - beta_k v_k v_k^T (v_k zero above row k+1, v_k[k+1] = 1) is
//      kept in row k of A, which the trailing update no longer touches, so
//      that A is the only n x n array (it fits shared memory up to order
//      ~220 in FP32);
//   2. the r largest eigenvalues of T by bisection on Sturm sequence sign
//      counts (Golub & Van Loan, Section 8.4.1), each warp taking two
//      eigenvalues at a time with 32 trial points per step (multisection:
//      each step shrinks the bracket 33-fold), until the bracket is within a
//      few ulps of ||T||;
//   3. their eigenvectors x_j of T by inverse iteration (Golub & Van Loan,
//      Section 8.2.2): two solves with T - lambda_j I, factored by
//      Gaussian elimination with partial pivoting; eigenvalues closer than
//      1e-3 ||T|| form a cluster, whose vectors one warp computes in order,
//      orthogonalizing every iterate against the cluster's earlier ones;
//   4. E = Q X (n x r, leading dimension lde), columns in descending order
//      of the eigenvalues: each warp applies H_{n-3}, ..., H_0 to its own
//      columns of X, with no group barrier between reflectors.
// The trailing matrix-vector product reads A by columns (A is symmetric):
// consecutive threads read consecutive addresses.  A is destroyed.  vec:
// trd_scratch_elems(n, r, G::nwarps()) elements; sc: >= 4 elements; cl: >= 64
// ints, all private to the group.  Every step has a fixed order, so results
// are reproducible.
template <class G, class S>
__device__ void trd_eig(int n, int r, S* A, int lda, S* E, int lde, S* vec, S* sc, int* cl) {
  const int tid = G::rank(), nt = G::size(), lane = tid & 31, warp = tid >> 5, nw = G::nwarps();
  S* d = vec;
  S* e = d + n;
  S* e2 = e + n;
  S* v = e2 + n;   // reflectors of even steps
  S* v2 = v + n;   // and of odd steps (the next one is formed while the current one is applied)
  S* pv = v2 + n;
  S* bet = pv + n;
  S* lam = bet + n;
  S* X = lam + 2 * r + 8;  // r x n, row j = eigenvector j of T
  S* wsc = X + r * n;
  // ---- Householder tridiagonalization ------------------------------------
  // Reflector of step k from row k (= column k below the diagonal, A being
  // symmetric), by warp 0: v_k into vk and into row k, which no later step
  // updates; beta_k, the off-diagonal e[k] and the diagonal d[k].
  auto reflector = [&](int k, S* vk) {
    const int m0 = k + 1;
    S sig = 0;
    for (int i = m0 + 1 + lane; i < n; i += 32) {
      const S x = A[k * lda + i];
      sig += x * x;
    }
    sig = warp_sum(sig);
    const S alpha = A[k * lda + m0];
    __syncwarp();  // every lane has read alpha before row k is overwritten
    S beta = 0, v1 = 1, mu = alpha;
    if (sig > S(0)) {
      mu = sqrt(alpha * alpha + sig);
      v1 = alpha <= S(0) ? alpha - mu : -sig / (alpha + mu);
      beta = S(2) * v1 * v1 / (sig + v1 * v1);
      const S inv = S(1) / v1;
      for (int i = m0 + lane; i < n; i += 32) {
        const S vi = (i == m0) ? S(1) : A[k * lda + i] * inv;
        vk[i] = vi;
        A[k * lda + i] = vi;
      }
    }
    if (lane == 0) {
      bet[k] = beta;
      e[k] = mu;
      d[k] = A[k * lda + k];
    }
  };
  // Two group barriers per step: (matrix-vector product) | (rank-2 update;
  // meanwhile warp 0 updates row k+1 first and forms the next reflector from
  // it, as no other thread touches that row).
  if (warp == 0 && n > 2) reflector(0, v);
  G::sync();
  for (int k = 0; k + 2 < n; ++k) {
    S* vk = (k & 1) ? v2 : v;
    S* vn = (k & 1) ? v : v2;
    const int m0 = k + 1, len = n - m0;
    const bool next = k + 3 < n;
    const S beta = bet[k];
    if (beta == S(0)) {  // the trailing block is unchanged
      if (warp == 0 && next) reflector(k + 1, vn);
      G::sync();
      continue;
    }
    // p = beta A' v on the trailing block A' (rows and columns >= m0); with
    // more threads than rows, g consecutive lanes (a power of two <= 32)
    // share a row and combine by shuffles
    {
      int g = 1;
      while (g < 32 && 2 * g * len <= nt) g *= 2;
      if (g == 1) {
        for (int i = m0 + tid; i < n; i += nt) {
          // eight loads of A issued before their FMAs (A may be in global memory)
          S acc = 0;
          int j = m0;
          for (; j + 8 <= n; j += 8) {
            S a[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] = A[(j + u) * lda + i];
#pragma unroll
            for (int u = 0; u < 8; ++u) acc += a[u] * vk[j + u];
          }
          for (; j < n; ++j) acc += A[j * lda + i] * vk[j];
          pv[i] = beta * acc;
        }
      } else {
        const int row = tid / g, sub = tid & (g - 1);
        const int i = m0 + row;
        S acc0 = 0, acc1 = 0;
        if (row < len) {
          // row i: consecutive lanes, consecutive j; two independent chains
          const S* ar = A + i * lda;
          int j = m0 + sub;
          for (; j + g < n; j += 2 * g) {
            acc0 += ar[j] * vk[j];
            acc1 += ar[j + g] * vk[j + g];
          }
          if (j < n) acc0 += ar[j] * vk[j];
        }
        S acc = acc0 + acc1;
        for (int o = g >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (row < len && sub == 0) pv[i] = beta * acc;
      }
    }
    G::sync();
    // K = beta/2 p^T v (every warp reduces it itself), w = p - K v, and the
    // rank-2 update A' -= v w^T + w v^T, consecutive threads on a row
    S kk = 0;
    for (int i = m0 + lane; i < n; i += 32) kk += pv[i] * vk[i];
    kk = warp_sum(kk) * (beta * S(0.5));
    if (warp == 0 && next) {
      const S vi = vk[m0], wi = pv[m0] - kk * vi;
      for (int j = m0 + lane; j < n; j += 32) {
        const S vj = vk[j], wj = pv[j] - kk * vj;
        A[m0 * lda + j] -= vi * wj + wi * vj;
      }
      __syncwarp();
      reflector(k + 1, vn);
    }
    {
      // rows and columns > m0 when the next step exists (its reflector reads
      // row m0, and column m0 below it is never read again), else the whole
      // trailing block, whose last 2 x 2 entries end the tridiagonal form
      const int lo = next ? m0 + 1 : m0, ln = n - lo;
      const int u0 = (next && nw > 1) ? 32 : 0;
      const int ut = tid - u0, un = nt - u0;
      if (ut >= 0 && ln > 0) {
        const int tot = ln * ln;
        const int di = un / ln, dj = un - di * ln;
        int i = ut / ln, j = ut - (ut / ln) * ln;
        for (int idx = ut; idx < tot; idx += un) {
          const int gi = lo + i, gj = lo + j;
          const S vi = vk[gi], vj = vk[gj];
          const S wi = pv[gi] - kk * vi, wj = pv[gj] - kk * vj;
          A[gi * lda + gj] -= vi * wj + wi * vj;
          j += dj;
          i += di;
          if (j >= ln) {
            j -= ln;
            ++i;
          }
        }
      }
    }
    G::sync();
  }
  if (tid == 0) {
    if (n >= 2) {
      d[n - 2] = A[(n - 2) * lda + (n - 2)];
      e[n - 2] = A[(n - 1) * lda + (n - 2)];
    }
    d[n - 1] = A[(n - 1) * lda + (n - 1)];
    // Gershgorin interval, pivmin
    S gl = d[0], gu = d[0], emax = 0;
    for (int i = 0; i < n; ++i) {
      const S a = i > 0 ? fabs(e[i - 1]) : S(0), b = i + 1 < n ? fabs(e[i]) : S(0);
      gl = fmin(gl, d[i] - a - b);
      gu = fmax(gu, d[i] + a + b);
      if (i + 1 < n) {
        e2[i] = e[i] * e[i];
        emax = fmax(emax, e2[i]);
      }
    }
    const S w = gu - gl;
    gl -= S(2) * Eps<S>::v() * w + Tiny<S>::v();
    gu += S(2) * Eps<S>::v() * w + Tiny<S>::v();
    sc[1] = gl;
    sc[2] = gu;
    sc[3] = Tiny<S>::v() * fmax(S(1), emax);
  }
  G::sync();
  // ---- the r largest eigenvalues: multisection on Sturm counts ----------
  {
    const S gl = sc[1], gu = sc[2], pivmin = sc[3];
    const S tnorm = fmax(fabs(gl), fabs(gu));
    const S conv = S(4) * Eps<S>::v() * tnorm + pivmin;
    // two eigenvalues per warp at a time (j and j + nw): their Sturm
    // recurrences interleave, so each hides the other's latency
    for (int j = warp; j < r; j += 2 * nw) {
      const int j2 = j + nw;
      const int m = n - 1 - j, m2 = n - 1 - j2;  // ascending indices of the j-th, j2-th largest
      S lo = gl, hi = gu, lo2 = gl, hi2 = gu;
      bool act = true, act2 = j2 < r;
      for (int step = 0; step < (sizeof(S) == 8 ? 24 : 12) && (act || act2); ++step) {
        const S x = lo + (hi - lo) * (S)(lane + 1) * (S(1) / S(33));
        const S x2 = lo2 + (hi2 - lo2) * (S)(lane + 1) * (S(1) / S(33));
        int cnt = 0, cnt2 = 0;
        S q = d[0] - x, q2 = d[0] - x2;
        if (fabs(q) < pivmin) q = -pivmin;
        if (fabs(q2) < pivmin) q2 = -pivmin;
        cnt += q < S(0);
        cnt2 += q2 < S(0);
        for (int i = 1; i < n; ++i) {
          const S di = d[i], ei = e2[i - 1];
          q = (di - x) - qdiv(ei, q);
          q2 = (di - x2) - qdiv(ei, q2);
          if (fabs(q) < pivmin) q = -pivmin;
          if (fabs(q2) < pivmin) q2 = -pivmin;
          cnt += q < S(0);
          cnt2 += q2 < S(0);
        }
        if (act) {
          const unsigned ball = __ballot_sync(0xffffffffu, cnt > m);
          const int L = ball ? __ffs(ball) - 1 : 32;
          const S nlo = L == 0 ? lo : lo + (hi - lo) * (S)L * (S(1) / S(33));
          const S nhi = L == 32 ? hi : lo + (hi - lo) * (S)(L + 1) * (S(1) / S(33));
          lo = nlo;
          hi = nhi;
          act = !(hi - lo <= conv);
        }
        if (act2) {
          const unsigned ball = __ballot_sync(0xffffffffu, cnt2 > m2);
          const int L = ball ? __ffs(ball) - 1 : 32;
          const S nlo = L == 0 ? lo2 : lo2 + (hi2 - lo2) * (S)L * (S(1) / S(33));
          const S nhi = L == 32 ? hi2 : lo2 + (hi2 - lo2) * (S)(L + 1) * (S(1) / S(33));
          lo2 = nlo;
          hi2 = nhi;
          act2 = !(hi2 - lo2 <= conv);
        }
      }
      if (lane == 0) {
        lam[j] = S(0.5) * (lo + hi);
        if (j2 < r) lam[j2] = S(0.5) * (lo2 + hi2);
      }
    }
  }
  G::sync();
  // ---- clusters of close eigenvalues (one warp each) ---------------------
  if (tid == 0) {
    const S ctol = S(1e-3) * fmax(fabs(sc[1]), fabs(sc[2]));
    int nc = 0;
    for (int j = 0; j < r; ++j)
      if (j == 0 || lam[j - 1] - lam[j] > ctol) cl[nc++] = j;
    cl[nc] = r;
    cl[63] = nc;
  }
  G::sync();
  const int nclus = cl[63];
  const int nwv = nw < r ? nw : r;
  if (warp < nwv) {
    S* xw = wsc + warp * 6 * n;
    S* ua = xw + n;   // reciprocals of U's diagonal
    S* ub = ua + n;   // first superdiagonal
    S* uc = ub + n;   // second superdiagonal
    S* ml = uc + n;   // multipliers
    S* pf = ml + n;   // pivot flags (1: rows swapped)
    const S tnorm = fmax(fabs(sc[1]), fabs(sc[2]));
    const S small = Eps<S>::v() * tnorm + Tiny<S>::v();
    for (int c = warp; c < nclus; c += nwv) {
      for (int j = cl[c]; j < cl[c + 1]; ++j) {
        // separate equal eigenvalues inside a cluster slightly
        S lj = lam[j];
        if (j > cl[c]) lj = fmin(lj, lam[j - 1] - S(10) * Eps<S>::v() * tnorm);
        if (lane == 0) {
          // LU with partial pivoting of T - lj I (rows i, i+1)
          S a = d[0] - lj, b = n > 1 ? e[0] : S(0);
          for (int i = 0; i < n - 1; ++i) {
            const S sub = e[i], nd = d[i + 1] - lj, ns = i + 2 < n ? e[i + 1] : S(0);
            if (fabs(a) >= fabs(sub)) {
              const S piv = fabs(a) < small ? (a < S(0) ? -small : small) : a;
              const S rp = S(1) / piv;
              const S mlt = sub * rp;
              ua[i] = rp; ub[i] = b; uc[i] = 0; ml[i] = mlt; pf[i] = 0;
              a = nd - mlt * b;
              b = ns;
            } else {
              const S rs = S(1) / sub;
              const S mlt = a * rs;
              ua[i] = rs; ub[i] = nd; uc[i] = ns; ml[i] = mlt; pf[i] = 1;
              a = b - mlt * nd;
              b = -mlt * ns;
            }
          }
          ua[n - 1] = S(1) / (fabs(a) < small ? (a < S(0) ? -small : small) : a);
          ub[n - 1] = 0;
          uc[n - 1] = 0;
        }
        __syncwarp();
        // start vector: deterministic, all components non-zero
        for (int i = lane; i < n; i += 32) xw[i] = S(1) + S(0.5) * (S)((i * 7 + j * 3) % 11) / S(11);
        __syncwarp();
        for (int itr = 0; itr < 2; ++itr) {
          if (lane == 0) {
            // forward: apply the row operations to the right-hand side; the
            // running entry xw[i] stays in a register
            S cur = xw[0];
            for (int i = 0; i < n - 1; ++i) {
              const S nxt = xw[i + 1], mi = ml[i];
              if (pf[i] != S(0)) {
                xw[i] = nxt;
                cur = cur - mi * nxt;
              } else {
                xw[i] = cur;
                cur = nxt - mi * cur;
              }
            }
            xw[n - 1] = cur;
            // back substitution with U (diagonal ua, superdiagonals ub, uc;
            // ub and uc are zero past the last row), x1 = xw[i+1], x2 = xw[i+2]
            S x1 = 0, x2 = 0;
            for (int i = n - 1; i >= 0; --i) {
              const S t = (xw[i] - ub[i] * x1 - uc[i] * x2) * ua[i];
              xw[i] = t;
              x2 = x1;
              x1 = t;
            }
          }
          __syncwarp();
          // orthogonalize against the cluster's earlier vectors, normalize
          for (int jj = cl[c]; jj < j; ++jj) {
            S dot = 0;
            for (int i = lane; i < n; i += 32) dot += X[jj * n + i] * xw[i];
            dot = warp_sum(dot);
            for (int i = lane; i < n; i += 32) xw[i] -= dot * X[jj * n + i];
            __syncwarp();
          }
          S nr = 0;
          for (int i = lane; i < n; i += 32) nr += xw[i] * xw[i];
          nr = warp_sum(nr);
          const S inv = nr > S(0) ? S(1) / sqrt(nr) : S(0);
          for (int i = lane; i < n; i += 32) xw[i] *= inv;
          __syncwarp();
        }
        for (int i = lane; i < n; i += 32) X[j * n + i] = xw[i];
        __syncwarp();
      }
    }
  }
  G::sync();
  // ---- back-transformation E = Q X^T: each warp applies H_{n-3} .. H_0 to
  // its own vectors (up to 4 at a time, held in its scratch) ---------------
  const int vpw = (r + nw - 1) / nw < 4 ? (r + nw - 1) / nw : 4;
  for (int j0 = warp * vpw; j0 < r; j0 += nw * vpw) {
    const int nv = (r - j0) < vpw ? (r - j0) : vpw;
    S* y = wsc + warp * 6 * n;  // nv contiguous vectors of n
    for (int c = 0; c < nv; ++c)
      for (int i = lane; i < n; i += 32) y[c * n + i] = X[(j0 + c) * n + i];
    __syncwarp();
    for (int k = n - 3; k >= 0; --k) {
      const S beta = bet[k];
      if (beta == S(0)) continue;
      const int m0 = k + 1;
      const S* vk = A + k * lda;  // v_k[m0..n), v_k[m0] = 1
      S dot[4] = {S(0), S(0), S(0), S(0)};
      for (int i = m0 + lane; i < n; i += 32) {
        const S vi = vk[i];
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (c < nv) dot[c] += vi * y[c * n + i];
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) dot[c] = warp_sum(dot[c]) * beta;
      for (int i = m0 + lane; i < n; i += 32) {
        const S vi = vk[i];
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (c < nv) y[c * n + i] -= dot[c] * vi;
      }
      __syncwarp();
    }
    for (int c = 0; c < nv; ++c)
      for (int i = lane; i < n; i += 32) E[i * lde + j0 + c] = y[c * n + i];
    __syncwarp();
  }
  G::sync();
}


// E (n x r, leading dimension lde) <- the eigenvectors (columns of V, n x n)
// of the r largest eigenvalues w, in descending order (ties by index).
template <class G, class S>
__device__ void select_top(int n, const S* w, const S* V, int r, S* E, int lde) {
  for (int i = G::rank(); i < n; i += G::size()) {
    const S wi = w[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const S wj = w[j];
      if (wj > wi || (wj == wi && j < i)) ++rank;
    }
    if (rank < r)
      for (int row = 0; row < n; ++row) E[row * lde + rank] = V[row * n + i];
  }
  G::sync();
}

}  // namespace tk
