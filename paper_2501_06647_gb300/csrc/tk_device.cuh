// Block-cooperative building blocks for the small dense linear algebra of a
// stitch or leaf job.  Every routine is called by all threads of the CTA,
// works on plain pointers (shared or global memory), uses a fixed reduction
// order (so repeated runs are bit-identical) and ends with __syncthreads().
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tk {

template <class S> struct Eps;
template <> struct Eps<double> { static __device__ __forceinline__ double v() { return 2.220446049250313e-16; } };
template <> struct Eps<float> { static __device__ __forceinline__ float v() { return 1.1920929e-7f; } };

template <class S> __device__ __forceinline__ S warp_sum(S v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of one value per thread; every thread gets the total.  red: >= 33 S.
template <class S> __device__ S block_sum(S v, S* red) {
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
  S r = red[32];
  __syncthreads();
  return r;
}

template <class S> __device__ S sum_squares(const S* x, int64_t n, S* red) {
  S a = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a += x[i] * x[i];
  return block_sum(a, red);
}

__device__ __forceinline__ int64_t prod_range(const int* d, int a, int b) {
  int64_t p = 1;
  for (int m = a; m < b; ++m) p *= d[m];
  return p;
}

// Mode-n product of a C-order tensor X (dims d[0..p-1]) with a matrix M of
// shape a x d[n], M(alpha, j) = M[alpha*mrs + j*mcs]:
//   Y[o, alpha, i] = sum_j M(alpha, j) X[o, j, i]   (Appendix A: mat_n(Y) = M mat_n(X)).
// Y has dims d with d[n] replaced by a.  accumulate: Y += result.
template <class S>
__device__ void ttm(const S* X, const int* d, int p, int n, const S* M, int64_t mrs, int64_t mcs,
                    int a, S* Y, bool accumulate) {
  const int64_t outer = prod_range(d, 0, n), inner = prod_range(d, n + 1, p);
  const int dn = d[n];
  const int64_t total = outer * a * inner;
  for (int64_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int64_t i = idx % inner;
    const int64_t t = idx / inner;
    const int al = (int)(t % a);
    const int64_t o = t / a;
    const S* xp = X + o * dn * inner + i;
    const S* mp = M + al * mrs;
    S acc = 0;
    for (int j = 0; j < dn; ++j) acc += mp[j * mcs] * xp[j * inner];
    if (accumulate) Y[idx] += acc; else Y[idx] = acc;
  }
  __syncthreads();
}

// Mode-n Gram mat_n(X) mat_n(X)^T (d[n] x d[n], leading dimension lda).
template <class S>
__device__ void mode_gram(const S* X, const int* d, int p, int n, S* A, int lda, bool accumulate) {
  const int64_t outer = prod_range(d, 0, n), inner = prod_range(d, n + 1, p);
  const int dn = d[n];
  for (int idx = threadIdx.x; idx < dn * dn; idx += blockDim.x) {
    const int a = idx / dn, b = idx % dn;
    if (a > b) continue;
    S acc = 0;
    for (int64_t o = 0; o < outer; ++o) {
      const S* pa = X + (o * dn + a) * inner;
      const S* pb = X + (o * dn + b) * inner;
      for (int64_t i = 0; i < inner; ++i) acc += pa[i] * pb[i];
    }
    if (accumulate) {
      A[a * lda + b] += acc;
      if (a != b) A[b * lda + a] += acc;
    } else {
      A[a * lda + b] = acc;
      A[b * lda + a] = acc;
    }
  }
  __syncthreads();
}

// C (M x N) = A (M x K) * B (K x N) with general strides; beta = 0 or 1.
template <class S>
__device__ void gemm(int M, int N, int K, const S* A, int64_t ars, int64_t acs, const S* B,
                     int64_t brs, int64_t bcs, S* C, int64_t crs, int64_t ccs, bool accumulate) {
  for (int64_t idx = threadIdx.x; idx < (int64_t)M * N; idx += blockDim.x) {
    const int i = (int)(idx / N), j = (int)(idx % N);
    S acc = 0;
    for (int k = 0; k < K; ++k) acc += A[i * ars + k * acs] * B[k * brs + j * bcs];
    if (accumulate) C[i * crs + j * ccs] += acc; else C[i * crs + j * ccs] = acc;
  }
  __syncthreads();
}

// Householder QR of the row-major m x n matrix A (leading dimension lda), in
// place (Golub & Van Loan, Algorithm 5.2.1, with LAPACK's dlarfg convention):
// on return the upper triangle holds R (min(m,n) x n) and the part below the
// diagonal holds the reflector vectors v_j (v_j[j] = 1 implicit), with
// H_j = I - tau_j v_j v_j^T and A_in = H_0 H_1 ... H_{k-1} R.  tau: min(m,n).
// sc: >= 3 S of shared scratch.
template <class S>
__device__ void householder_qr(S* A, int m, int n, int64_t lda, S* tau, S* sc) {
  const int kmax = m < n ? m : n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
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
    __syncthreads();
    const S t = sc[0], scale = sc[1], beta = sc[2];
    if (t != S(0)) {
      for (int i = j + 1 + (int)threadIdx.x; i < m; i += blockDim.x) A[i * lda + j] *= scale;
      __syncthreads();
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
    __syncthreads();
    if (threadIdx.x == 0) A[j * lda + j] = beta;
    __syncthreads();
  }
}

// Y (m x ncols, leading dimension ldy) <- H_0 H_1 ... H_{k-1} Y, the Q factor
// of householder_qr applied to Y.  To form Q [E; 0], fill Y with E on its
// first rows and zeros below before the call.
template <class S>
__device__ void householder_apply_q(const S* A, int m, int kmax, int64_t lda, const S* tau, S* Y,
                                    int ncols, int64_t ldy) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
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
    __syncthreads();
  }
}

// Shared scratch of jacobi_eig for order n: pairs of the round-robin schedule.
struct JacobiScratch {
  int* pq;    // >= n/2+1
  int* flag;  // 1
};

// Symmetric eigendecomposition of the n x n matrix A (leading dimension lda)
// by the cyclic two-sided Jacobi method with the round-robin parallel
// ordering (Golub & Van Loan, Sections 8.5.2-8.5.5: every round applies n/2
// disjoint rotations J(p,q) with the Rutishauser formula of Algorithm 8.5.1,
// A <- J^T A J, V <- V J).  A is destroyed (its diagonal ends as the
// eigenvalues, copied to w); V (ldv) receives the eigenvectors as columns.
// A rotation is skipped when |a_pq| <= eps sqrt(|a_pp a_qq|) or
// |a_pq| <= 1e-3 eps ||A||_F; the sweep loop stops when a whole sweep skips
// every rotation or after max_sweeps.  Returns the number of sweeps run.
template <class S>
__device__ int jacobi_eig(int n, S* A, int64_t lda, S* V, int64_t ldv, S* w, S* cs, JacobiScratch js,
                          S* red, int max_sweeps) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int idx = tid; idx < n * n; idx += nt) {
    const int i = idx / n, j = idx % n;
    V[i * ldv + j] = (i == j) ? S(1) : S(0);
  }
  S a2 = 0;
  for (int idx = tid; idx < n * n; idx += nt) {
    const S v = A[(idx / n) * lda + (idx % n)];
    a2 += v * v;
  }
  const S normA = sqrt(block_sum(a2, red));
  const S eps = Eps<S>::v();
  const S floor_abs = S(1e-3) * eps * normA;
  const int m = n + (n & 1), half = m / 2;
  S* cc = cs;
  S* ss = cs + half + 1;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) *js.flag = 0;
    __syncthreads();
    for (int rd = 0; rd < m - 1; ++rd) {
      for (int k = tid; k < half; k += nt) {
        int a, b;
        if (k == 0) {
          a = rd;
          b = m - 1;
        } else {
          a = (rd + k) % (m - 1);
          b = (rd - k + m - 1) % (m - 1);
        }
        const int pp = a < b ? a : b, qq = a < b ? b : a;
        int code = -1;
        S c = 1, s = 0;
        if (qq < n) {
          const S apq = A[pp * lda + qq];
          const S app = A[pp * lda + pp], aqq = A[qq * lda + qq];
          const S aapq = fabs(apq);
          if (aapq > floor_abs && aapq > eps * sqrt(fabs(app * aqq))) {
            const S theta = (aqq - app) / (S(2) * apq);
            S t;
            if (fabs(theta) > S(1e15)) t = S(0.5) / theta;
            else t = (theta >= S(0) ? S(1) : S(-1)) / (fabs(theta) + sqrt(S(1) + theta * theta));
            c = S(1) / sqrt(S(1) + t * t);
            s = t * c;
            code = pp | (qq << 16);
            *js.flag = 1;
          }
        }
        js.pq[k] = code;
        cc[k] = c;
        ss[k] = s;
      }
      __syncthreads();
      for (int idx = tid; idx < half * n; idx += nt) {
        const int k = idx / n, j = idx % n;
        const int code = js.pq[k];
        if (code < 0) continue;
        const int pp = code & 0xffff, qq = code >> 16;
        const S c = cc[k], s = ss[k];
        const S apj = A[pp * lda + j], aqj = A[qq * lda + j];
        A[pp * lda + j] = c * apj - s * aqj;
        A[qq * lda + j] = s * apj + c * aqj;
      }
      __syncthreads();
      for (int idx = tid; idx < half * n; idx += nt) {
        const int k = idx / n, i = idx % n;
        const int code = js.pq[k];
        if (code < 0) continue;
        const int pp = code & 0xffff, qq = code >> 16;
        const S c = cc[k], s = ss[k];
        const S aip = A[i * lda + pp], aiq = A[i * lda + qq];
        S nip = c * aip - s * aiq, niq = s * aip + c * aiq;
        if (i == pp) niq = 0;
        if (i == qq) nip = 0;
        A[i * lda + pp] = nip;
        A[i * lda + qq] = niq;
        const S vip = V[i * ldv + pp], viq = V[i * ldv + qq];
        V[i * ldv + pp] = c * vip - s * viq;
        V[i * ldv + qq] = s * vip + c * viq;
      }
      __syncthreads();
    }
    const int any = *js.flag;
    __syncthreads();
    if (!any) break;
  }
  for (int i = tid; i < n; i += nt) w[i] = A[i * lda + i];
  __syncthreads();
  return sweep;
}

// E (n x r, leading dimension lde) <- the eigenvectors (columns of V) of the
// r largest eigenvalues w, in descending order (ties by index).
template <class S>
__device__ void select_top(int n, const S* w, const S* V, int64_t ldv, int r, S* E, int64_t lde) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const S wi = w[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const S wj = w[j];
      if (wj > wi || (wj == wi && j < i)) ++rank;
    }
    if (rank < r)
      for (int row = 0; row < n; ++row) E[row * lde + rank] = V[row * ldv + i];
  }
  __syncthreads();
}

}  // namespace tk
