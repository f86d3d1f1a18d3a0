// Tensor-core Gram matrices for the leaf kernel (sm_103a, tcgen05).
//
// gram_tc computes A = sum over a range of columns c of x_c x_c^T for the
// columns x_c (length D <= 256) of a mode-n matricization, the SYRK at the
// heart of the HOSVD start of Tucker-ALS (Section 2).  One CTA:
//   * every thread stages chunks of KC columns into shared memory, in the
//     canonical K-major layout without swizzle that tcgen05 reads through a
//     matrix descriptor (8-row x 16-byte core matrices), converting each
//     value to TF32 (hi) and, for the split form, also its remainder
//     (lo = x - hi, then TF32);
//   * one thread issues tcgen05.mma.kind::tf32 (M = 128 rows of the Gram per
//     tile, N = D rounded up to 16), FP32 accumulation in tensor memory;
//     split form: hi*hi^T + hi*lo^T + lo*hi^T, which keeps FP32 accuracy;
//   * chunks are double-buffered: tcgen05.commit arrives on an mbarrier
//     when the MMAs that read a buffer are done, and the buffer is refilled
//     only after that (every wait is bounded: on a timeout the status is set
//     and the remaining work is skipped, barriers still reached);
//   * the accumulator is read back with tcgen05.ld (each warp of the first
//     four reads its 32 lanes) and written to A (D x D, lda).
#pragma once
#include <cstdint>

#include "tk_internal.h"

namespace tk {

constexpr int kTcMaxD = 256;      // largest Gram order of this path
constexpr int kTcSBO = 128;       // bytes between 8-row groups (M/N direction)
constexpr int kTcTmemCols = 512;  // two 128 x 256 FP32 accumulators
constexpr int kTcItems = 4;       // staged float4 items per thread and chunk (at most)
constexpr long long kTcSpin = 1ll << 26;  // bound on every mbarrier wait (~1 s)

// Staged rows of an operand tile for Gram order D (one or two M-tiles of 128).
__host__ __device__ inline int tc_rows(int D) { return D > 128 ? 256 : 128; }
// Bytes between core-matrix columns (K direction): a column of rows x 16 B,
// plus 16 B so that a warp writing 32 consecutive k of one row hits 32 banks.
__host__ __device__ inline int tc_lbo(int D) { return tc_rows(D) * 16 + 16; }
// Columns per staged chunk for order D in `bytes` of staging shared memory
// (two buffers of hi and lo tiles), a multiple of 8, at most 64; 0 if none fits.
__host__ __device__ inline int tc_chunk(int D, int64_t bytes, int threads) {
  int kc = 64;
  while (kc >= 8 && ((int64_t)4 * (kc / 4) * tc_lbo(D) > bytes || D * (kc / 4) > kTcItems * threads)) kc -= 8;
  return kc >= 8 ? kc : 0;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// TF32 value of x (round to nearest, ties away), as an FP32 bit pattern
// whose 13 low mantissa bits are cleared, so that it is exactly the value
// the tensor core multiplies and x - to_tf32(x) is the exact remainder.
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r & 0xFFFFE000u);
}

// Shared-memory matrix descriptor: K-major, no swizzle, core-matrix columns
// lbo bytes apart.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, int lbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((kTcSBO >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture
  return d;                // base offset 0, swizzle none
}

// Instruction descriptor: kind::tf32, FP32 accumulator, A and B K-major, M x N.
__device__ __forceinline__ uint32_t tc_idesc(int M, int N) {
  uint32_t d = 0;
  d |= 1u << 4;                       // D format F32
  d |= 2u << 7;                       // A format TF32
  d |= 2u << 10;                      // B format TF32
  d |= (uint32_t)(N >> 3) << 17;
  d |= (uint32_t)(M >> 4) << 24;
  return d;
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}

// Wait until the mbarrier's phase `parity` has completed; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity) {
  const uint32_t a = smem_u32(mbar);
  for (long long i = 0; i < kTcSpin; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Tensor memory of the CTA: allocated by warp 0 (the address is written to
// *slot), released by warp 0 at the end.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, int ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, int ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 16 consecutive FP32 columns of this thread's lane (32x32b shape).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row m, column k) of a staged operand tile.
__device__ __forceinline__ int tc_off(int m, int k, int lbo) {
  return (m >> 3) * kTcSBO + (m & 7) * 16 + (k >> 2) * lbo + (k & 3) * 4;
}

// State of the tensor-core path in a CTA: its tensor memory and mbarriers.
struct TcState {
  uint32_t tmem;       // base address of kTcTmemCols columns
  uint64_t* mbar;      // two mbarriers (one per staging buffer), in shared memory
  uint32_t phase[2];   // next parity to wait for, per buffer
  int pending[2];      // an MMA group that reads the buffer is in flight
  int failed;          // a wait timed out: no more tensor-core work in this launch
};

// A (D x D, lda) = sum over columns c in [c0, c1) of x_c x_c^T, x_c[a] =
// X[(o D + a) inner + i], c = o inner + i (the columns of the mode-n
// matricization of a C-order tensor seen as (outer, D, inner)), D <= 256.
// split: the three-product split-TF32 form (FP32 accuracy), else plain TF32.
// stage: `stage_bytes` of 16-byte aligned shared memory, kc columns per chunk
// (tc_chunk).  Executed by the whole CTA (blockDim.x a multiple of 128, at
// most 512).  Returns false (on every thread) if the path failed; the status
// word is then set and A is not written.
static __device__ bool gram_tc(const float* X, int D, int64_t inner, int64_t c0, int64_t c1, float* A, int lda,
                        unsigned char* stage, int kc, TcState& st, bool split, int* status) {
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31;
  const int N = (D + 15) & ~15;
  const int nmt = D > 128 ? 2 : 1;
  const int lbo = tc_lbo(D);
  const int tile = (kc / 4) * lbo;  // bytes of one operand tile (hi or lo)
  const int g4 = kc / 4;
  const int items = D * g4;
  const uint32_t idesc = tc_idesc(128, N);
  const int64_t nchunk = (c1 - c0 + kc - 1) / kc;
  __shared__ int s_fail;
  if (tid == 0) s_fail = st.failed;
  __syncthreads();
  if (s_fail) return false;

  float v[kTcItems][4];
  auto load = [&](int64_t ch) {
    const int64_t cb = c0 + ch * kc;
    const int kk = (int)((c1 - cb) < kc ? (c1 - cb) : kc);
#pragma unroll
    for (int u = 0; u < kTcItems; ++u) {
      const int it = tid + u * nt;
      int a, g;
      if (inner == 1) {  // consecutive threads: consecutive rows (coalesced along a)
        a = it % D;
        g = it / D;
      } else {           // consecutive threads: consecutive column groups (coalesced along i)
        g = it % g4;
        a = it / g4;
      }
      const bool on = it < items;
      int64_t c = cb + 4 * g, o = 0, i = 0;
      if (on && inner > 1) {
        o = c / inner;
        i = c - o * inner;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float x = 0.f;
        if (on && 4 * g + q < kk) x = inner == 1 ? X[(c + q) * D + a] : X[(o * D + a) * inner + i];
        v[u][q] = x;
        if (inner > 1 && ++i == inner) {
          i = 0;
          ++o;
        }
      }
    }
  };
  auto store = [&](unsigned char* hi, unsigned char* lo) {
#pragma unroll
    for (int u = 0; u < kTcItems; ++u) {
      const int it = tid + u * nt;
      if (it >= items) continue;
      const int a = inner == 1 ? it % D : it / g4, g = inner == 1 ? it / D : it % g4;
      float4 h;
      h.x = to_tf32(v[u][0]); h.y = to_tf32(v[u][1]); h.z = to_tf32(v[u][2]); h.w = to_tf32(v[u][3]);
      *reinterpret_cast<float4*>(hi + tc_off(a, 4 * g, lbo)) = h;
      if (split) {
        float4 l;
        l.x = to_tf32(v[u][0] - h.x); l.y = to_tf32(v[u][1] - h.y);
        l.z = to_tf32(v[u][2] - h.z); l.w = to_tf32(v[u][3] - h.w);
        *reinterpret_cast<float4*>(lo + tc_off(a, 4 * g, lbo)) = l;
      }
    }
  };

  if (nchunk > 0) load(0);
  for (int64_t ch = 0; ch < nchunk; ++ch) {
    const int b = (int)(ch & 1);
    unsigned char* hi = stage + b * 2 * tile;
    unsigned char* lo = hi + tile;
    // the buffer is refilled once the MMAs that read it have completed
    if (st.pending[b]) {
      if (!mbar_wait(st.mbar + b, st.phase[b])) s_fail = 1;
      st.phase[b] ^= 1u;
      st.pending[b] = 0;
    }
    tc_fence_after();
    store(hi, lo);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    const bool issue = s_fail == 0;
    if (tid == 0 && issue) {
      tc_fence_after();
      const uint32_t sh = smem_u32(hi), sl = smem_u32(lo);
      for (int ks = 0; ks < kc / 8; ++ks) {
        const uint32_t koff = ks * 2 * lbo;  // 8 columns = two core-matrix columns
        for (int mt = 0; mt < nmt; ++mt) {
          const uint32_t d = st.tmem + mt * 256;
          const uint32_t moff = mt * (128 / 8) * kTcSBO;  // 128 rows = 16 row groups
          const int acc = (ch == 0 && ks == 0) ? 0 : 1;
          tc_mma(d, tc_desc(sh + koff + moff, lbo), tc_desc(sh + koff, lbo), idesc, acc);
          if (split) {
            tc_mma(d, tc_desc(sh + koff + moff, lbo), tc_desc(sl + koff, lbo), idesc, 1);
            tc_mma(d, tc_desc(sl + koff + moff, lbo), tc_desc(sh + koff, lbo), idesc, 1);
          }
        }
      }
      tc_commit(st.mbar + b);
    }
    st.pending[b] = issue ? 1 : 0;
    if (ch + 1 < nchunk) load(ch + 1);  // in flight while the MMAs run
  }
  // all MMAs done, then the accumulator
  for (int b = 0; b < 2; ++b) {
    if (st.pending[b]) {
      if (!mbar_wait(st.mbar + b, st.phase[b])) s_fail = 1;
      st.phase[b] ^= 1u;
      st.pending[b] = 0;
    }
  }
  tc_fence_after();
  __syncthreads();
  const bool fail = s_fail != 0;
  if (fail) {
    st.failed = 1;
    if (tid == 0) atomicCAS(status, 0, TK_DEV_ERR_WORKSPACE);
  } else if (nchunk == 0) {  // an empty range of columns: the zero matrix
    for (int e = tid; e < D * D; e += nt) A[(int64_t)(e / D) * lda + e % D] = 0.f;
  } else if (warp < 4) {
    // warp w reads tensor-memory lanes [32w, 32w + 32): rows m = 128 mt + 32 w + lane
    for (int mt = 0; mt < nmt; ++mt) {
      const int m = mt * 128 + warp * 32 + lane;
      for (int cc = 0; cc < N; cc += 16) {
        float r[16];
        tmem_ld16(st.tmem + ((uint32_t)(warp * 32) << 16) + mt * 256 + cc, r);
        if (m < D) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (cc + j < D) A[(int64_t)m * lda + cc + j] = r[j];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  return !fail;
}

}  // namespace tk
