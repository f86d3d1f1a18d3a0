// Kernels of the range-query Tucker engine: the batch planner, the hit-set
// kernel and the host launchers.  The stitch kernels are defined in
// tk_stitch.cuh and instantiated in tk_stitch_{f32,f64}.cu and
// tk_batch_{f32,f64}.cu; tk_leaf.cu holds the leaf kernel.
#include <cstdio>

#include "tk_stitch.cuh"
#include "tk_inst.h"

namespace tk {

// Longest-first processing order of a query batch: queries sorted by
// decreasing hit-set size (a proxy of their cost: the eigenproblem orders
// grow with it), by a counting sort in one CTA.  Ties keep no particular order;
// the order only schedules work (every query writes its own outputs).
__global__ void k_plan(TkTreeView tv, int n, const int64_t* ranges, const int64_t* tq, int heavy_hits, int* split,
                       int* order) {
  constexpr int NB = TK_MAXH + 1;
  __shared__ int hist[NB];
  __shared__ int base[NB];
  for (int b = threadIdx.x; b < NB; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const TkEpoch ep = (tq && tq[q] <= tv.T) ? epoch_at(tv, tq[q]) : epoch_now(tv);
    int c = recall_count(tv, ep, ranges[2 * q], ranges[2 * q + 1]);
    atomicAdd(&hist[c < NB ? c : NB - 1], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0, heavy = 0;
    for (int b = NB - 1; b >= 0; --b) {
      base[b] = acc;
      acc += hist[b];
      if (b >= heavy_hits) heavy += hist[b];
    }
    *split = heavy;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const TkEpoch ep = (tq && tq[q] <= tv.T) ? epoch_at(tv, tq[q]) : epoch_now(tv);
    int c = recall_count(tv, ep, ranges[2 * q], ranges[2 * q + 1]);
    const int pos = atomicAdd(&base[c < NB ? c : NB - 1], 1);
    order[pos] = q;
  }
}

__global__ void k_hitset(TkTreeView tv, int n, const int64_t* ranges, tk_hit* out, int cap, int* counts) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  HitRec hits[TK_MAXH];
  const int nh = recall_dev(tv, epoch_now(tv), ranges[2 * q], ranges[2 * q + 1], hits, TK_MAXH);
  counts[q] = nh;
  for (int i = 0; i < nh && i < cap; ++i) {
    tk_hit& o = out[(int64_t)q * cap + i];
    o.level = hits[i].level;
    o.partial = hits[i].partial;
    o.index = hits[i].index;
    o.node_lo = hits[i].node_lo;
    o.node_hi = hits[i].node_hi;
    o.lo = hits[i].lo;
    o.hi = hits[i].hi;
  }
}

}  // namespace tk

using namespace tk;

// Dynamic shared bytes of a k_stitch CTA (one job group per CTA).
size_t tk_stitch_smem_bytes(int dtype, size_t arena) {
  return dtype == TK_F64 ? group_smem_bytes<double>(arena) : group_smem_bytes<float>(arena);
}

static const void* stitch_fn(int dtype) { return dtype == TK_F64 ? tk_stitch_kernel_f64() : tk_stitch_kernel_f32(); }

static int set_smem_attr(const void* fn, size_t smem) {
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return TK_ERR_CUDA;
  return TK_OK;
}

int tk_occupancy(int dtype, size_t smem, int threads) {
  const void* fn = stitch_fn(dtype);
  if (set_smem_attr(fn, smem) != TK_OK) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess) return 0;
  return nb;
}

static int launch_stitch(int dtype, const TkTreeView& tv, int mode, int level, int64_t k0, int njobs,
                         const TkQueryBatch& qb, const TkWorkspace& ws, int grid, cudaStream_t stream) {
  const size_t smem = tk_stitch_smem_bytes(dtype, ws.smem_arena);
  if (ws.warps * 32 > 2 * TK_NT) return TK_ERR_ARG;
  if (cudaMemsetAsync(ws.counter, 0, sizeof(unsigned), stream) != cudaSuccess) return TK_ERR_CUDA;
  if (set_smem_attr(stitch_fn(dtype), smem)) return TK_ERR_CUDA;
  if (dtype == TK_F64)
    tk_stitch_launch_f64(grid, 32 * ws.warps, smem, stream, tv, mode, level, k0, njobs, qb, ws);
  else
    tk_stitch_launch_f32(grid, 32 * ws.warps, smem, stream, tv, mode, level, k0, njobs, qb, ws);
  return cudaGetLastError() == cudaSuccess ? TK_OK : TK_ERR_CUDA;
}

int tk_launch_merge(int dtype, const TkTreeView& tv, int level, int64_t k0, int njobs, const TkWorkspace& ws,
                    int grid, cudaStream_t stream) {
  if (njobs <= 0) return TK_OK;
  TkQueryBatch qb{};
  return launch_stitch(dtype, tv, TK_JOB_MERGE, level, k0, njobs, qb, ws, grid, stream);
}

int tk_launch_query(int dtype, const TkTreeView& tv, const TkQueryBatch& qb, const TkWorkspace& ws, int grid,
                    cudaStream_t stream) {
  if (qb.n <= 0) return TK_OK;
  return launch_stitch(dtype, tv, TK_JOB_QUERY, 0, 0, qb.n, qb, ws, grid, stream);
}

size_t tk_batch_smem_bytes(int dtype, size_t half_arena) {
  const size_t hdr = dtype == TK_F64 ? align16(sizeof(WarpSm<double>)) : align16(sizeof(WarpSm<float>));
  return 2 * hdr + 2 * align16(half_arena);
}

int tk_launch_batch(int dtype, const TkTreeView& tv, const TkQueryBatch& qb, const TkWorkspace& ws, int grid,
                    cudaStream_t stream) {
  if (qb.n <= 0) return TK_OK;
  const size_t smem = tk_batch_smem_bytes(dtype, ws.smem_arena);
  if (cudaMemsetAsync(ws.counter, 0, sizeof(unsigned), stream) != cudaSuccess) return TK_ERR_CUDA;
  if (set_smem_attr(dtype == TK_F64 ? tk_batch_kernel_f64() : tk_batch_kernel_f32(), smem)) return TK_ERR_CUDA;
  if (dtype == TK_F64)
    tk_batch_launch_f64(grid, 2 * TK_NT, smem, stream, tv, qb, ws);
  else
    tk_batch_launch_f32(grid, 2 * TK_NT, smem, stream, tv, qb, ws);
  return cudaGetLastError() == cudaSuccess ? TK_OK : TK_ERR_CUDA;
}

int tk_launch_plan(const TkTreeView& tv, int n, const int64_t* ranges, const int64_t* tq, int heavy_hits, int* split,
                   int* order, cudaStream_t stream) {
  if (n <= 0) return TK_OK;
  k_plan<<<1, 1024, 0, stream>>>(tv, n, ranges, tq, heavy_hits, split, order);
  return cudaGetLastError() == cudaSuccess ? TK_OK : TK_ERR_CUDA;
}

int tk_launch_hitset(const TkTreeView& tv, int n, const int64_t* ranges, tk_hit* out, int cap, int* counts,
                     cudaStream_t stream) {
  if (n <= 0) return TK_OK;
  const int nt = 32;
  k_hitset<<<(n + nt - 1) / nt, nt, 0, stream>>>(tv, n, ranges, out, cap, counts);
  return cudaGetLastError() == cudaSuccess ? TK_OK : TK_ERR_CUDA;
}

// ---- FMA-rate probe ----------------------------------------------------------
// Every thread runs 8 independent chains of fused multiply-adds (enough in
// flight to cover the FMA latency on every scheduler); the result is written
// so that the chains are not optimized away.
namespace {

template <class S>
__global__ void __launch_bounds__(256) k_fma_rate(S* out, int iters, S a, S b) {
  S x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = S(threadIdx.x) * S(1e-7) + S(i);
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
  }
  S s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class S> int fma_rate(int device, double* flops_per_s) {
  int sms = 0;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return TK_ERR_CUDA;
  const int blocks = 8 * sms, threads = 256;
  const int iters = sizeof(S) == 8 ? 64 : 2048;
  S* out = nullptr;
  if (cudaMalloc(&out, sizeof(S) * (size_t)blocks * threads) != cudaSuccess) return TK_ERR_NOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 0.f;
  for (int rep = 0; rep < 4; ++rep) {  // the first run is a warm-up
    cudaEventRecord(e0);
    k_fma_rate<S><<<blocks, threads>>>(out, iters, S(0.9999), S(1e-6));
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  const int rc = cudaGetLastError() == cudaSuccess ? TK_OK : TK_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (rc == TK_OK) *flops_per_s = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3);
  return rc;
}

}  // namespace

extern "C" int tk_probe_fma_rate(int dtype, int device, double* flops_per_s) {
  if (!flops_per_s || (dtype != TK_F64 && dtype != TK_F32)) return TK_ERR_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  const int rc = dtype == TK_F64 ? fma_rate<double>(device, flops_per_s) : fma_rate<float>(device, flops_per_s);
  if (prev >= 0) cudaSetDevice(prev);
  return rc;
}
