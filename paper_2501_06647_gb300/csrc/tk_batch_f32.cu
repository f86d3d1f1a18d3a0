// k_batch<float>: planned query batches.
#include "tk_inst.h"
#include "tk_stitch.cuh"

using namespace tk;

const void* tk_batch_kernel_f32() { return (const void*)k_batch<float>; }

void tk_batch_launch_f32(int grid, int threads, size_t smem, cudaStream_t stream, const TkTreeView& tv,
                         const TkQueryBatch& qb, const TkWorkspace& ws) {
  k_batch<float><<<grid, threads, smem, stream>>>(tv, qb.n, qb, ws);
}
