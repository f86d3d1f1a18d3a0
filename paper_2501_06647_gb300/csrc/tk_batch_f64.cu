// k_batch<double>: planned query batches.
#include "tk_inst.h"
#include "tk_stitch.cuh"

using namespace tk;

const void* tk_batch_kernel_f64() { return (const void*)k_batch<double>; }

void tk_batch_launch_f64(int grid, int threads, size_t smem, cudaStream_t stream, const TkTreeView& tv,
                         const TkQueryBatch& qb, const TkWorkspace& ws) {
  k_batch<double><<<grid, threads, smem, stream>>>(tv, qb.n, qb, ws);
}
