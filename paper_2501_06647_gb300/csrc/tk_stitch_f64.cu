// k_stitch<double>: node merges, single queries and the allocation-free batch.
#include "tk_inst.h"
#include "tk_stitch.cuh"

using namespace tk;

const void* tk_stitch_kernel_f64() { return (const void*)k_stitch<double, BlockGroup>; }

void tk_stitch_launch_f64(int grid, int threads, size_t smem, cudaStream_t stream, const TkTreeView& tv, int mode,
                          int level, int64_t k0, int njobs, const TkQueryBatch& qb, const TkWorkspace& ws) {
  k_stitch<double, BlockGroup><<<grid, threads, smem, stream>>>(tv, mode, level, k0, njobs, qb, ws);
}
