// Entry points of the translation units that instantiate the stitch kernels
// (tk_stitch_f32.cu, tk_stitch_f64.cu, tk_batch_f32.cu, tk_batch_f64.cu): the
// kernel's address (for attributes and occupancy) and an asynchronous launch.
#pragma once
#include "tk_internal.h"

const void* tk_stitch_kernel_f32();
const void* tk_stitch_kernel_f64();
void tk_stitch_launch_f32(int grid, int threads, size_t smem, cudaStream_t stream, const TkTreeView& tv, int mode,
                          int level, int64_t k0, int njobs, const TkQueryBatch& qb, const TkWorkspace& ws);
void tk_stitch_launch_f64(int grid, int threads, size_t smem, cudaStream_t stream, const TkTreeView& tv, int mode,
                          int level, int64_t k0, int njobs, const TkQueryBatch& qb, const TkWorkspace& ws);
const void* tk_batch_kernel_f32();
const void* tk_batch_kernel_f64();
void tk_batch_launch_f32(int grid, int threads, size_t smem, cudaStream_t stream, const TkTreeView& tv,
                         const TkQueryBatch& qb, const TkWorkspace& ws);
void tk_batch_launch_f64(int grid, int threads, size_t smem, cudaStream_t stream, const TkTreeView& tv,
                         const TkQueryBatch& qb, const TkWorkspace& ws);
