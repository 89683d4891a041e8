// Launchers of the same-sign tangent augmentation (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gfs_kernels.h"

namespace gfs {

// Refine the plain query's outputs in place (a.fl_out and a.arg_out are read
// and rewritten; a.s_out / a.s64_out rewritten where non-null).
cudaError_t launch_query_tangent(const QueryArgs& a, int box_cull, cudaStream_t st);

// Backward of the TANGENT results into the fixed-point accumulators of a
// (run after launch_grad with null outputs), then the conversion of the
// per-sample sums to FP32 outputs (grad_p n*3, grad_sv n; each nullable).
cudaError_t launch_tangent_grad(const GradArgs& a, int64_t n, float* grad_p, float* grad_sv, cudaStream_t st);

// q* of every point (out: m x 3 FP64) from a query's argmin and flags
cudaError_t launch_argmin_points(const QueryArgs& a, const int64_t* argmin, const uint16_t* flags, double* out,
                                 cudaStream_t st);

// kernels this file has launched in this process
unsigned long long tangent_launch_count();

}  // namespace gfs
