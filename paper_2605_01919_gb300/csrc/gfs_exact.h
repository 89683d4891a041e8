// Launcher of the exact uncovered test per sphere (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gfs_kernels.h"

namespace gfs {

// out[i] (device, n bytes, input order): 1 uncovered, 0 covered, 2 undecided
cudaError_t launch_sphere_uncovered(const QueryArgs& a, uint8_t* out, cudaStream_t st);

unsigned long long exact_launch_count();

}  // namespace gfs
