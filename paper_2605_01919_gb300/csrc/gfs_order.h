// Launcher of the cell coverage count (Sec. 4.2 refinement order; internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gfs_kernels.h"

namespace gfs {

// counts[c] = covered sub-points of cell c (cells: device, ncells x 3 int32);
// one warp per cell
cudaError_t launch_cell_coverage(const QueryArgs& a, const int32_t* cells, int64_t ncells, const double* origin,
                                 double h, int sub, uint32_t* counts, cudaStream_t st);

unsigned long long order_launch_count();

}  // namespace gfs
