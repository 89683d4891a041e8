// Covered area ratio of grid cells for the refinement order (Sec. 4.2).
#include <cuda_runtime.h>

#include "gfs_order.cuh"
#include "gfs_order.h"

namespace gfs {

namespace {

// one warp per cell; the lanes split the cell's sub-points and the warp sums
// its count (no atomics: the result does not depend on scheduling)
__global__ void __launch_bounds__(128) k_cell_coverage(QueryArgs a, const int32_t* __restrict__ cells,
                                                       int64_t ncells, double ox, double oy, double oz, double h,
                                                       int sub, uint32_t* __restrict__ counts) {
  const int64_t c = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= ncells) return;  // c is the same for the whole warp
  unsigned cnt = order::cell_cover_count(a, cells + 3 * c, ox, oy, oz, h, sub, lane, 32);
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  if (lane == 0) counts[c] = cnt;
}

unsigned long long g_order_launches = 0;

}  // namespace

cudaError_t launch_cell_coverage(const QueryArgs& a, const int32_t* cells, int64_t ncells, const double* origin,
                                 double h, int sub, uint32_t* counts, cudaStream_t st) {
  if (ncells <= 0) return cudaSuccess;
  const int64_t threads = ncells * 32;
  k_cell_coverage<<<(unsigned int)((threads + 127) / 128), 128, 0, st>>>(a, cells, ncells, origin[0], origin[1],
                                                                          origin[2], h, sub, counts);
  ++g_order_launches;
  return cudaGetLastError();
}

unsigned long long order_launch_count() { return g_order_launches; }

}  // namespace gfs
