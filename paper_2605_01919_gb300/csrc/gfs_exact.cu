// Exact uncovered test per sphere (Prop. 1 (ii)): one warp per sphere.
#include <cuda_runtime.h>

#include "gfs_exact.cuh"
#include "gfs_exact.h"

namespace gfs {

namespace {

// One warp per sphere, spheres in hierarchy (Morton) order: lane 0 gathers
// the balls that meet the sphere into shared memory, then the lanes split
// the circle and triple points and the warp votes.
constexpr int kWarps = 4;

__global__ void __launch_bounds__(32 * kWarps) k_sphere_uncovered(QueryArgs a, uint8_t* __restrict__ out) {
  __shared__ int s_meet[kWarps][exact::kMaxMeet];
  __shared__ int s_found[kWarps];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  if (j >= a.n) return;  // the same for the whole warp
  const int i = a.sid[j];
  int nn = 0;
  if (lane == 0) {
    s_found[w] = 0;
    if (fabs(a.sph64[i].w) != 0.0) nn = exact::gather_meet(a, i, s_meet[w]);
  }
  nn = __shfl_sync(0xffffffffu, nn, 0);
  __syncwarp();
  int res = -1;
  if (lane == 0) res = exact::trivial_case(a, i, nn);
  res = __shfl_sync(0xffffffffu, res, 0);
  if (res < 0) {
    const bool mine = exact::lane_candidates(a, i, s_meet[w], nn, lane, 32, &s_found[w]);
    if (mine) s_found[w] = 1;
    res = __any_sync(0xffffffffu, mine) ? 1 : 0;
  }
  if (lane == 0) out[i] = uint8_t(res);
}

unsigned long long g_exact_launches = 0;

}  // namespace

cudaError_t launch_sphere_uncovered(const QueryArgs& a, uint8_t* out, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  k_sphere_uncovered<<<(unsigned int)((a.n + kWarps - 1) / kWarps), 32 * kWarps, 0, st>>>(a, out);
  ++g_exact_launches;
  return cudaGetLastError();
}

unsigned long long exact_launch_count() { return g_exact_launches; }

}  // namespace gfs
