// Exact uncovered test per sphere (Prop. 1 (ii)): one thread per sphere.
#include <cuda_runtime.h>

#include "gfs_exact.cuh"
#include "gfs_exact.h"

namespace gfs {

namespace {

// threads take the spheres in hierarchy (Morton) order, so a warp's spheres
// are neighbours and walk similar paths
__global__ void __launch_bounds__(128) k_sphere_uncovered(QueryArgs a, uint8_t* __restrict__ out) {
  const int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (j >= a.n) return;
  const int i = a.sid[j];
  out[i] = uint8_t(exact::sphere_uncovered(a, i));
}

unsigned long long g_exact_launches = 0;

}  // namespace

cudaError_t launch_sphere_uncovered(const QueryArgs& a, uint8_t* out, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  k_sphere_uncovered<<<(unsigned int)((a.n + 127) / 128), 128, 0, st>>>(a, out);
  ++g_exact_launches;
  return cudaGetLastError();
}

unsigned long long exact_launch_count() { return g_exact_launches; }

}  // namespace gfs
