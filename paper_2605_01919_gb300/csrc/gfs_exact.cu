// Exact uncovered test per sphere (Prop. 1 (ii)) and the uncovered
// intersection circles and points (Sec. 4.1): one thread per sphere.
#include <cuda_runtime.h>

#include "gfs_exact.cuh"
#include "gfs_exact.h"

namespace gfs {

namespace {

// One thread per sphere, spheres in hierarchy (Morton) order so that a
// warp's spheres are neighbours and walk the same part of the hierarchy.
__global__ void __launch_bounds__(128) k_sphere_uncovered(QueryArgs a, uint8_t* __restrict__ out,
                                                          double* __restrict__ witness) {
  const int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (j >= a.n) return;
  const int i = a.sid[j];
  int S[exact::kMaxSet];
  uint32_t stack[kStack];
  double w[3];
  const int res = exact::sphere_uncovered(a, i, S, stack, w);
  out[i] = uint8_t(res);
  if (witness)
    for (int c = 0; c < 3; ++c) witness[3 * int64_t(i) + c] = res == 1 ? w[c] : __longlong_as_double(0x7ff8000000000000ll);
}

// One thread per uncovered sphere, spheres in hierarchy (Morton) order: its
// circles with the spheres after it and their uncovered points.
__global__ void __launch_bounds__(128) k_intersections(QueryArgs a, const uint8_t* __restrict__ uncov,
                                                       exact::UDOut o) {
  const int64_t u = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (u >= a.n) return;
  const int i = a.sid[u];
  if (uncov[i] == 0) return;
  int M[exact::kMaxSet];
  uint32_t stacks[3 * kStack];
  exact::sphere_intersections(a, i, uncov, M, stacks, o);
}

// Sort keys: circles (i << 32) | j; points first by (m << 1) | side, then
// (stable) by (i << 32) | j.
__global__ void k_ud_circle_keys(const int64_t* __restrict__ circ, int64_t nc, unsigned long long* __restrict__ key) {
  const int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (k >= nc) return;
  key[k] = (static_cast<unsigned long long>(circ[2 * k]) << 32) | static_cast<unsigned long long>(circ[2 * k + 1]);
}

__global__ void k_ud_point_keys(const int64_t* __restrict__ quad, const int* __restrict__ order, int64_t np,
                                int primary, unsigned long long* __restrict__ key, int* __restrict__ val) {
  const int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (k >= np) return;
  const int64_t s = order ? order[k] : k;
  const int64_t* q = quad + 4 * s;
  key[k] = primary ? (static_cast<unsigned long long>(q[0]) << 32) | static_cast<unsigned long long>(q[1])
                   : (static_cast<unsigned long long>(q[2]) << 1) | static_cast<unsigned long long>(q[3]);
  val[k] = int(s);
}

__global__ void k_ud_gather(const unsigned long long* __restrict__ ckey, int64_t nc, int64_t* __restrict__ circ_out,
                            const int* __restrict__ order, const int64_t* __restrict__ quad,
                            const double* __restrict__ pts, int64_t np, int64_t* __restrict__ quad_out,
                            double* __restrict__ pts_out) {
  const int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (k < nc) {
    circ_out[2 * k] = int64_t(ckey[k] >> 32);
    circ_out[2 * k + 1] = int64_t(ckey[k] & 0xffffffffull);
  }
  if (k < np) {
    const int64_t s = order[k];
    for (int c = 0; c < 4; ++c) quad_out[4 * k + c] = quad[4 * s + c];
    for (int c = 0; c < 3; ++c) pts_out[3 * k + c] = pts[3 * s + c];
  }
}

unsigned long long g_exact_launches = 0;

}  // namespace

cudaError_t launch_intersections(const QueryArgs& a, const uint8_t* uncov, const exact::UDOut& o, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  k_intersections<<<(unsigned int)((a.n + 127) / 128), 128, 0, st>>>(a, uncov, o);
  ++g_exact_launches;
  return cudaGetLastError();
}

cudaError_t launch_ud_circle_keys(const int64_t* circ, int64_t nc, unsigned long long* key, cudaStream_t st) {
  if (nc <= 0) return cudaSuccess;
  k_ud_circle_keys<<<(unsigned int)((nc + 255) / 256), 256, 0, st>>>(circ, nc, key);
  ++g_exact_launches;
  return cudaGetLastError();
}

cudaError_t launch_ud_point_keys(const int64_t* quad, const int* order, int64_t np, int primary,
                                 unsigned long long* key, int* val, cudaStream_t st) {
  if (np <= 0) return cudaSuccess;
  k_ud_point_keys<<<(unsigned int)((np + 255) / 256), 256, 0, st>>>(quad, order, np, primary, key, val);
  ++g_exact_launches;
  return cudaGetLastError();
}

cudaError_t launch_ud_gather(const unsigned long long* ckey, int64_t nc, int64_t* circ_out, const int* order,
                             const int64_t* quad, const double* pts, int64_t np, int64_t* quad_out, double* pts_out,
                             cudaStream_t st) {
  const int64_t n = nc > np ? nc : np;
  if (n <= 0) return cudaSuccess;
  k_ud_gather<<<(unsigned int)((n + 255) / 256), 256, 0, st>>>(ckey, nc, circ_out, order, quad, pts, np, quad_out,
                                                                 pts_out);
  ++g_exact_launches;
  return cudaGetLastError();
}

cudaError_t launch_sphere_uncovered(const QueryArgs& a, uint8_t* out, double* witness, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  k_sphere_uncovered<<<(unsigned int)((a.n + 127) / 128), 128, 0, st>>>(a, out, witness);
  ++g_exact_launches;
  return cudaGetLastError();
}

unsigned long long exact_launch_count() { return g_exact_launches; }

}  // namespace gfs
