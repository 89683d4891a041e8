// Same-sign tangent augmentation of the query (Def. 1 tangent points T;
// Sec. 6 min_valid_radius candidates) and its backward.
#include <cuda_runtime.h>

#include "gfs.h"
#include "gfs_tangent.cuh"
#include "gfs_tangent.h"
#include "gfs_tangent_warp.cuh"

namespace gfs {

namespace {

// one warp per point (the lanes walk the hierarchy together, gfs_tangent_warp.cuh),
// points taken in the order a.perm gives (Morton order: consecutive warps
// walk similar paths)
constexpr int kTanWarps = 4;

__global__ void __launch_bounds__(32 * kTanWarps) k_query_tangent(QueryArgs a, int box_cull) {
  __shared__ uint32_t s_stk[kTanWarps][tangent::kWarpStack + kFan];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t slot = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  if (slot >= a.m) return;  // the same for the whole warp
  tangent::warp_tangent_one(a, box_cull, a.perm ? int64_t(a.perm[slot]) : slot, s_stk[w], lane);
}

__global__ void __launch_bounds__(128) k_argmin_points(QueryArgs a, const int64_t* __restrict__ argmin,
                                                       const uint16_t* __restrict__ flags, double* __restrict__ out) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= a.m) return;
  double x, y, z;
  tangent::load_point(a, q, x, y, z);
  tangent::argmin_point(a, x, y, z, flags[q] & 15, argmin[q], out + 3 * q);
}

constexpr double kFixScale = 1099511627776.0;  // 2^40, the backward's fixed-point scale

__device__ __forceinline__ void acc_add(long long* dst, double v) {
  atomicAdd(reinterpret_cast<unsigned long long*>(dst), (unsigned long long)(long long)llrint(v * kFixScale));
}

// Value m = |x - t| with t = p_j + e r (x - p_j)/|x - p_j|, e = +1 near,
// -1 far: m = |d - e r|, d = |x - p_j|.  With w = (x - p_j)/d and
// h = sign(d - e r): dm/dx = h w, dm/dp_j = -h w, dm/dr = -e h; the signed
// value is sigma m and r = |s_j| (dr/ds_j = sign(s_j)).
__global__ void __launch_bounds__(128) k_tangent_grad(GradArgs a, int64_t n) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= a.m || (a.flags[q] & 15) != GFS_CODE_TANGENT) return;
  if (a.arg[q] < 0 || (a.arg[q] >> 1) >= n) return;  // not a tangent id of this state
  const float sv = a.s[q];
  const double sigma = sv > 0.f ? 1.0 : (sv < 0.f ? -1.0 : 0.0);
  if (sigma == 0.0) return;
  double x, y, z;
  if (a.x32) {
    x = a.x32[3 * q]; y = a.x32[3 * q + 1]; z = a.x32[3 * q + 2];
  } else {
    x = a.x64[3 * q]; y = a.x64[3 * q + 1]; z = a.x64[3 * q + 2];
  }
  const int64_t j = a.arg[q] >> 1;
  const double e = (a.arg[q] & 1) ? -1.0 : 1.0;
  const D4 P = a.sph64[j];
  const double r = fabs(P.w);
  double wx = x - P.x, wy = y - P.y, wz = z - P.z;
  const double d = sqrt(wx * wx + wy * wy + wz * wz);
  if (!(d > 0.0)) return;
  wx /= d; wy /= d; wz /= d;
  const double h = d - e * r >= 0.0 ? 1.0 : -1.0;
  const double g = a.grad_s[q];
  const double gx = g * sigma * h * wx, gy = g * sigma * h * wy, gz = g * sigma * h * wz;
  if (a.acc_p) {
    acc_add(a.acc_p + 3 * j, -gx);
    acc_add(a.acc_p + 3 * j + 1, -gy);
    acc_add(a.acc_p + 3 * j + 2, -gz);
  }
  const double sj = P.w > 0 ? 1.0 : -1.0;
  if (a.acc_s) acc_add(a.acc_s + j, g * sigma * (-e * h) * sj);
  if (a.grad_x) {
    a.grad_x[3 * q] = float(gx);
    a.grad_x[3 * q + 1] = float(gy);
    a.grad_x[3 * q + 2] = float(gz);
  }
}

__global__ void k_acc_to_float(const long long* __restrict__ acc, int64_t n, float* __restrict__ out) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n) out[i] = float(double(acc[i]) / kFixScale);
}

unsigned long long g_tangent_launches = 0;

inline unsigned int blocks(int64_t n, int b) { return (unsigned int)((n + b - 1) / b); }

}  // namespace

cudaError_t launch_query_tangent(const QueryArgs& a, int box_cull, cudaStream_t st) {
  if (a.m <= 0) return cudaSuccess;
  k_query_tangent<<<blocks(a.m, kTanWarps), 32 * kTanWarps, 0, st>>>(a, box_cull);
  ++g_tangent_launches;
  return cudaGetLastError();
}

cudaError_t launch_tangent_grad(const GradArgs& a, int64_t n, float* grad_p, float* grad_sv, cudaStream_t st) {
  if (a.m > 0) {
    k_tangent_grad<<<blocks(a.m, 128), 128, 0, st>>>(a, n);
    ++g_tangent_launches;
  }
  if (grad_p) {
    k_acc_to_float<<<blocks(3 * n, 256), 256, 0, st>>>(a.acc_p, 3 * n, grad_p);
    ++g_tangent_launches;
  }
  if (grad_sv) {
    k_acc_to_float<<<blocks(n, 256), 256, 0, st>>>(a.acc_s, n, grad_sv);
    ++g_tangent_launches;
  }
  return cudaGetLastError();
}

cudaError_t launch_argmin_points(const QueryArgs& a, const int64_t* argmin, const uint16_t* flags, double* out,
                                 cudaStream_t st) {
  if (a.m <= 0) return cudaSuccess;
  k_argmin_points<<<blocks(a.m, 128), 128, 0, st>>>(a, argmin, flags, out);
  ++g_tangent_launches;
  return cudaGetLastError();
}

unsigned long long tangent_launch_count() { return g_tangent_launches; }

}  // namespace gfs
