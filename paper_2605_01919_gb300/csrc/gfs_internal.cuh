// Internal device-side definitions shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gfs {

// ---------------------------------------------------------------------------
// Bounding hierarchy: an implicit 8-ary tree over Morton-sorted items.
// Level 0 node j ("leaf") covers items [8j, 8j+8); a node j at level l >= 1
// covers nodes [8j, 8j+8) of level l-1.  Node boxes are tight over the FP32
// item positions and widened by one ulp, so they also contain the FP64
// positions the FP32 ones were rounded from.
//
// Sphere nodes also carry two centres and four radii, each radius an upper
// bound over the node's spheres (p_j, r_j):
//   wp, wn -- max over spheres of sign + (resp. -) of |p_j - C| + r_j: their
//             balls lie in B(C, w), so |x - p_j| - r_j >= |x - C| - w;
//   w0     -- max over all spheres of |p_j - C| (their centres lie in
//             B(C, w0): a query point equal to a sample lies in it);
//   wf     -- max over all spheres of |p_j - F| - r_j about a second centre
//             F, so that |x - p_j| + r_j >= |x - F| - wf.
// Stored as na = (C, max(wp, wn)) -- all a coverage test reads --,
// nb = (wp, wn, w0, 0) and nf = (F, wf).  C is the centre of a small ball
// enclosing the node's balls; F is chosen for the far bound alone (it leans
// towards the small spheres, C towards the large ones).  Exact SDF samples
// are close to nested along the gradient (a deeper ball contains a shallower
// one), which balls exploit and an axis box cannot.  Empty classes have -inf.
// ---------------------------------------------------------------------------
constexpr int kLeaf = 8;
constexpr int kFan = 8;
constexpr int kMaxLevels = 12;
constexpr int kStack = 112;  // >= (kFan-1)*kMaxLevels + kFan

struct Tree {
  int nlevels;                    // levels in use (level nlevels-1 has <= kFan nodes)
  int64_t nitems;
  int64_t count[kMaxLevels];      // nodes per level
  int64_t offset[kMaxLevels];     // first node of each level in the node arrays
  float4* lo;                     // (min x, min y, min z, -)
  float4* hi;                     // (max x, max y, max z, -)
  float4* na;                     // sphere trees: (C, max(wp, wn))
  float4* nb;                     // sphere trees: (wp, wn, w0, 0)
  float4* nf;                     // sphere trees: (F, wf)
};

__host__ __device__ inline uint32_t pack_node(int level, int64_t idx) {
  return (uint32_t(level) << 27) | uint32_t(idx);
}
__host__ __device__ inline int node_level(uint32_t v) { return int(v >> 27); }
__host__ __device__ inline int64_t node_index(uint32_t v) { return int64_t(v & ((1u << 27) - 1)); }

// FP64 sample record in input order: position and signed value.
struct alignas(32) D4 {
  double x, y, z, w;
};

// ---------------------------------------------------------------------------
// Exact FP64 predicates.  Each operation is rounded on its own, in the order
// written (the intrinsics are never contracted into FMAs), which makes every
// value bit-identical to a plain IEEE-754 evaluation of the same expression.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double ex_d2(double ax, double ay, double az, double bx, double by, double bz) {
  double dx = __dsub_rn(ax, bx), dy = __dsub_rn(ay, by), dz = __dsub_rn(az, bz);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// q lies in the open ball of sphere (p, s) shrunk by tol (Sec. 3.1, App. B)
__device__ __forceinline__ bool ex_cov(double qx, double qy, double qz, const D4& p, double tol) {
  double r = fabs(p.w);
  if (!(r > tol)) return false;
  double rt = __dsub_rn(r, tol);
  return ex_d2(qx, qy, qz, p.x, p.y, p.z) < __dmul_rn(rt, rt);
}

// candidate q = p + |s| u (product, then sum, per component)
__device__ __forceinline__ void ex_cand(const D4& p, double ux, double uy, double uz, double& qx, double& qy,
                                        double& qz) {
  double r = fabs(p.w);
  qx = __dadd_rn(p.x, __dmul_rn(r, ux));
  qy = __dadd_rn(p.y, __dmul_rn(r, uy));
  qz = __dadd_rn(p.z, __dmul_rn(r, uz));
}

__device__ __forceinline__ bool ex_inbox(double qx, double qy, double qz) {
  return fabs(qx) <= 1.0 && fabs(qy) <= 1.0 && fabs(qz) <= 1.0;
}

// squared distance from a point to a node box (FP32)
__device__ __forceinline__ float box_d2(float x, float y, float z, const float4& lo, const float4& hi) {
  float dx = fmaxf(fmaxf(lo.x - x, x - hi.x), 0.f);
  float dy = fmaxf(fmaxf(lo.y - y, y - hi.y), 0.f);
  float dz = fmaxf(fmaxf(lo.z - z, z - hi.z), 0.f);
  return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// squared distance from a point to a node box (FP64); the float box corners
// convert exactly, so this is a lower bound of the distance to every item in
// the node up to one rounding per operation.
__device__ __forceinline__ double box_d2_64(double x, double y, double z, const float4& lo, const float4& hi) {
  double dx = fmax(fmax(double(lo.x) - x, x - double(hi.x)), 0.0);
  double dy = fmax(fmax(double(lo.y) - y, y - double(hi.y)), 0.0);
  double dz = fmax(fmax(double(lo.z) - z, z - double(hi.z)), 0.0);
  return dx * dx + dy * dy + dz * dz;
}

// squared distance from a point to a bounding-ball centre
__device__ __forceinline__ float ball_d2(float x, float y, float z, const float4& b) {
  const float dx = x - b.x, dy = y - b.y, dz = z - b.z;
  return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}
__device__ __forceinline__ double ball_d2_64(double x, double y, double z, const float4& b) {
  const double dx = x - double(b.x), dy = y - double(b.y), dz = z - double(b.z);
  return dx * dx + dy * dy + dz * dz;
}

__device__ __forceinline__ bool inside_box(float x, float y, float z, const float4& lo, const float4& hi) {
  return x >= lo.x && x <= hi.x && y >= lo.y && y <= hi.y && z >= lo.z && z <= hi.z;
}

// Morton code of a point, 10 bits per axis over [-1, 1] (clamped)
__device__ __forceinline__ uint32_t spread10(uint32_t v) {
  v &= 1023u;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}
__device__ __forceinline__ uint32_t morton3(float x, float y, float z) {
  auto q = [](float v) {
    int t = int(floorf((v + 1.0f) * 512.0f));
    return uint32_t(t < 0 ? 0 : (t > 1023 ? 1023 : t));
  };
  return (spread10(q(x)) << 2) | (spread10(q(y)) << 1) | spread10(q(z));
}

// Launch-wide constants derived from the data at build time (device memory)
struct BuildConsts {
  float A;        // max(1, max |p_c|): coordinate magnitude bound
  float R;        // max |s|
  float eq;       // bound on |q32 - q64| for a candidate coordinate
  float ea;       // FP32 error bound on |x-p| -+ r for queries
  float ed_lin;   // survivor distance^2 error: ed_lin * sqrt(D) + ed_quad * D
  float ed_quad;
  float eprune;   // additive slack for FP32 node pruning
  float pad;
};

struct Counters {
  unsigned long long cull_rechecks;
  unsigned long long query_rechecks;
  unsigned int nsurv[2];
  unsigned int ndefer;
  unsigned int walk_err;  // bit 0: a warp walk's stack guard tripped (cannot happen)
  unsigned long long q_sphere_ntests;  // child-node bound tests of the query sphere pass
  unsigned long long q_sphere_items;   // spheres tested by the query sphere pass
  unsigned long long q_surv_ntests;    // child-node bound tests of the survivor pass
  unsigned long long q_band_passes;    // FP64 band passes run to settle near-ties
  unsigned long long q_surv_items;     // survivors tested by the survivor pass
  unsigned long long c_ntests;         // child-node coverage tests of the cull (open lanes)
  unsigned long long c_items;          // sphere coverage tests of the cull (open lanes)
};

}  // namespace gfs
