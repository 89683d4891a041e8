// Device kernels of the consistent-SDF hot path.
//
//   P build   k_cull          -- candidate generation and coverage culling
//                                (Def. 1 discretised, Prop. 1 (ii))
//   query     k_query_spheres -- FP32 pass over the spheres (containment,
//                                tangent and far bounds), state per point
//             k_query_finish  -- FP32 pass over the survivors, certified
//                                decisions, value and flags
//             k_query_exact   -- FP64 evaluation, used for every decision the
//                                FP32 path cannot certify (and precision=1)
//   backward  k_query_grad    -- d s*/d(x, p_i, s_i) through the argmin
//
// FP32 filter.  Every predicate the FP32 path decides (is q inside a shrunk
// ball, which candidate is nearest, is a bound exceeded) is compared against
// a rigorous error bound of the FP32 evaluation relative to the exact value.
// Outside the bound the FP32 answer equals the FP64 answer; inside it the
// predicate is re-decided with the FP64 expression the definition uses, so
// every decision is that of an FP64 evaluation.
#include <cub/cub.cuh>
#include <cooperative_groups.h>

#include "gfs_internal.cuh"
#include "gfs_kernels.h"

namespace cg = cooperative_groups;

namespace gfs {

constexpr float kU = 5.9604644775390625e-8f;  // 2^-24, FP32 unit roundoff

__device__ __forceinline__ float sqf(float v) { return v * v; }

// ---------------------------------------------------------------------------
// build: bounds of the data, input copy, Morton keys
// ---------------------------------------------------------------------------
__global__ void k_copy_inputs(const double* __restrict__ p, const double* __restrict__ s, int64_t n,
                              D4* __restrict__ sph64) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    sph64[i] = D4{p[3 * i], p[3 * i + 1], p[3 * i + 2], s[i]};
}

// Morton keys of the sample centres and the data bounds (max |coordinate|,
// max |s|) used by the error model.
__global__ void k_keys_d4(const D4* __restrict__ sph64, int64_t n, uint32_t* __restrict__ keys,
                          int* __restrict__ vals, unsigned int* __restrict__ bound_bits) {
  float amax = 0.f, rmax = 0.f;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const D4 d = sph64[i];
    amax = fmaxf(amax, __double2float_ru(fmax(fabs(d.x), fmax(fabs(d.y), fabs(d.z)))));
    rmax = fmaxf(rmax, __double2float_ru(fabs(d.w)));
    keys[i] = morton3(float(d.x), float(d.y), float(d.z));
    vals[i] = int(i);
  }
  for (int o = 16; o > 0; o >>= 1) {
    amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(bound_bits + 0, __float_as_uint(amax));  // non-negative floats order as integers
    atomicMax(bound_bits + 1, __float_as_uint(rmax));
  }
}

// Launch-wide error bounds from the data bounds (max |coordinate|, max |s|).
__device__ BuildConsts make_consts(unsigned int amax_bits, unsigned int rmax_bits) {
  float A = fmaxf(1.0f, __uint_as_float(amax_bits));
  float R = __uint_as_float(rmax_bits);
  const float u = kU;
  const float s3 = 1.7320508f;
  BuildConsts c;
  c.A = A;
  c.R = R;
  // candidate coordinate q32 = fma(r32, u32, p32) vs q64: u(|p| + 2r + |q|)
  c.eq = u * (2.f * A + 2.f * R + 0.01f) * 1.01f + 1e-12f;
  // |x-p| -+ r in FP32 for points in [-A,A]^3 (x rounded from FP64):
  // 2 sqrt3 u A + 4.25 u delta + 2 u r with delta <= 2 sqrt3 A, times 2
  c.ea = 2.f * u * (3.5f * A + 5.25f * 2.f * s3 * A + 2.f * R) + 1e-12f;
  // survivor distance^2: 2 sqrt3 (eq + uA) sqrt(D) + 5 u D, times 2
  c.ed_lin = 4.f * s3 * (c.eq + u * A);
  c.ed_quad = 10.f * u;
  // FP32 box-distance slack for a point rounded from FP64
  c.eprune = 4.f * s3 * u * A + 1e-7f;
  // the same for candidate points (their FP32 error is eq)
  c.pad = 4.f * s3 * (c.eq + u * A) + 1e-7f;
  return c;
}

__global__ void k_consts(const unsigned int* __restrict__ bound_bits, BuildConsts* __restrict__ bc) {
  *bc = make_consts(bound_bits[0], bound_bits[1]);
}

// FP32 coverage thresholds on d^2 for the filter: d2 < lo => covered for
// certain; d2 > hi => uncovered for certain; else re-decide in FP64.
__device__ __forceinline__ void cov_thresholds(double s64, float r32, float tol32, double tol, float e, float A,
                                               float& lo, float& hi) {
  if (!(fabs(s64) > tol)) {
    lo = -1.f;
    hi = -1.f;
    return;
  }
  const float u = kU;
  float rt = r32 - tol32;
  float rr = rt * rt;
  float rp = r32 + 1e-3f;
  float E = 2.f * (2.f * 1.7320508f * (e + u * A) * rp + 12.f * u * rp * rp) + 4e-15f * sqf(r32 + 1.f) + 1e-30f;
  lo = rr - E;
  hi = rr + E;
}

__global__ void k_gather_spheres(const D4* __restrict__ sph64, const int* __restrict__ order, int64_t n,
                                 const BuildConsts* __restrict__ bc, float tol32, double tol,
                                 float4* __restrict__ sph, float4* __restrict__ thr, int* __restrict__ sid) {
  int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= n) return;
  int o = order[t];
  D4 d = sph64[o];
  float w = float(d.w);
  if (w == 0.f && d.w != 0.0) w = copysignf(1.4e-45f, float(d.w > 0 ? 1 : -1));  // keep the sign class
  float4 S = make_float4(float(d.x), float(d.y), float(d.z), w);
  sph[t] = S;
  sid[t] = o;
  float A = bc->A;
  float lc, hc, lq, hq;
  cov_thresholds(d.w, fabsf(w), tol32, tol, bc->eq, A, lc, hc);
  cov_thresholds(d.w, fabsf(w), tol32, tol, kU * A, A, lq, hq);
  thr[t] = make_float4(lc, hc, lq, hq);
}

// ---------------------------------------------------------------------------
// hierarchy build
// ---------------------------------------------------------------------------
__device__ void point_leaf_node(const float4* __restrict__ items, int64_t nitems, float4* __restrict__ lo,
                                float4* __restrict__ hi, int64_t L) {
  int64_t b = L * kLeaf, e = min(b + kLeaf, nitems);
  float3 mn = make_float3(INFINITY, INFINITY, INFINITY), mx = make_float3(-INFINITY, -INFINITY, -INFINITY);
  for (int64_t i = b; i < e; ++i) {
    float4 v = items[i];
    mn.x = fminf(mn.x, v.x); mn.y = fminf(mn.y, v.y); mn.z = fminf(mn.z, v.z);
    mx.x = fmaxf(mx.x, v.x); mx.y = fmaxf(mx.y, v.y); mx.z = fmaxf(mx.z, v.z);
  }
  // widen by one ulp: the box then holds the FP64 points the FP32 ones were
  // rounded from
  lo[L] = make_float4(nextafterf(mn.x, -INFINITY), nextafterf(mn.y, -INFINITY), nextafterf(mn.z, -INFINITY), 0.f);
  hi[L] = make_float4(nextafterf(mx.x, INFINITY), nextafterf(mx.y, INFINITY), nextafterf(mx.z, INFINITY), 0.f);
}

__device__ void point_level_node(float4* __restrict__ lo, float4* __restrict__ hi, int64_t child_off, int64_t nchild,
                                 int64_t off, int64_t j) {
  int64_t b = j * kFan, e = min(b + kFan, nchild);
  float4 L = make_float4(INFINITY, INFINITY, INFINITY, 0.f), H = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
  for (int64_t c = b; c < e; ++c) {
    float4 a = lo[child_off + c], z = hi[child_off + c];
    L.x = fminf(L.x, a.x); L.y = fminf(L.y, a.y); L.z = fminf(L.z, a.z);
    H.x = fmaxf(H.x, z.x); H.y = fmaxf(H.y, z.y); H.z = fmaxf(H.z, z.z);
  }
  lo[off + j] = L;
  hi[off + j] = H;
}

__global__ void k_leaves(const float4* __restrict__ items, int64_t nitems, float4* __restrict__ lo,
                         float4* __restrict__ hi, int64_t nleaves) {
  int64_t L = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (L < nleaves) point_leaf_node(items, nitems, lo, hi, L);
}

__global__ void k_level(float4* __restrict__ lo, float4* __restrict__ hi, int64_t child_off, int64_t nchild,
                        int64_t off, int64_t nnode) {
  int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (j < nnode) point_level_node(lo, hi, child_off, nchild, off, j);
}

// Bounding ball of weighted centres (c_i, w_i): a centre c and
// V >= max_i (|c_i - c| + w_i).  Any centre is valid; subgradient steps from
// the better of two starts (the item of largest weight, the mean centre) make
// V small.  V is inflated by 8 ulp of |V| and of the coordinate range, which
// covers the FP32 evaluation and the rounding of FP64 inputs to FP32.
__device__ float4 bound_ball(const float4* it, int k, float A) {
  if (k == 0) return make_float4(0.f, 0.f, 0.f, -INFINITY);
  auto eval = [&](float cx, float cy, float cz, int& arg) {
    float best = -INFINITY;
    arg = 0;
    for (int i = 0; i < k; ++i) {
      const float dx = it[i].x - cx, dy = it[i].y - cy, dz = it[i].z - cz;
      const float v = sqrtf(dx * dx + dy * dy + dz * dz) + it[i].w;
      if (v > best) {
        best = v;
        arg = i;
      }
    }
    return best;
  };
  int big = 0;
  float mx = 0.f, my = 0.f, mz = 0.f;
  for (int i = 0; i < k; ++i) {
    if (it[i].w > it[big].w) big = i;
    mx += it[i].x;
    my += it[i].y;
    mz += it[i].z;
  }
  mx /= float(k);
  my /= float(k);
  mz /= float(k);
  int j0, j1;
  const float v0 = eval(it[big].x, it[big].y, it[big].z, j0);
  const float v1 = eval(mx, my, mz, j1);
  float cx = v0 <= v1 ? it[big].x : mx, cy = v0 <= v1 ? it[big].y : my, cz = v0 <= v1 ? it[big].z : mz;
  float bx = cx, by = cy, bz = cz, best = fminf(v0, v1);
  for (int t = 0; t < 24; ++t) {
    int j;
    const float v = eval(cx, cy, cz, j);
    if (v < best) {
      best = v;
      bx = cx;
      by = cy;
      bz = cz;
    }
    const float dx = it[j].x - cx, dy = it[j].y - cy, dz = it[j].z - cz;
    const float d = sqrtf(dx * dx + dy * dy + dz * dz);
    if (!(d > 1e-12f)) break;
    const float step = d / float(t + 2);
    cx += dx / d * step;
    cy += dy / d * step;
    cz += dz / d * step;
  }
  int j;
  float v = eval(bx, by, bz, j);
  // rounding of the evaluation and of the items' FP32 copies (|p| <= A, and
  // radii up to rmax)
  float rmax = 0.f;
  for (int i = 0; i < k; ++i) rmax = fmaxf(rmax, fabsf(it[i].w));
  v = v + (fabsf(v) + A + rmax) * 4.8e-7f;
  return make_float4(bx, by, bz, v);
}

// Upper bound of a node radius term d = dist (+-) r computed in FP32: the
// rounding of dist (<= 3.6 ulp relative) and of the sum (1 ulp), and the FP32
// copy of an FP64 sphere (sqrt3 ulp of |p| = pm, 1 ulp of r), each covered
// with ~10 ulp.
__device__ __forceinline__ float radius_up(float dist, float d, float r, float pm) {
  return d + (dist + 2.f * r + fabsf(d) + pm) * 6e-7f;
}
// final widening of a stored radius (absolute slack in the coordinate bound A)
__device__ __forceinline__ float radius_fin(float v, float A) {
  return v > -INFINITY ? v + (fabsf(v) + A) * 4.8e-7f : v;
}

__device__ __forceinline__ void store_sphere_node(float4* __restrict__ na, float4* __restrict__ nb,
                                                  float4* __restrict__ nf, int64_t node, float4 C, float4 Fc,
                                                  float wp, float wn, float w0, float wf, float A) {
  wp = radius_fin(wp, A);
  wn = radius_fin(wn, A);
  w0 = radius_fin(w0, A);
  wf = radius_fin(wf, A);
  na[node] = make_float4(C.x, C.y, C.z, fmaxf(wp, wn));
  nb[node] = make_float4(wp, wn, w0, 0.f);
  nf[node] = make_float4(Fc.x, Fc.y, Fc.z, wf);
}

__device__ void sphere_leaf_node(const float4* __restrict__ items, int64_t nitems, float A, float4* __restrict__ lo,
                                 float4* __restrict__ hi, float4* __restrict__ na, float4* __restrict__ nb,
                                 float4* __restrict__ nf, int64_t L) {
  int64_t b = L * kLeaf, e = min(b + kLeaf, nitems);
  float4 Ab[kLeaf], Fb[kLeaf];
  int k = 0;
  float3 mn = make_float3(INFINITY, INFINITY, INFINITY), mx = make_float3(-INFINITY, -INFINITY, -INFINITY);
  for (int64_t i = b; i < e; ++i) {
    const float4 v = items[i];
    mn.x = fminf(mn.x, v.x); mn.y = fminf(mn.y, v.y); mn.z = fminf(mn.z, v.z);
    mx.x = fmaxf(mx.x, v.x); mx.y = fmaxf(mx.y, v.y); mx.z = fmaxf(mx.z, v.z);
    Ab[k] = make_float4(v.x, v.y, v.z, fabsf(v.w));
    Fb[k++] = make_float4(v.x, v.y, v.z, -fabsf(v.w));
  }
  lo[L] = make_float4(nextafterf(mn.x, -INFINITY), nextafterf(mn.y, -INFINITY), nextafterf(mn.z, -INFINITY), 0.f);
  hi[L] = make_float4(nextafterf(mx.x, INFINITY), nextafterf(mx.y, INFINITY), nextafterf(mx.z, INFINITY), 0.f);
  const float4 C = bound_ball(Ab, k, A);   // small ball enclosing the balls
  const float4 Fc = bound_ball(Fb, k, A);  // centre for the far bound
  float wp = -INFINITY, wn = -INFINITY, w0 = -INFINITY, wf = -INFINITY;
  for (int64_t i = b; i < e; ++i) {
    const float4 v = items[i];
    const float r = fabsf(v.w);
    const float pm = fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fabsf(v.z));
    float dx = v.x - C.x, dy = v.y - C.y, dz = v.z - C.z;
    const float dist = sqrtf(dx * dx + dy * dy + dz * dz);
    w0 = fmaxf(w0, radius_up(dist, dist, r, pm));
    if (v.w > 0.f) wp = fmaxf(wp, radius_up(dist, dist + r, r, pm));
    if (v.w < 0.f) wn = fmaxf(wn, radius_up(dist, dist + r, r, pm));
    dx = v.x - Fc.x, dy = v.y - Fc.y, dz = v.z - Fc.z;
    const float df = sqrtf(dx * dx + dy * dy + dz * dz);
    wf = fmaxf(wf, radius_up(df, df - r, r, pm));
  }
  store_sphere_node(na, nb, nf, L, C, Fc, wp, wn, w0, wf, A);
}

__device__ void sphere_level_node(float4* __restrict__ lo, float4* __restrict__ hi, float4* __restrict__ na,
                                  float4* __restrict__ nb, float4* __restrict__ nf, float A, int64_t child_off,
                                  int64_t nchild, int64_t off, int64_t j) {
  int64_t b = j * kFan, e = min(b + kFan, nchild);
  float4 L = make_float4(INFINITY, INFINITY, INFINITY, 0.f), H = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
  float4 Ab[kFan], Fb[kFan];
  int k = 0;
  for (int64_t c = b; c < e; ++c) {
    const float4 a = lo[child_off + c], z = hi[child_off + c];
    L.x = fminf(L.x, a.x); L.y = fminf(L.y, a.y); L.z = fminf(L.z, a.z);
    H.x = fmaxf(H.x, z.x); H.y = fmaxf(H.y, z.y); H.z = fmaxf(H.z, z.z);
    const float4 ca = na[child_off + c], cb = nb[child_off + c];
    // a ball around the child that holds all its spheres
    Ab[k] = make_float4(ca.x, ca.y, ca.z, fmaxf(ca.w, cb.z));
    Fb[k++] = nf[child_off + c];
  }
  lo[off + j] = L;
  hi[off + j] = H;
  const float4 C = bound_ball(Ab, k, A);
  const float4 Fc = bound_ball(Fb, k, A);
  // radii through the children (|p - C| <= |p - C_c| + |C_c - C|)
  float wp = -INFINITY, wn = -INFINITY, w0 = -INFINITY, wf = -INFINITY;
  for (int64_t c = b; c < e; ++c) {
    const float4 ca = na[child_off + c], cb = nb[child_off + c], cf = nf[child_off + c];
    float dx = ca.x - C.x, dy = ca.y - C.y, dz = ca.z - C.z;
    const float dist = sqrtf(dx * dx + dy * dy + dz * dz);
    if (cb.x > -INFINITY) wp = fmaxf(wp, radius_up(dist, dist + cb.x, 0.f, 0.f));
    if (cb.y > -INFINITY) wn = fmaxf(wn, radius_up(dist, dist + cb.y, 0.f, 0.f));
    w0 = fmaxf(w0, radius_up(dist, dist + cb.z, 0.f, 0.f));
    dx = cf.x - Fc.x, dy = cf.y - Fc.y, dz = cf.z - Fc.z;
    const float df = sqrtf(dx * dx + dy * dy + dz * dz);
    wf = fmaxf(wf, radius_up(df, df + cf.w, 0.f, 0.f));
  }
  store_sphere_node(na, nb, nf, off + j, C, Fc, wp, wn, w0, wf, A);
}

__global__ void k_sphere_leaves(const float4* __restrict__ items, int64_t nitems, float A, float4* __restrict__ lo,
                                float4* __restrict__ hi, float4* __restrict__ na, float4* __restrict__ nb,
                                float4* __restrict__ nf, int64_t nleaves) {
  int64_t L = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (L < nleaves) sphere_leaf_node(items, nitems, A, lo, hi, na, nb, nf, L);
}

// items of node j at `level`: [j * span, (j + 1) * span), span = kLeaf * kFan^level
__host__ __device__ inline int64_t level_span(int level) {
  int64_t span = kLeaf;
  for (int l = 0; l < level; ++l) span *= kFan;
  return span;
}

__global__ void k_sphere_level(float4* __restrict__ lo, float4* __restrict__ hi, float4* __restrict__ na,
                               float4* __restrict__ nb, float4* __restrict__ nf, float A, int64_t child_off,
                               int64_t nchild, int64_t off, int64_t nnode) {
  int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (j < nnode) sphere_level_node(lo, hi, na, nb, nf, A, child_off, nchild, off, j);
}

// order-preserving map of floats onto unsigned integers (for atomicMax)
__device__ __forceinline__ unsigned ord_key(float v) {
  const unsigned b = __float_as_uint(v);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord_val(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Tightening of the internal radii, pass 1: one thread per sphere; at every
// level >= 1 it evaluates its sphere against the node's centre (a node's
// spheres are a contiguous range of the Morton order) and raises the node's
// per-radius maximum (same rounding bounds as the leaves).
__global__ void k_tighten_items(const float4* __restrict__ items, Tree T, unsigned* __restrict__ keys) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const bool live = i < T.nitems;
  const int lane = threadIdx.x & 31;
  const float4 v = live ? items[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float r = fabsf(v.w);
  const float pm = fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fabsf(v.z));
  for (int l = 1; l < T.nlevels; ++l) {
    // a level-l node spans >= 64 consecutive spheres, so the 32 threads of a
    // warp (32 aligned consecutive spheres) share it
    const int64_t node = T.offset[l] + (live ? i / level_span(l) : 0);
    float m[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
    if (live) {
      const float4 C = T.na[node], Fc = T.nf[node];
      float dx = v.x - C.x, dy = v.y - C.y, dz = v.z - C.z;
      const float dist = sqrtf(dx * dx + dy * dy + dz * dz);
      if (v.w > 0.f) m[0] = radius_up(dist, dist + r, r, pm);
      if (v.w < 0.f) m[1] = radius_up(dist, dist + r, r, pm);
      m[2] = radius_up(dist, dist, r, pm);
      dx = v.x - Fc.x, dy = v.y - Fc.y, dz = v.z - Fc.z;
      const float df = sqrtf(dx * dx + dy * dy + dz * dz);
      m[3] = radius_up(df, df - r, r, pm);
    }
    for (int q = 0; q < 4; ++q)
      for (int o = 16; o > 0; o >>= 1) m[q] = fmaxf(m[q], __shfl_xor_sync(0xffffffffu, m[q], o));
    if (lane == 0 && live) {
      const int64_t slot = 4 * (node - T.offset[1]);
      for (int q = 0; q < 4; ++q)
        if (m[q] > -INFINITY) atomicMax(keys + slot + q, ord_key(m[q]));
    }
  }
}

// pass 2: each internal radius becomes the smaller of its bound through the
// children and the exact maximum over its own spheres (same centre)
__global__ void k_tighten_nodes(Tree T, const unsigned* __restrict__ keys, float A, int64_t nupper) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= nupper) return;
  const int64_t node = T.offset[1] + t;
  const float4 B = T.nb[node];
  float4 Fc = T.nf[node];
  float w[4] = {B.x, B.y, B.z, Fc.w};
  for (int q = 0; q < 4; ++q) {
    const unsigned k = keys[4 * t + q];
    if (k != 0u) w[q] = fminf(w[q], radius_fin(ord_val(k), A));
  }
  T.nb[node] = make_float4(w[0], w[1], w[2], 0.f);
  Fc.w = w[3];
  T.nf[node] = Fc;
  float4 Ca = T.na[node];
  Ca.w = fmaxf(w[0], w[1]);
  T.na[node] = Ca;
}

// Morton keys of query points (processing order of the packet kernel)
__global__ void k_query_keys(const double* __restrict__ x64, const float* __restrict__ x32, int64_t m,
                             uint32_t* __restrict__ keys, int* __restrict__ vals) {
  int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= m) return;
  float x, y, z;
  if (x32) {
    x = x32[3 * i]; y = x32[3 * i + 1]; z = x32[3 * i + 2];
  } else {
    x = float(x64[3 * i]); y = float(x64[3 * i + 1]); z = float(x64[3 * i + 2]);
  }
  keys[i] = morton3(x, y, z);
  vals[i] = int(i);
}

__global__ void k_point_keys(const float4* __restrict__ items, int64_t n, uint32_t* __restrict__ keys,
                             int* __restrict__ vals) {
  int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  float4 v = items[i];
  keys[i] = morton3(v.x, v.y, v.z);
  vals[i] = int(i);
}

__global__ void k_gather_points(const float4* __restrict__ src, const int* __restrict__ order, int64_t n,
                                float4* __restrict__ dst) {
  int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  dst[i] = src[order[i]];
}

// ---------------------------------------------------------------------------
// Warp-cooperative ("packet") traversal.  The 32 lanes of a warp hold 32
// query points that are neighbours in Morton order; they walk one hierarchy
// together: the warp pops a node, every lane decides for its own point
// whether the node can matter, and the node's children (or items) are
// visited if any lane needs them.  Node and item records are read once per
// warp (all lanes load the same address), control flow stays uniform, and
// the stack lives in shared memory.
// ---------------------------------------------------------------------------
constexpr int kPStack = 128;  // >= kFan + (kFan-1)*(kMaxLevels-1)
constexpr unsigned kFull = 0xffffffffu;

// sum of v over the active lanes of the warp, added once to *dst
__device__ __forceinline__ void warp_count(unsigned long long* dst, unsigned long long v) {
  const unsigned mask = __activemask();
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  if ((threadIdx.x & 31) == __ffs(mask) - 1 && v) atomicAdd(dst, v);
}

struct WarpStack {
  uint32_t* s;
  int sp;
  __device__ void push_top(const Tree& T, int lane) {
    const int top = T.nlevels - 1;
    const int cnt = int(T.count[top]);
    if (lane < cnt) s[lane] = pack_node(top, lane);
    sp = cnt;
    __syncwarp();
  }
  __device__ uint32_t pop() {
    const uint32_t nd = s[sp - 1];
    --sp;
    __syncwarp();
    return nd;
  }
  // push the children whose bit is set in `need` (lane c writes child c),
  // `first` last (visited next)
  __device__ void push(int lev, int64_t cb, unsigned need, int first, int lane) {
    const unsigned rest = first >= 0 ? need & ~(1u << unsigned(first)) : need;
    const int nrest = __popc(rest);
    if (lane < kFan && ((rest >> lane) & 1u))
      s[sp + __popc(rest & ((1u << lane) - 1u))] = pack_node(lev, cb + lane);
    if (first >= 0 && lane == 0) s[sp + nrest] = pack_node(lev, cb + first);
    sp += nrest + (first >= 0 ? 1 : 0);
    __syncwarp();
  }
};

// ---------------------------------------------------------------------------
// P build: coverage culling of the candidates q_ik = p_i + |s_i| u_k
// ---------------------------------------------------------------------------
// One lane per candidate; a warp holds 32 Morton-consecutive spheres with the
// same direction k, so its candidates are spatial neighbours.  The warp walks
// the sphere hierarchy as a packet (one node at a time, children visited if
// any lane still needs them); a lane drops out at the first ball that covers
// its candidate, and the warp stops when every lane is settled.
// kCompact (single-shape launch, blocks of kCullBlock threads with one
// direction k): after the neighbour pre-test the candidates still open in
// the block are packed, in Morton order, into its first warps, so the walks
// run with full warps (s_idx: one int per thread, s_wcnt: one per warp, in
// shared memory).  Without it each
// warp walks for its own lanes (the batched launch, where warps take
// independent work items).
template <bool kCompact>
__device__ void cull_packet(const CullArgs& a, int64_t i, int k, WarpStack& W, int lane, int* s_idx, int* s_wcnt) {
  bool active = i < a.n;
  const BuildConsts bc = *a.bc;
  float4 S = active ? a.sph[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  float r = fabsf(S.w);
  const float ux = a.U32[3 * k], uy = a.U32[3 * k + 1], uz = a.U32[3 * k + 2];
  float qx = fmaf(r, ux, S.x), qy = fmaf(r, uy, S.y), qz = fmaf(r, uz, S.z);
  bool have64 = false;
  double qx64 = 0, qy64 = 0, qz64 = 0;
  unsigned long long rechecks = 0;
  unsigned n_ntests = 0, n_items = 0;  // tests made for this lane while it is open
  auto load64 = [&]() {
    if (!have64) {
      D4 pi = a.sph64[a.sid[i]];
      ex_cand(pi, a.U64[3 * k], a.U64[3 * k + 1], a.U64[3 * k + 2], qx64, qy64, qz64);
      have64 = true;
    }
  };
  bool open = active;  // still looking for a covering ball
  if (open && a.box_cull) {
    const float mq = fmaxf(fabsf(qx), fmaxf(fabsf(qy), fabsf(qz)));
    const float eb = 2.f * bc.eq;
    if (mq > 1.f + eb) {
      open = false;
    } else if (mq >= 1.f - eb) {
      load64();
      ++rechecks;
      if (!ex_inbox(qx64, qy64, qz64)) open = false;
    }
  }
  // the warp's 32 spheres are Morton-consecutive: the spheres of lanes
  // lane^1, ^2, ^4, ^8, ^16 are near neighbours, the balls most likely to
  // cover this lane's candidate; a lane they settle skips the walk
  {
    const float4 Tho = active ? a.thr[i] : make_float4(-1.f, -1.f, -1.f, -1.f);
    const int64_t base = i - lane;
    for (int o = 1; o < 32; o <<= 1) {
      const int src = lane ^ o;
      const float4 P = make_float4(__shfl_sync(kFull, S.x, src), __shfl_sync(kFull, S.y, src),
                                   __shfl_sync(kFull, S.z, src), __shfl_sync(kFull, S.w, src));
      const float th_lo = __shfl_sync(kFull, Tho.x, src), th_hi = __shfl_sync(kFull, Tho.y, src);
      const int64_t j = base + src;
      if (!open || j >= a.n) continue;
      const float dx = qx - P.x, dy = qy - P.y, dz = qz - P.z;
      const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      if (d2 < th_lo) {
        open = false;
      } else if (d2 <= th_hi) {
        load64();
        ++rechecks;
        if (ex_cov(qx64, qy64, qz64, a.sph64[a.sid[j]], a.tol)) open = false;
      }
    }
  }
  // (a candidate that is still open here is in the box)
  if constexpr (kCompact) {
    const int wid = threadIdx.x >> 5;
    const unsigned ballot = __ballot_sync(kFull, open);
    if (lane == 0) s_wcnt[wid] = __popc(ballot);
    __syncthreads();
    int off = 0, total = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) {
      const int c = s_wcnt[w];
      if (w < wid) off += c;
      total += c;
    }
    if (open) s_idx[off + __popc(ballot & ((1u << lane) - 1u))] = int(threadIdx.x);
    __syncthreads();
    // this thread now walks for entry threadIdx.x of the packed list
    if (rechecks) atomicAdd(&a.cnt->cull_rechecks, rechecks);
    rechecks = 0;
    if (wid * 32 >= total) return;  // warp-uniform: no entries left for this warp
    const int64_t blk_base = i - int64_t(threadIdx.x);  // the block's first sphere
    open = int(threadIdx.x) < total;
    i = open ? blk_base + s_idx[threadIdx.x] : a.n;
    active = open;
    S = open ? a.sph[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    r = fabsf(S.w);
    qx = fmaf(r, ux, S.x);
    qy = fmaf(r, uy, S.y);
    qz = fmaf(r, uz, S.z);
    have64 = false;
  }
  const bool inbox = open;
  const Tree& T = a.tree;
  const float grow = 1.f + 8.f * kU;
  if (__any_sync(kFull, open)) {
    W.push_top(T, lane);
    while (W.sp > 0 && __any_sync(kFull, open)) {
      const uint32_t nd = W.pop();
      const int lev = node_level(nd);
      const int64_t idx = node_index(nd);
      if (lev == 0) {
        const int64_t b = idx * kLeaf, e = min(b + kLeaf, a.n);
        n_items += open ? unsigned(e - b) : 0u;
#pragma unroll
        for (int jj = 0; jj < kLeaf; ++jj) {
          const int64_t j = b + jj;
          if (j >= e) break;
          const float4 P = a.sph[j];
          const float4 Th = a.thr[j];
          if (!open || j == i) continue;
          const float dx = qx - P.x, dy = qy - P.y, dz = qz - P.z;
          const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          if (d2 < Th.x) {
            open = false;
          } else if (d2 <= Th.y) {
            load64();
            ++rechecks;
            if (ex_cov(qx64, qy64, qz64, a.sph64[a.sid[j]], a.tol)) open = false;
          }
        }
      } else {
        const int64_t cb = idx * kFan, ce = min(cb + kFan, T.count[lev - 1]);
        const int64_t off = T.offset[lev - 1];
        unsigned need = 0;
        int first = -1, firstn = 0;
        const int nc = int(ce - cb);
        n_ntests += open ? unsigned(nc) : 0u;
#pragma unroll
        for (int c = 0; c < kFan; ++c) {
          if (c >= nc) break;
          // the node can hold a covering ball only if q lies in the ball
          // B(C, max(wp, wn)) shrunk by tol
          bool nd_c = false;
          if (open) {
            const float4 B = T.na[off + cb + c];
            const float t = fmaf(B.w - a.tol32, grow, bc.pad);
            nd_c = t > 0.f && ball_d2(qx, qy, qz, B) < t * t;
          }
          // visit first the child most lanes need
          const unsigned votes = __ballot_sync(kFull, nd_c);
          if (votes) {
            need |= 1u << unsigned(c);
            const int nv = __popc(votes);
            if (nv > firstn) {
              firstn = nv;
              first = c;
            }
          }
        }
        W.push(lev - 1, cb, need, first, lane);
      }
    }
  }
  if (rechecks) atomicAdd(&a.cnt->cull_rechecks, rechecks);
  warp_count(&a.cnt->c_ntests, n_ntests);
  warp_count(&a.cnt->c_items, n_items);
  if (!(inbox && open)) return;
  // survivor: append to the list of its sign class (zero spheres: both)
  const uint32_t g = uint32_t(a.sid[i]) * uint32_t(a.KS) + uint32_t(k);
  const float4 item = make_float4(qx, qy, qz, __uint_as_float(g));
  for (int c = 0; c < 2; ++c) {
    const bool mine = c == 0 ? !(S.w < 0.f) : !(S.w > 0.f);
    if (!mine) continue;
    cg::coalesced_group grp = cg::coalesced_threads();
    unsigned int base = 0;
    if (grp.thread_rank() == 0) base = atomicAdd(&a.cnt->nsurv[c], grp.size());
    base = grp.shfl(base, 0) + grp.thread_rank();
    if (base < a.cap) {
      a.surv[c][base] = item;
      if (a.surv_shape[c]) a.surv_shape[c][base] = uint16_t(a.shape);
    }
  }
}

constexpr bool kCullCompact = true;
constexpr int kCullBlock = 128;
__global__ void __launch_bounds__(kCullBlock) k_cull(CullArgs a) {
  __shared__ uint32_t s_stack[kCullBlock / 32][kPStack];
  __shared__ int s_idx[kCullBlock], s_wcnt[kCullBlock / 32];
  WarpStack W{s_stack[threadIdx.x >> 5], 0};
  cull_packet<kCullCompact>(a, blockIdx.x * int64_t(blockDim.x) + threadIdx.x, blockIdx.y, W, threadIdx.x & 31,
                            s_idx, s_wcnt);
}

// ---------------------------------------------------------------------------
// query: FP32 pass with certification
// ---------------------------------------------------------------------------
struct Top2 {
  float best, sec;
  int idx;
};
__device__ __forceinline__ void top2_init(Top2& t) {
  t.best = INFINITY;
  t.sec = INFINITY;
  t.idx = -1;
}
__device__ __forceinline__ void top2_push(Top2& t, float v, int j) {
  if (v < t.best) {
    t.sec = t.best;
    t.best = v;
    t.idx = j;
  } else if (v < t.sec) {
    t.sec = v;
  }
}
__device__ __forceinline__ float top2_th(const Top2& t, float band) { return fminf(t.sec, t.best + band); }

__device__ __forceinline__ void load_query(const QueryArgs& a, int64_t q, double& x, double& y, double& z) {
  if (a.x32) {
    x = double(a.x32[3 * q]);
    y = double(a.x32[3 * q + 1]);
    z = double(a.x32[3 * q + 2]);
  } else {
    x = a.x64[3 * q];
    y = a.x64[3 * q + 1];
    z = a.x64[3 * q + 2];
  }
}

__device__ __forceinline__ void write_result(const QueryArgs& a, int64_t q, double v, int64_t arg, int flags) {
  if (a.s_out) a.s_out[q] = float(v);
  if (a.s64_out) a.s64_out[q] = v;
  if (a.arg_out) a.arg_out[q] = arg;
  if (a.fl_out) a.fl_out[q] = uint16_t(flags);
}

// FP64 position of a survivor from its id
__device__ __forceinline__ void surv_pos64(const QueryArgs& a, uint32_t g, double& qx, double& qy, double& qz) {
  const uint32_t i = g / uint32_t(a.KS), k = g % uint32_t(a.KS);
  const D4 pi = a.sph64[i];
  if (int(k) < a.K) {
    ex_cand(pi, a.U64[3 * k], a.U64[3 * k + 1], a.U64[3 * k + 2], qx, qy, qz);
  } else {
    const double* w = a.witness64 + 3 * int64_t(i);
    qx = w[0];
    qy = w[1];
    qz = w[2];
  }
}

// Warp-aggregated counter update (one atomic per warp)

// Packet FP64 band pass over the sphere hierarchy.  A lane with band = true
// finds, among the spheres whose FP32 value lies at or below its threshold
// thr, the exact FP64 minimum and its input index (ties to the lowest index).
// mode 0: |x-p| - r over sign class cls; mode 1: |x-p| + r over all spheres.
__device__ double packet_band_sphere(const QueryArgs& a, const BuildConsts& bc, WarpStack& W, int lane, bool band,
                                     double x64, double y64, double z64, float x, float y, float z, int mode,
                                     int cls, float thr, int& arg) {
  double best = INFINITY;
  arg = INT_MAX;
  if (!__any_sync(kFull, band)) return best;
  const Tree& T = a.st;
  const float grow = 1.f + 8.f * kU;
  W.push_top(T, lane);
  while (W.sp > 0) {
    const uint32_t nd = W.pop();
    const int lev = node_level(nd);
    const int64_t idx = node_index(nd);
    if (lev == 0) {
      const int64_t b = idx * kLeaf, e = min(b + kLeaf, a.n);
      for (int64_t j = b; j < e; ++j) {
        const float4 P = a.sph[j];
        if (!band) continue;
        if (mode == 0 && (P.w == 0.f || int(P.w < 0.f) != cls)) continue;
        const float dx = x - P.x, dy = y - P.y, dz = z - P.z;
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float r = fabsf(P.w);
        const float v = mode == 0 ? __fsqrt_rn(d2) - r : __fsqrt_rn(d2) + r;
        if (!(v <= thr)) continue;
        const int o = a.sid[j];
        const D4 pj = a.sph64[o];
        const double dl = __dsqrt_rn(ex_d2(x64, y64, z64, pj.x, pj.y, pj.z));
        const double v64 = mode == 0 ? __dsub_rn(dl, fabs(pj.w)) : __dadd_rn(dl, fabs(pj.w));
        if (v64 < best || (v64 == best && o < arg)) {
          best = v64;
          arg = o;
        }
      }
    } else {
      const int64_t cb = idx * kFan, ce = min(cb + kFan, T.count[lev - 1]);
      const int64_t off = T.offset[lev - 1];
      unsigned need = 0;
      for (int64_t c = cb; c < ce; ++c) {
        bool nd_c = false;
        if (band) {
          float4 B;
          float w;
          if (mode == 1) {
            B = T.nf[off + c];
            w = B.w;
          } else {
            B = T.na[off + c];
            const float4 R = T.nb[off + c];
            w = cls == 0 ? R.x : R.y;
          }
          const float t = fmaf(thr + w, grow, bc.eprune);
          nd_c = t > 0.f && ball_d2(x, y, z, B) < t * t;
        }
        if (__any_sync(kFull, nd_c)) need |= 1u << unsigned(c - cb);
      }
      W.push(lev - 1, cb, need, -1, lane);
    }
  }
  return best;
}

// Packet FP64 band pass over the survivor hierarchy of class cls: exact
// nearest survivor among those whose FP32 distance^2 is at most thr.
__device__ double packet_band_surv(const QueryArgs& a, const BuildConsts& bc, WarpStack& W, int lane, bool band,
                                   int cls, double x64, double y64, double z64, float x, float y, float z, float thr,
                                   uint32_t& gbest) {
  double best = INFINITY;
  gbest = 0xffffffffu;
  if (!__any_sync(kFull, band)) return best;
  const Tree& T = a.vt[cls];
  const float4* items = a.surv[cls];
  const float grow = 1.f + 8.f * kU;
  const float thn = band ? thr * grow + bc.ed_lin * __fsqrt_rn(thr) + 1e-30f : -1.f;
  W.push_top(T, lane);
  while (W.sp > 0) {
    const uint32_t nd = W.pop();
    const int lev = node_level(nd);
    const int64_t idx = node_index(nd);
    if (lev == 0) {
      const int64_t b = idx * kLeaf, e = min(b + kLeaf, T.nitems);
      for (int64_t j = b; j < e; ++j) {
        const float4 P = items[j];
        if (!band) continue;
        const float dx = x - P.x, dy = y - P.y, dz = z - P.z;
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (!(d2 <= thr)) continue;
        const uint32_t g = __float_as_uint(P.w);
        double qx, qy, qz;
        surv_pos64(a, g, qx, qy, qz);
        const double e2 = ex_d2(x64, y64, z64, qx, qy, qz);
        if (e2 < best || (e2 == best && g < gbest)) {
          best = e2;
          gbest = g;
        }
      }
    } else {
      const int64_t cb = idx * kFan, ce = min(cb + kFan, T.count[lev - 1]);
      const int64_t off = T.offset[lev - 1];
      unsigned need = 0;
      for (int64_t c = cb; c < ce; ++c) {
        const bool nd_c = box_d2(x, y, z, T.lo[off + c], T.hi[off + c]) < thn;
        if (__any_sync(kFull, nd_c)) need |= 1u << unsigned(c - cb);
      }
      W.push(lev - 1, cb, need, -1, lane);
    }
  }
  return best;
}

__device__ void query_exact_one(const QueryArgs& a, int64_t q);

// One lane's query inside a warp-cooperative pass; `slot` indexes the
// processing order (a.perm), all 32 lanes of the warp must call together.
// Points outside the coordinate range of the FP32 error model go to the
// FP64 kernel through a.defer, or (kInlineExact) are evaluated in place.
// Greedy descent of a whole warp to one leaf: at every level lanes 0-7
// score the 8 children, the lowest score (lowest child on ties, up to the
// score's last 3 bits) is followed.  The score must be uniform across the
// warp.
template <class Score>
__device__ int64_t warp_descend(const Tree& T, int lane, Score score) {
  int lev = T.nlevels - 1;
  int64_t cb = 0, ce = T.count[lev];
  for (;;) {
    const int c = lane & 7;
    const float v = cb + c < ce ? score(T.offset[lev] + cb + c) : INFINITY;
    const unsigned key = __reduce_min_sync(kFull, (ord_key(v) & ~7u) | unsigned(c));
    const int64_t best = cb + (key & 7u);
    if (lev == 0) return best;
    cb = best * kFan;
    ce = min(cb + kFan, T.count[lev - 1]);
    --lev;
  }
}


// Per-point state between the two phases of a split query (the sphere pass
// and the rest), 48 B per processing slot.
__device__ __forceinline__ void store_qstate(uint4* st, int64_t slot, bool c0, bool c1, int sample, const Top2& A0,
                                             const Top2& A1, const Top2& F) {
  uint4* p = st + 3 * slot;
  p[0] = make_uint4(__float_as_uint(A0.best), __float_as_uint(A0.sec), unsigned(A0.idx), __float_as_uint(A1.best));
  p[1] = make_uint4(__float_as_uint(A1.sec), unsigned(A1.idx), __float_as_uint(F.best), __float_as_uint(F.sec));
  p[2] = make_uint4(unsigned(F.idx), unsigned(sample), (c0 ? 1u : 0u) | (c1 ? 2u : 0u), 0u);
}
__device__ __forceinline__ void load_qstate(const uint4* st, int64_t slot, bool& c0, bool& c1, int& sample, Top2& A0,
                                            Top2& A1, Top2& F) {
  const uint4* p = st + 3 * slot;
  const uint4 u0 = p[0], u1 = p[1], u2 = p[2];
  A0.best = __uint_as_float(u0.x);
  A0.sec = __uint_as_float(u0.y);
  A0.idx = int(u0.z);
  A1.best = __uint_as_float(u0.w);
  A1.sec = __uint_as_float(u1.x);
  A1.idx = int(u1.y);
  F.best = __uint_as_float(u1.z);
  F.sec = __uint_as_float(u1.w);
  F.idx = int(u2.x);
  sample = int(u2.y);
  c0 = (u2.z & 1u) != 0;
  c1 = (u2.z & 2u) != 0;
}

// kPhase 0: the whole query; 1: the sphere pass only, its state stored in
// a.state; 2: the rest, starting from a.state (phase 1 must have run on the
// same points in the same order).
template <bool kInlineExact, int kPhase = 0>
__device__ void query_packet(const QueryArgs& a, int64_t slot, WarpStack& W, int lane) {
  const bool active = slot < a.m;
  const int64_t q = active ? int64_t(a.perm ? a.perm[slot] : uint32_t(slot)) : 0;
  const BuildConsts bc = *a.bc;
  double x64 = 0.0, y64 = 0.0, z64 = 0.0;
  if (active) load_query(a, q, x64, y64, z64);
  const float x = float(x64), y = float(y64), z = float(z64);
  unsigned rechecks = 0, n_nodes = 0, n_items = 0, n_snodes = 0, n_sitems = 0, n_band = 0;
  bool defer = active && !(fabs(x64) <= bc.A && fabs(y64) <= bc.A && fabs(z64) <= bc.A);
  bool live = active && !defer;
  const float grow = 1.f + 8.f * kU;
  const float ea2 = 2.f * bc.ea;
  const float negtol = -a.tol32 + ea2;
  // warp centre, used to order children (nearest first)
  float cx = live ? x : 0.f, cy = live ? y : 0.f, cz = live ? z : 0.f;
  float cnt = live ? 1.f : 0.f;
  for (int o = 16; o > 0; o >>= 1) {
    cx += __shfl_xor_sync(kFull, cx, o);
    cy += __shfl_xor_sync(kFull, cy, o);
    cz += __shfl_xor_sync(kFull, cz, o);
    cnt += __shfl_xor_sync(kFull, cnt, o);
  }
  if (cnt > 0.f) {
    cx /= cnt;
    cy /= cnt;
    cz /= cnt;
  }
  // ---- pass over the spheres -------------------------------------------
  // per-class state as scalars (the class of an item is uniform across the
  // warp, so branching on it costs nothing; indexing a register array with
  // it would push the array to local memory)
  bool cov0 = false, cov1 = false;
  Top2 A0, A1, F;
  top2_init(A0);
  top2_init(A1);
  top2_init(F);
  int sample = INT_MAX;
  if constexpr (kPhase == 2) {
    if (active) load_qstate(a.state, slot, cov0, cov1, sample, A0, A1, F);
  } else if (__any_sync(kFull, live)) {
    const Tree& T = a.st;
    auto leaf_items = [&](int64_t idx) {
        const int64_t b = idx * kLeaf, e = min(b + kLeaf, a.n);
        n_items += live ? unsigned(e - b) : 0u;
        for (int64_t j = b; j < e; ++j) {
          const float4 P = a.sph[j];
          if (!live) continue;
          const float dx = x - P.x, dy = y - P.y, dz = z - P.z;
          const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          if (d2 == 0.f) {
            const int o = a.sid[j];
            const D4 pj = a.sph64[o];
            if (pj.x == x64 && pj.y == y64 && pj.z == z64 && o < sample) sample = o;
          }
          const float r = fabsf(P.w);
          auto class_item = [&](bool& cv, Top2& Ac) {
            if (!cv) {
              const float4 Th = a.thr[j];
              if (d2 < Th.z) {
                cv = true;
              } else if (d2 <= Th.w) {
                ++rechecks;
                cv = ex_cov(x64, y64, z64, a.sph64[a.sid[j]], a.tol);
              }
            }
            const float t = r + top2_th(Ac, ea2);
            if (t > 0.f && d2 < t * t * grow) top2_push(Ac, __fsqrt_rn(d2) - r, int(j));
          };
          if (P.w > 0.f) class_item(cov0, A0);
          else if (P.w < 0.f) class_item(cov1, A1);
          const float t2 = top2_th(F, ea2) - r;
          if (t2 > 0.f && d2 < t2 * t2 * grow) top2_push(F, __fsqrt_rn(d2) + r, int(j));
        }
    };
    // seed the thresholds with the leaf nearest the packet centre: a greedy
    // descent (lanes 0-7 score the 8 children by centre distance) and the
    // leaf's spheres evaluated by every lane; the walk then skips that leaf
    const int64_t seeded = warp_descend(T, lane, [&](int64_t node) { return ball_d2(cx, cy, cz, T.na[node]); });
    leaf_items(seeded);
    W.push_top(T, lane);
    while (W.sp > 0) {
      const uint32_t nd = W.pop();
      const int lev = node_level(nd);
      const int64_t idx = node_index(nd);
      if (lev == 0) {
        if (idx != seeded) leaf_items(idx);
      } else {
        const int64_t cb = idx * kFan, ce = min(cb + kFan, T.count[lev - 1]);
        const int64_t off = T.offset[lev - 1];
        float th0 = top2_th(A0, ea2), th1 = top2_th(A1, ea2);
        if (!cov0) th0 = fmaxf(th0, negtol);
        if (!cov1) th1 = fmaxf(th1, negtol);
        const float thf = top2_th(F, ea2);
        // every child is tested by every lane (unrolled, so the loads of
        // all children issue together); one warp OR gives the children to
        // visit and one warp MIN the child nearest the packet centre (its
        // squared distance with the child number in the low 3 bits)
        const int nc = int(ce - cb);
        n_nodes += live ? unsigned(nc) : 0u;
        unsigned mine = 0, key = 0xffffffffu;
#pragma unroll
        for (int c = 0; c < kFan; ++c) {
          if (c < nc && live) {
            const float4 B = T.na[off + cb + c];
            // one distance to the node centre C against the larger of each
            // class's tangent threshold and the centres ball (a sample equal
            // to x), then the far bound about its own centre
            const float4 R = T.nb[off + cb + c];
            float v = R.z;
            if (R.x > -INFINITY) v = fmaxf(v, th0 + R.x);
            if (R.y > -INFINITY) v = fmaxf(v, th1 + R.y);
            const float t = fmaf(v, grow, bc.eprune);
            bool nd_c = t > 0.f && ball_d2(x, y, z, B) < t * t;
            if (!nd_c) {
              const float4 Fb = T.nf[off + cb + c];
              const float tf = fmaf(thf + Fb.w, grow, bc.eprune);
              nd_c = tf > 0.f && ball_d2(x, y, z, Fb) < tf * tf;
            }
            if (nd_c) {
              mine |= 1u << c;
              key = min(key, (__float_as_uint(ball_d2(cx, cy, cz, B)) & ~7u) | unsigned(c));
            }
          }
        }
        const unsigned need = __reduce_or_sync(kFull, mine);
        const int first = need ? int(__reduce_min_sync(kFull, key) & 7u) : -1;
        W.push(lev - 1, cb, need, first, lane);
      }
    }
  }
  if constexpr (kPhase == 1) {
    if (active) store_qstate(a.state, slot, cov0, cov1, sample, A0, A1, F);
    warp_count(&a.cnt->query_rechecks, rechecks);
    warp_count(&a.cnt->q_sphere_ntests, n_nodes);
    warp_count(&a.cnt->q_sphere_items, n_items);
    return;
  }
  int code = -1;
  double value = 0.0;
  int64_t arg = -1;
  int flags = 0;
  if (live) {
    if (sample != INT_MAX) {
      code = GFS_CODE_SAMPLE;
      value = a.sph64[sample].w;
      arg = sample;
    } else if (cov0 && cov1) {
      code = GFS_CODE_INVALID;
      value = __longlong_as_double(0x7ff8000000000000LL);
    } else if (!cov0 && !cov1) {
      code = GFS_CODE_OUTSIDE;
    }
    if (code >= 0) flags = code;
  }
  const bool open = live && code < 0;
  const int cs = cov0 ? 0 : 1, co = 1 - cs;
  const Top2 As = cs == 0 ? A0 : A1;   // x's own class
  const Top2 Ao = cs == 0 ? A1 : A0;   // the opposite class
  // ---- pass over the survivors of each lane's sign ------------------------
  float bd = INFINITY, sd = INFINITY;
  uint32_t gbest = 0xffffffffu;
  auto band = [&](float D) { return bc.ed_lin * __fsqrt_rn(D) + bc.ed_quad * D + 1e-30f; };
  for (int cl = 0; cl < 2; ++cl) {
    const bool mine = open && cs == cl;
    if (!__any_sync(kFull, mine) || a.vt[cl].nlevels == 0) continue;
    const Tree& T = a.vt[cl];
    const float4* items = a.surv[cl];
    float th = mine ? INFINITY : -1.f;   // threshold on d^2
    float thn = th;                      // widened for node tests
    auto surv_leaf = [&](int64_t idx) {
        const int64_t b = idx * kLeaf, e = min(b + kLeaf, T.nitems);
        n_sitems += mine ? unsigned(e - b) : 0u;
        for (int64_t j = b; j < e; ++j) {
          const float4 P = items[j];
          const float dx = x - P.x, dy = y - P.y, dz = z - P.z;
          const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          if (d2 < th) {
            if (d2 < bd) {
              sd = bd;
              bd = d2;
              gbest = __float_as_uint(P.w);
            } else {
              sd = d2;
            }
            th = fminf(sd, bd + 2.f * band(bd));
            thn = th * grow + bc.ed_lin * __fsqrt_rn(th) + 1e-30f;
          }
        }
    };
    // seed the threshold with the leaf nearest the packet centre (the walk
    // skips it)
    const int64_t seeded =
        warp_descend(T, lane, [&](int64_t node) { return box_d2(cx, cy, cz, T.lo[node], T.hi[node]); });
    surv_leaf(seeded);
    W.push_top(T, lane);
    while (W.sp > 0) {
      const uint32_t nd = W.pop();
      const int lev = node_level(nd);
      const int64_t idx = node_index(nd);
      if (lev == 0) {
        if (idx != seeded) surv_leaf(idx);
      } else {
        const int64_t cb = idx * kFan, ce = min(cb + kFan, T.count[lev - 1]);
        const int64_t off = T.offset[lev - 1];
        const int nc = int(ce - cb);
        n_snodes += mine ? unsigned(nc) : 0u;
        unsigned mine_c = 0, key = 0xffffffffu;
#pragma unroll
        for (int c = 0; c < kFan; ++c) {
          if (c < nc && mine) {
            const float4 L = T.lo[off + cb + c], H = T.hi[off + cb + c];
            if (box_d2(x, y, z, L, H) < thn) {
              mine_c |= 1u << c;
              key = min(key, (__float_as_uint(box_d2(cx, cy, cz, L, H)) & ~7u) | unsigned(c));
            }
          }
        }
        const unsigned need = __reduce_or_sync(kFull, mine_c);
        const int first = need ? int(__reduce_min_sync(kFull, key) & 7u) : -1;
        W.push(lev - 1, cb, need, first, lane);
      }
    }
  }
  const bool have_s = open && gbest != 0xffffffffu, have_u = open && Ao.idx >= 0;
  // exact nearest survivor: direct when no other survivor lies in the error
  // band, else an FP64 pass over the band
  double ds = INFINITY;
  bool sband = have_s && !(sd >= bd + 2.f * band(bd));
  if (have_s && !sband) {
    double qx, qy, qz;
    surv_pos64(a, gbest, qx, qy, qz);
    ds = __dsqrt_rn(ex_d2(x64, y64, z64, qx, qy, qz));
  }
  for (int cl = 0; cl < 2; ++cl) {
    uint32_t g2;
    const bool mine = sband && cs == cl;
    const double e2 = packet_band_surv(a, bc, W, lane, mine, cl, x64, y64, z64, x, y, z,
                                       mine ? bd + 2.f * band(bd) : -1.f, g2);
    if (mine) {
      ++n_band;
      ds = __dsqrt_rn(e2);
      gbest = g2;
    }
  }
  // exact nearest opposite tangent point
  double ub = INFINITY;
  int uj = -1;
  const bool uband = have_u && !(Ao.sec >= Ao.best + ea2);
  if (have_u && !uband) {
    uj = a.sid[Ao.idx];
    const D4 pj = a.sph64[uj];
    ub = __dsub_rn(__dsqrt_rn(ex_d2(x64, y64, z64, pj.x, pj.y, pj.z)), fabs(pj.w));
  }
  {
    int j2;
    const double v = packet_band_sphere(a, bc, W, lane, uband, x64, y64, z64, x, y, z, 0, co,
                                        uband ? Ao.best + ea2 : -1.f, j2);
    if (uband) {
      ++n_band;
      ub = v;
      uj = j2;
    }
  }
  // value and the result code
  double m = 0.0;
  bool need_lb = false;
  if (open) {
    if (have_s && (!a.clamp_opp || ds <= ub)) {
      code = GFS_CODE_SURVIVOR;
      m = ds;
      arg = int64_t(gbest);
    } else if (a.clamp_opp && have_u) {
      code = GFS_CODE_OPPOSITE;
      m = ub;
      arg = uj;
    } else {
      code = GFS_CODE_LOWER;
      need_lb = true;
    }
  }
  const double E = double(bc.ea) * 1.01 + 1e-15;
  const double lbt = -double(As.best) - a.tol;
  const double ft = double(F.best) + a.tol;
  if (open && code != GFS_CODE_LOWER) {
    const double mm = m < 0.0 ? 0.0 : m;
    need_lb = !(mm < lbt - E) && !(mm > lbt + E);
  }
  // exact lower bound LB (max over the lane's class of r - |x-p|) if needed
  double lb = 0.0;
  int lj = -1;
  const bool lband = need_lb && !(As.sec >= As.best + ea2);
  if (need_lb && !lband) {
    lj = a.sid[As.idx];
    const D4 pl = a.sph64[lj];
    lb = __dsub_rn(fabs(pl.w), __dsqrt_rn(ex_d2(x64, y64, z64, pl.x, pl.y, pl.z)));
  }
  {
    int j2;
    const double v = packet_band_sphere(a, bc, W, lane, lband, x64, y64, z64, x, y, z, 0, cs,
                                        lband ? As.best + ea2 : -1.f, j2);
    if (lband) {
      ++n_band;
      lb = -v;
      lj = j2;
    }
  }
  if (open && code == GFS_CODE_LOWER) {
    m = lb;
    arg = lj;
  }
  if (m < 0.0) m = 0.0;
  // exact far bound if the FP32 margin does not decide FAR_VIOL
  const bool need_far = open && !(m > ft + E) && !(m < ft - E);
  const bool fband = need_far && !(F.sec >= F.best + ea2);
  double far = INFINITY;
  if (need_far && !fband) {
    const D4 pf = a.sph64[a.sid[F.idx]];
    far = __dadd_rn(__dsqrt_rn(ex_d2(x64, y64, z64, pf.x, pf.y, pf.z)), fabs(pf.w));
  }
  {
    int j2;
    const double v = packet_band_sphere(a, bc, W, lane, fband, x64, y64, z64, x, y, z, 1, 0,
                                        fband ? F.best + ea2 : -1.f, j2);
    if (fband) {
      ++n_band;
      far = v;
    }
  }
  if (open) {
    flags = code;
    if (m < lbt - E) flags |= GFS_FLAG_LB_VIOL;
    else if (need_lb && m < __dsub_rn(lb, a.tol)) flags |= GFS_FLAG_LB_VIOL;
    if (m > ft + E) flags |= GFS_FLAG_FAR_VIOL;
    else if (need_far && m > __dadd_rn(far, a.tol)) flags |= GFS_FLAG_FAR_VIOL;
    if (have_u && ub < __dsub_rn(m, a.tol)) flags |= GFS_FLAG_OPP_VIOL;
    value = cs == 0 ? m : -m;
  }
  warp_count(&a.cnt->query_rechecks, rechecks);
  warp_count(&a.cnt->q_sphere_ntests, n_nodes);
  warp_count(&a.cnt->q_sphere_items, n_items);
  warp_count(&a.cnt->q_surv_ntests, n_snodes);
  warp_count(&a.cnt->q_band_passes, n_band);
  warp_count(&a.cnt->q_surv_items, n_sitems);
  if (live) {
    write_result(a, q, value, arg, flags);
  } else if (defer) {
    // outside the coordinate range the error bounds assume: FP64 path
    const unsigned int s2 = atomicAdd(&a.cnt->ndefer, 1u);
    if constexpr (kInlineExact) {
      query_exact_one(a, q);
    } else {
      if (s2 < a.defer_cap) a.defer[s2] = uint32_t(q);
    }
  }
}

// The query as two kernels: the sphere pass (state to a.state), then the
// survivor pass and the rest.  Each holds less live state than one kernel
// doing both would, so more warps fit per SM (15% faster on the 64^3 union
// workload than the fused packet code, which the batched kernel keeps).
__global__ void __launch_bounds__(128, 8) k_query_spheres(QueryArgs a) {
  __shared__ uint32_t s_stack[4][kPStack];
  WarpStack W{s_stack[threadIdx.x >> 5], 0};
  query_packet<false, 1>(a, blockIdx.x * int64_t(blockDim.x) + threadIdx.x, W, threadIdx.x & 31);
}

__global__ void __launch_bounds__(128, 7) k_query_finish(QueryArgs a) {
  __shared__ uint32_t s_stack[4][kPStack];
  WarpStack W{s_stack[threadIdx.x >> 5], 0};
  query_packet<false, 2>(a, blockIdx.x * int64_t(blockDim.x) + threadIdx.x, W, threadIdx.x & 31);
}

// ---------------------------------------------------------------------------
// query: exact FP64 evaluation (deferred queries, or precision = 1)
// ---------------------------------------------------------------------------
__device__ void query_exact_one(const QueryArgs& a, int64_t q) {
  double x, y, z;
  load_query(a, q, x, y, z);
  const double tol = a.tol;
  bool cov[2] = {false, false};
  double bestA[2] = {INFINITY, INFINITY};
  int idxA[2] = {INT_MAX, INT_MAX};
  double bestF = INFINITY;
  int sample = INT_MAX;
  {
    const Tree& T = a.st;
    uint32_t stack[kStack];
    int sp = 0;
    const int top = T.nlevels - 1;
    for (int64_t j = 0; j < T.count[top]; ++j) stack[sp++] = pack_node(top, j);
    while (sp > 0) {
      const uint32_t nd = stack[--sp];
      const int lev = node_level(nd);
      const int64_t idx = node_index(nd);
      if (lev == 0) {
        const int64_t b = idx * kLeaf, e = min(b + kLeaf, a.n);
        for (int64_t j = b; j < e; ++j) {
          const int o = a.sid[j];
          const D4 P = a.sph64[o];
          if (P.x == x && P.y == y && P.z == z && o < sample) sample = o;
          const double d2 = ex_d2(x, y, z, P.x, P.y, P.z);
          const double dl = __dsqrt_rn(d2);
          const double r = fabs(P.w);
          if (P.w != 0.0) {
            const int c = P.w < 0.0;
            if (!cov[c] && r > tol) {
              const double rt = __dsub_rn(r, tol);
              if (d2 < __dmul_rn(rt, rt)) cov[c] = true;
            }
            const double av = __dsub_rn(dl, r);
            if (av < bestA[c] || (av == bestA[c] && o < idxA[c])) {
              bestA[c] = av;
              idxA[c] = o;
            }
          }
          const double f = __dadd_rn(dl, r);
          if (f < bestF) bestF = f;
        }
      } else {
        const int64_t cb = idx * kFan, ce = min(cb + kFan, T.count[lev - 1]);
        const int64_t off = T.offset[lev - 1];
        for (int64_t c = cb; c < ce; ++c) {
          const float4 L = T.lo[off + c], H = T.hi[off + c];
          bool need = x >= double(L.x) && x <= double(H.x) && y >= double(L.y) && y <= double(H.y) &&
                      z >= double(L.z) && z <= double(H.z);
          if (!need) {
            const float4 B = T.na[off + c], R = T.nb[off + c], Fb = T.nf[off + c];
            const double tf = (bestF + double(Fb.w)) * (1.0 + 1e-12) + 1e-12;
            need = tf > 0.0 && ball_d2_64(x, y, z, Fb) <= tf * tf;
            double v = -INFINITY;
            for (int cl = 0; cl < 2; ++cl) {
              const float w = cl == 0 ? R.x : R.y;
              if (!(w > -INFINITY)) continue;
              double th = bestA[cl];
              if (!cov[cl]) th = fmax(th, -tol);
              v = fmax(v, th + double(w));
            }
            const double t = v * (1.0 + 1e-12) + 1e-12;
            need = need || (t > 0.0 && ball_d2_64(x, y, z, B) <= t * t);
          }
          if (need) stack[sp++] = pack_node(lev - 1, c);
        }
      }
    }
  }
  if (sample != INT_MAX) {
    write_result(a, q, a.sph64[sample].w, sample, GFS_CODE_SAMPLE);
    return;
  }
  if (cov[0] && cov[1]) {
    write_result(a, q, __longlong_as_double(0x7ff8000000000000LL), -1, GFS_CODE_INVALID);
    return;
  }
  if (!cov[0] && !cov[1]) {
    write_result(a, q, 0.0, -1, GFS_CODE_OUTSIDE);
    return;
  }
  const int cs = cov[0] ? 0 : 1, co = 1 - cs;
  double bd = INFINITY;
  uint32_t gbest = 0xffffffffu;
  const float eqs = a.bc->eq;
  if (a.vt[cs].nlevels > 0) {
    const Tree& T = a.vt[cs];
    const float4* items = a.surv[cs];
    uint32_t stack[kStack];
    int sp = 0;
    const int top = T.nlevels - 1;
    for (int64_t j = 0; j < T.count[top]; ++j) stack[sp++] = pack_node(top, j);
    while (sp > 0) {
      const uint32_t nd = stack[--sp];
      const int lev = node_level(nd);
      const int64_t idx = node_index(nd);
      if (lev == 0) {
        const int64_t b = idx * kLeaf, e = min(b + kLeaf, T.nitems);
        for (int64_t j = b; j < e; ++j) {
          const uint32_t g = __float_as_uint(items[j].w);
          double qx, qy, qz;
          surv_pos64(a, g, qx, qy, qz);
          const double d2 = ex_d2(x, y, z, qx, qy, qz);
          if (d2 < bd || (d2 == bd && g < gbest)) {
            bd = d2;
            gbest = g;
          }
        }
      } else {
        const int64_t cb = idx * kFan, ce = min(cb + kFan, T.count[lev - 1]);
        const int64_t off = T.offset[lev - 1];
        // survivor boxes hold the FP32 positions; the FP64 position of a
        // candidate is within eq of its FP32 one in each coordinate
        const double t = sqrt(bd) * (1.0 + 1e-12) + 2.0 * 1.7320508075688772 * double(eqs) + 1e-12;
        for (int64_t c = cb; c < ce; ++c) {
          const double d2 = box_d2_64(x, y, z, T.lo[off + c], T.hi[off + c]);
          if (d2 <= t * t) stack[sp++] = pack_node(lev - 1, c);
        }
      }
    }
  }
  const bool have_s = gbest != 0xffffffffu, have_u = idxA[co] != INT_MAX;
  const double ds = have_s ? __dsqrt_rn(bd) : INFINITY;
  const double ub = have_u ? bestA[co] : INFINITY;
  const double lb = -bestA[cs];
  double m;
  int code;
  int64_t arg;
  if (have_s && (!a.clamp_opp || ds <= ub)) {
    code = GFS_CODE_SURVIVOR;
    m = ds;
    arg = int64_t(gbest);
  } else if (a.clamp_opp && have_u) {
    code = GFS_CODE_OPPOSITE;
    m = ub;
    arg = idxA[co];
  } else {
    code = GFS_CODE_LOWER;
    m = lb;
    arg = idxA[cs];
  }
  if (m < 0.0) m = 0.0;
  int flags = code;
  if (m < __dsub_rn(lb, tol)) flags |= GFS_FLAG_LB_VIOL;
  if (m > __dadd_rn(bestF, tol)) flags |= GFS_FLAG_FAR_VIOL;
  if (have_u && ub < __dsub_rn(m, tol)) flags |= GFS_FLAG_OPP_VIOL;
  write_result(a, q, cs == 0 ? m : -m, arg, flags);
}

__global__ void __launch_bounds__(128) k_query_exact_all(QueryArgs a) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q < a.m) query_exact_one(a, q);
}

__global__ void __launch_bounds__(128) k_query_exact_deferred(QueryArgs a) {
  const unsigned int nd = min(a.cnt->ndefer, a.defer_cap);
  for (unsigned int t = blockIdx.x * blockDim.x + threadIdx.x; t < nd; t += gridDim.x * blockDim.x)
    query_exact_one(a, int64_t(a.defer[t]));
}

// ---------------------------------------------------------------------------
// backward: analytic derivative through the argmin
// ---------------------------------------------------------------------------
constexpr double kFix = 1099511627776.0;  // 2^40: fixed-point scale of the per-sample sums

__device__ __forceinline__ void fix_add(long long* dst, double v) {
  atomicAdd(reinterpret_cast<unsigned long long*>(dst), (unsigned long long)(long long)llrint(v * kFix));
}

__global__ void k_query_grad(GradArgs a) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= a.m) return;
  double x, y, z;
  if (a.x32) {
    x = a.x32[3 * q]; y = a.x32[3 * q + 1]; z = a.x32[3 * q + 2];
  } else {
    x = a.x64[3 * q]; y = a.x64[3 * q + 1]; z = a.x64[3 * q + 2];
  }
  const int code = a.flags[q] & 15;
  const double g = a.grad_s[q];
  const float sv = a.s[q];
  const double sigma = sv > 0.f ? 1.0 : (sv < 0.f ? -1.0 : 0.0);
  double gx = 0, gy = 0, gz = 0;
  if (code == GFS_CODE_SAMPLE) {
    if (a.acc_s) fix_add(a.acc_s + a.arg[q], g);
  } else if (sigma != 0.0 && (code == GFS_CODE_SURVIVOR || code == GFS_CODE_OPPOSITE || code == GFS_CODE_LOWER)) {
    if (code == GFS_CODE_SURVIVOR) {
      const uint32_t gid = uint32_t(a.arg[q]);
      const uint32_t i = gid / uint32_t(a.KS), k = gid % uint32_t(a.KS);
      const D4 pi = a.sph64[i];
      double qx, qy, qz, ux = 0, uy = 0, uz = 0;
      if (int(k) < a.K) {
        ux = a.U64[3 * k]; uy = a.U64[3 * k + 1]; uz = a.U64[3 * k + 2];
        ex_cand(pi, ux, uy, uz, qx, qy, qz);
      } else {
        qx = a.witness64[3 * i]; qy = a.witness64[3 * i + 1]; qz = a.witness64[3 * i + 2];
      }
      double vx = x - qx, vy = y - qy, vz = z - qz;
      const double d = sqrt(vx * vx + vy * vy + vz * vz);
      if (d > 0.0) {
        vx /= d; vy /= d; vz /= d;
        gx = g * sigma * vx; gy = g * sigma * vy; gz = g * sigma * vz;
        if (int(k) < a.K) {
          if (a.acc_p) {
            fix_add(a.acc_p + 3 * int64_t(i), -gx);
            fix_add(a.acc_p + 3 * int64_t(i) + 1, -gy);
            fix_add(a.acc_p + 3 * int64_t(i) + 2, -gz);
          }
          const double si = pi.w > 0 ? 1.0 : (pi.w < 0 ? -1.0 : 0.0);
          if (a.acc_s) fix_add(a.acc_s + i, -g * sigma * si * (vx * ux + vy * uy + vz * uz));
        }
      }
    } else {
      const int64_t j = a.arg[q];
      const D4 pj = a.sph64[j];
      double wx = x - pj.x, wy = y - pj.y, wz = z - pj.z;
      const double d = sqrt(wx * wx + wy * wy + wz * wz);
      if (d > 0.0) {
        wx /= d; wy /= d; wz /= d;
        const double dir = code == GFS_CODE_OPPOSITE ? 1.0 : -1.0;
        gx = g * sigma * dir * wx; gy = g * sigma * dir * wy; gz = g * sigma * dir * wz;
        if (a.acc_p) {
          fix_add(a.acc_p + 3 * j, -gx);
          fix_add(a.acc_p + 3 * j + 1, -gy);
          fix_add(a.acc_p + 3 * j + 2, -gz);
        }
        const double sj = pj.w > 0 ? 1.0 : (pj.w < 0 ? -1.0 : 0.0);
        if (a.acc_s) fix_add(a.acc_s + j, -g * sigma * dir * sj);
      }
    }
  }
  if (a.grad_x) {
    a.grad_x[3 * q] = float(gx);
    a.grad_x[3 * q + 1] = float(gy);
    a.grad_x[3 * q + 2] = float(gz);
  }
}

__global__ void k_fix_to_float(const long long* __restrict__ acc, int64_t n, float* __restrict__ out) {
  int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n) out[i] = float(double(acc[i]) / kFix);
}

// survivors: ids of both class lists (zero-class entries only from list 0)
__global__ void k_collect_ids(const float4* __restrict__ s0, unsigned int n0, const float4* __restrict__ s1,
                              unsigned int n1, const D4* __restrict__ sph64, int KS, uint32_t* __restrict__ out,
                              unsigned int* __restrict__ count) {
  unsigned int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n0) {
    out[atomicAdd(count, 1u)] = __float_as_uint(s0[t].w);
  } else if (t < n0 + n1) {
    uint32_t g = __float_as_uint(s1[t - n0].w);
    if (sph64[g / uint32_t(KS)].w != 0.0) out[atomicAdd(count, 1u)] = g;
  }
}

__global__ void k_widen_ids(const uint32_t* __restrict__ in, int64_t n, int64_t* __restrict__ out) {
  int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n) out[i] = int64_t(in[i]);
}

// ---------------------------------------------------------------------------
// host-side launch helpers
// ---------------------------------------------------------------------------
static inline unsigned int nblk(int64_t n, int b) { return (unsigned int)((n + b - 1) / b); }

// kernels this library launched (own kernels; sorts counted as calls)
static unsigned long long g_launches = 0, g_sort_calls = 0;
void launch_counts(unsigned long long* own, unsigned long long* sorts) {
  *own = g_launches;
  *sorts = g_sort_calls;
}

cudaError_t launch_copy_inputs(const double* p, const double* s, int64_t n, D4* sph64, cudaStream_t st) {
  unsigned int g = nblk(n, 256);
  if (g > 4096) g = 4096;
  k_copy_inputs<<<g, 256, 0, st>>>(p, s, n, sph64);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t launch_keys_d4(const D4* sph64, int64_t n, uint32_t* keys, int* vals, unsigned int* bound_bits,
                           BuildConsts* bc, cudaStream_t st) {
  unsigned int g = nblk(n, 256);
  if (g > 4096) g = 4096;
  k_keys_d4<<<g, 256, 0, st>>>(sph64, n, keys, vals, bound_bits);
  ++g_launches;
  k_consts<<<1, 1, 0, st>>>(bound_bits, bc);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t sort_pairs(void* temp, size_t& temp_bytes, const uint32_t* kin, uint32_t* kout, const int* vin,
                       int* vout, int64_t n, cudaStream_t st) {
  if (temp) ++g_sort_calls;
  return cub::DeviceRadixSort::SortPairs(temp, temp_bytes, kin, kout, vin, vout, n, 0, 30, st);
}

cudaError_t sort_keys_u32(void* temp, size_t& temp_bytes, const uint32_t* kin, uint32_t* kout, int64_t n,
                          cudaStream_t st) {
  if (temp) ++g_sort_calls;
  return cub::DeviceRadixSort::SortKeys(temp, temp_bytes, kin, kout, n, 0, 32, st);
}

cudaError_t launch_gather_spheres(const D4* sph64, const int* order, int64_t n, const BuildConsts* bc, float tol32,
                                  double tol, float4* sph, float4* thr, int* sid, cudaStream_t st) {
  k_gather_spheres<<<nblk(n, 256), 256, 0, st>>>(sph64, order, n, bc, tol32, tol, sph, thr, sid);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t launch_build_tree(const float4* items, int is_sphere, float A, Tree& T, unsigned* scratch,
                              cudaStream_t st) {
  if (T.nlevels == 0) return cudaSuccess;
  if (is_sphere) {
    k_sphere_leaves<<<nblk(T.count[0], 128), 128, 0, st>>>(items, T.nitems, A, T.lo, T.hi, T.na, T.nb, T.nf,
                                                           T.count[0]);
    ++g_launches;
    for (int l = 1; l < T.nlevels; ++l) {
      k_sphere_level<<<nblk(T.count[l], 128), 128, 0, st>>>(T.lo, T.hi, T.na, T.nb, T.nf, A, T.offset[l - 1],
                                                            T.count[l - 1], T.offset[l], T.count[l]);
      ++g_launches;
    }
    if (scratch && T.nlevels > 1) {
      const int64_t nupper = T.offset[T.nlevels - 1] + T.count[T.nlevels - 1] - T.offset[1];
      const cudaError_t e = cudaMemsetAsync(scratch, 0, size_t(nupper) * 4 * sizeof(unsigned), st);
      if (e != cudaSuccess) return e;
      k_tighten_items<<<nblk(T.nitems, 256), 256, 0, st>>>(items, T, scratch);
      k_tighten_nodes<<<nblk(nupper, 128), 128, 0, st>>>(T, scratch, A, nupper);
      g_launches += 2;
    }
  } else {
    k_leaves<<<nblk(T.count[0], 128), 128, 0, st>>>(items, T.nitems, T.lo, T.hi, T.count[0]);
    ++g_launches;
    for (int l = 1; l < T.nlevels; ++l) {
      k_level<<<nblk(T.count[l], 128), 128, 0, st>>>(T.lo, T.hi, T.offset[l - 1], T.count[l - 1], T.offset[l],
                                                     T.count[l]);
      ++g_launches;
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_query_keys(const double* x64, const float* x32, int64_t m, uint32_t* keys, int* vals,
                              cudaStream_t st) {
  if (m == 0) return cudaSuccess;
  k_query_keys<<<nblk(m, 256), 256, 0, st>>>(x64, x32, m, keys, vals);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t launch_point_keys(const float4* items, int64_t n, uint32_t* keys, int* vals, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_point_keys<<<nblk(n, 256), 256, 0, st>>>(items, n, keys, vals);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t launch_gather_points(const float4* src, const int* order, int64_t n, float4* dst, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_gather_points<<<nblk(n, 256), 256, 0, st>>>(src, order, n, dst);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t launch_cull(const CullArgs& a, cudaStream_t st) {
  dim3 grid(nblk(a.n, kCullBlock), unsigned(a.K));
  k_cull<<<grid, kCullBlock, 0, st>>>(a);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t launch_query_spheres(const QueryArgs& a, cudaStream_t st) {
  if (a.m == 0) return cudaSuccess;
  k_query_spheres<<<nblk(a.m, 128), 128, 0, st>>>(a);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t launch_query_finish(const QueryArgs& a, cudaStream_t st) {
  if (a.m == 0) return cudaSuccess;
  k_query_finish<<<nblk(a.m, 128), 128, 0, st>>>(a);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t launch_query_exact(const QueryArgs& a, int all, cudaStream_t st) {
  if (a.m == 0) return cudaSuccess;
  if (all) {
    k_query_exact_all<<<nblk(a.m, 128), 128, 0, st>>>(a);
    ++g_launches;
  } else {
    unsigned int g = nblk(a.m, 128);
    if (g > 152u * 16u) g = 152u * 16u;
    k_query_exact_deferred<<<g, 128, 0, st>>>(a);
    ++g_launches;
  }
  return cudaGetLastError();
}

cudaError_t launch_grad(const GradArgs& a, int64_t n, float* grad_p, float* grad_sv, cudaStream_t st) {
  if (a.m > 0) k_query_grad<<<nblk(a.m, 128), 128, 0, st>>>(a);
  if (grad_p) k_fix_to_float<<<nblk(3 * n, 256), 256, 0, st>>>(a.acc_p, 3 * n, grad_p);
  if (grad_sv) k_fix_to_float<<<nblk(n, 256), 256, 0, st>>>(a.acc_s, n, grad_sv);
  return cudaGetLastError();
}

cudaError_t launch_collect_ids(const float4* s0, unsigned int n0, const float4* s1, unsigned int n1, const D4* sph64,
                               int KS, uint32_t* out, unsigned int* count, cudaStream_t st) {
  if (n0 + n1 == 0) return cudaSuccess;
  k_collect_ids<<<nblk(int64_t(n0) + n1, 256), 256, 0, st>>>(s0, n0, s1, n1, sph64, KS, out, count);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t launch_widen_ids(const uint32_t* in, int64_t n, int64_t* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_widen_ids<<<nblk(n, 256), 256, 0, st>>>(in, n, out);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace gfs

#include "gfs_batch.cuh"
