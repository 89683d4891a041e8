// Device kernels of the consistent-SDF hot path.
//
//   P build   k_cull          -- candidate generation and coverage culling
//                                (Def. 1 discretised, Prop. 1 (ii))
//   query     k_query_fast    -- FP32 evaluation with certified decisions
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

// Derive the launch-wide error bounds from the data bounds (one thread).
__global__ void k_consts(const unsigned int* __restrict__ bound_bits, BuildConsts* __restrict__ bc) {
  float A = fmaxf(1.0f, __uint_as_float(bound_bits[0]));
  float R = __uint_as_float(bound_bits[1]);
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
  *bc = c;
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
__global__ void k_leaves(const float4* __restrict__ items, int64_t nitems, float4* __restrict__ lo,
                         float4* __restrict__ hi, int64_t nleaves) {
  int64_t L = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (L >= nleaves) return;
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

__global__ void k_level(float4* __restrict__ lo, float4* __restrict__ hi, int64_t child_off, int64_t nchild,
                        int64_t off, int64_t nnode) {
  int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (j >= nnode) return;
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
  v = v + (fabsf(v) + A) * 4.8e-7f;
  return make_float4(bx, by, bz, v);
}

__global__ void k_sphere_leaves(const float4* __restrict__ items, int64_t nitems, float A, float4* __restrict__ lo,
                                float4* __restrict__ hi, float4* __restrict__ bp, float4* __restrict__ bn,
                                float4* __restrict__ bf, int64_t nleaves) {
  int64_t L = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (L >= nleaves) return;
  int64_t b = L * kLeaf, e = min(b + kLeaf, nitems);
  float4 P[kLeaf], N[kLeaf], F[kLeaf];
  int np = 0, nn = 0, nf = 0;
  float3 mn = make_float3(INFINITY, INFINITY, INFINITY), mx = make_float3(-INFINITY, -INFINITY, -INFINITY);
  for (int64_t i = b; i < e; ++i) {
    const float4 v = items[i];
    mn.x = fminf(mn.x, v.x); mn.y = fminf(mn.y, v.y); mn.z = fminf(mn.z, v.z);
    mx.x = fmaxf(mx.x, v.x); mx.y = fmaxf(mx.y, v.y); mx.z = fmaxf(mx.z, v.z);
    const float r = fabsf(v.w);
    if (v.w > 0.f) P[np++] = make_float4(v.x, v.y, v.z, r);
    if (v.w < 0.f) N[nn++] = make_float4(v.x, v.y, v.z, r);
    F[nf++] = make_float4(v.x, v.y, v.z, -r);
  }
  lo[L] = make_float4(nextafterf(mn.x, -INFINITY), nextafterf(mn.y, -INFINITY), nextafterf(mn.z, -INFINITY), 0.f);
  hi[L] = make_float4(nextafterf(mx.x, INFINITY), nextafterf(mx.y, INFINITY), nextafterf(mx.z, INFINITY), 0.f);
  bp[L] = bound_ball(P, np, A);
  bn[L] = bound_ball(N, nn, A);
  bf[L] = bound_ball(F, nf, A);
}

__global__ void k_sphere_level(float4* __restrict__ lo, float4* __restrict__ hi, float4* __restrict__ bp,
                               float4* __restrict__ bn, float4* __restrict__ bf, float A, int64_t child_off,
                               int64_t nchild, int64_t off, int64_t nnode) {
  int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (j >= nnode) return;
  int64_t b = j * kFan, e = min(b + kFan, nchild);
  float4 L = make_float4(INFINITY, INFINITY, INFINITY, 0.f), H = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
  float4 P[kFan], N[kFan], F[kFan];
  int np = 0, nn = 0, nf = 0;
  for (int64_t c = b; c < e; ++c) {
    const float4 a = lo[child_off + c], z = hi[child_off + c];
    L.x = fminf(L.x, a.x); L.y = fminf(L.y, a.y); L.z = fminf(L.z, a.z);
    H.x = fmaxf(H.x, z.x); H.y = fmaxf(H.y, z.y); H.z = fmaxf(H.z, z.z);
    const float4 u = bp[child_off + c], v = bn[child_off + c], w = bf[child_off + c];
    if (u.w > -INFINITY) P[np++] = u;
    if (v.w > -INFINITY) N[nn++] = v;
    if (w.w > -INFINITY) F[nf++] = w;
  }
  lo[off + j] = L;
  hi[off + j] = H;
  bp[off + j] = bound_ball(P, np, A);
  bn[off + j] = bound_ball(N, nn, A);
  bf[off + j] = bound_ball(F, nf, A);
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
// P build: coverage culling of the candidates q_ik = p_i + |s_i| u_k
// ---------------------------------------------------------------------------
// One thread per candidate; a warp holds 32 Morton-consecutive spheres with
// the same direction k, so its candidates are spatial neighbours and walk
// similar parts of the hierarchy.  The walk visits the child with the
// largest covering margin first and stops at the first covering ball.
__global__ void __launch_bounds__(128) k_cull(CullArgs a) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int k = blockIdx.y;
  if (i >= a.n) return;
  const BuildConsts bc = *a.bc;
  const float4 S = a.sph[i];
  const float r = fabsf(S.w);
  const float ux = a.U32[3 * k], uy = a.U32[3 * k + 1], uz = a.U32[3 * k + 2];
  const float qx = fmaf(r, ux, S.x), qy = fmaf(r, uy, S.y), qz = fmaf(r, uz, S.z);
  bool have64 = false;
  double qx64 = 0, qy64 = 0, qz64 = 0;
  unsigned long long rechecks = 0;
  auto load64 = [&]() {
    if (!have64) {
      D4 pi = a.sph64[a.sid[i]];
      ex_cand(pi, a.U64[3 * k], a.U64[3 * k + 1], a.U64[3 * k + 2], qx64, qy64, qz64);
      have64 = true;
    }
  };
  if (a.box_cull) {
    float mq = fmaxf(fabsf(qx), fmaxf(fabsf(qy), fabsf(qz)));
    float eb = 2.f * bc.eq;
    if (mq > 1.f + eb) return;
    if (mq >= 1.f - eb) {
      load64();
      ++rechecks;
      if (!ex_inbox(qx64, qy64, qz64)) {
        atomicAdd(&a.cnt->cull_rechecks, rechecks);
        return;
      }
    }
  }
  const Tree& T = a.tree;
  uint32_t stack[kStack];
  int sp = 0;
  const int top = T.nlevels - 1;
  for (int64_t j = 0; j < T.count[top]; ++j) stack[sp++] = pack_node(top, j);
  bool covered = false;
  const float grow = 1.f + 8.f * kU;
  while (sp > 0 && !covered) {
    const uint32_t nd = stack[--sp];
    const int lev = node_level(nd);
    const int64_t idx = node_index(nd);
    if (lev == 0) {
      const int64_t b = idx * kLeaf, e = min(b + kLeaf, a.n);
      for (int64_t j = b; j < e; ++j) {
        if (j == i) continue;
        const float4 P = a.sph[j];
        const float dx = qx - P.x, dy = qy - P.y, dz = qz - P.z;
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float4 Th = a.thr[j];
        if (d2 < Th.x) { covered = true; break; }
        if (d2 <= Th.y) {
          load64();
          ++rechecks;
          if (ex_cov(qx64, qy64, qz64, a.sph64[a.sid[j]], a.tol)) { covered = true; break; }
        }
      }
    } else {
      const int64_t cb = idx * kFan, ce = min(cb + kFan, T.count[lev - 1]);
      const int64_t off = T.offset[lev - 1];
      int best = -1;
      float bestm = -INFINITY;
      uint32_t pend[kFan];
      int np = 0;
      for (int64_t c = cb; c < ce; ++c) {
        // the node can hold a covering ball only if q lies in one of its
        // bounding balls shrunk by tol
        float margin = -INFINITY;
        const float4 Bs[2] = {T.bp[off + c], T.bn[off + c]};
        for (int cl = 0; cl < 2; ++cl) {
          const float t = fmaf(Bs[cl].w - a.tol32, grow, bc.pad);
          if (!(t > 0.f)) continue;
          const float dx = qx - Bs[cl].x, dy = qy - Bs[cl].y, dz = qz - Bs[cl].z;
          const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          if (d2 < t * t) margin = fmaxf(margin, t * t - d2);
        }
        if (margin > -INFINITY) {
          if (margin > bestm) {
            if (best >= 0) pend[np++] = pack_node(lev - 1, best);
            best = int(c);
            bestm = margin;
          } else {
            pend[np++] = pack_node(lev - 1, c);
          }
        }
      }
      for (int q = 0; q < np; ++q) stack[sp++] = pend[q];
      if (best >= 0) stack[sp++] = pack_node(lev - 1, best);
    }
  }
  if (rechecks) atomicAdd(&a.cnt->cull_rechecks, rechecks);
  if (covered) return;
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
    if (base < a.cap) a.surv[c][base] = item;
  }
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
__device__ __forceinline__ void warp_count(unsigned long long* dst, unsigned long long v) {
  const unsigned mask = __activemask();
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  if ((threadIdx.x & 31) == __ffs(mask) - 1 && v) atomicAdd(dst, v);
}

// FP64 band pass over the sphere hierarchy.  Finds, among the spheres whose
// FP32 value lies at or below thr, the exact FP64 minimum and its input index
// (ties to the lowest index).  mode 0: value |x-p| - r over sign class c;
// mode 1: value |x-p| + r over all spheres.  The FP32 threshold is chosen so
// that the exact minimiser always lies in the band.
__device__ double band_sphere(const QueryArgs& a, const BuildConsts& bc, double x64, double y64, double z64, float x,
                              float y, float z, int mode, int c, float thr, int& arg) {
  const Tree& T = a.st;
  const float grow = 1.f + 8.f * 5.9604644775390625e-8f;
  double best = INFINITY;
  arg = INT_MAX;
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
        const float4 P = a.sph[j];
        if (mode == 0 && (P.w == 0.f || int(P.w < 0.f) != c)) continue;
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
      for (int64_t cc = cb; cc < ce; ++cc) {
        const float4 B = mode == 1 ? T.bf[off + cc] : (c == 0 ? T.bp[off + cc] : T.bn[off + cc]);
        if (!(B.w > -INFINITY)) continue;
        const float t = fmaf(thr + B.w, grow, bc.eprune);
        if (t > 0.f && ball_d2(x, y, z, B) < t * t) stack[sp++] = pack_node(lev - 1, cc);
      }
    }
  }
  return best;
}

// FP64 band pass over a survivor hierarchy: exact nearest survivor among
// those whose FP32 distance^2 is at most thr (ties to the lowest id).
__device__ double band_surv(const QueryArgs& a, const BuildConsts& bc, int cls, double x64, double y64, double z64,
                            float x, float y, float z, float thr, uint32_t& gbest) {
  const Tree& T = a.vt[cls];
  const float4* items = a.surv[cls];
  const float grow = 1.f + 8.f * 5.9604644775390625e-8f;
  const float thn = thr * grow + bc.ed_lin * __fsqrt_rn(thr) + 1e-30f;
  double best = INFINITY;
  gbest = 0xffffffffu;
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
        const float4 P = items[j];
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
      for (int64_t cc = cb; cc < ce; ++cc)
        if (box_d2(x, y, z, T.lo[off + cc], T.hi[off + cc]) < thn) stack[sp++] = pack_node(lev - 1, cc);
    }
  }
  return best;
}

__global__ void __launch_bounds__(128) k_query_fast(QueryArgs a) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= a.m) return;
  const BuildConsts bc = *a.bc;
  double x64, y64, z64;
  load_query(a, q, x64, y64, z64);
  const float x = float(x64), y = float(y64), z = float(z64);
  unsigned long long rechecks = 0, n_nodes = 0, n_items = 0, n_snodes = 0, n_sitems = 0, n_band = 0;
  bool defer = !(fabs(x64) <= bc.A && fabs(y64) <= bc.A && fabs(z64) <= bc.A);
  const float grow = 1.f + 8.f * kU;
  const float ea2 = 2.f * bc.ea;
  const float negtol = -a.tol32 + ea2;
  // ---- pass over the spheres -------------------------------------------
  bool cov[2] = {false, false};
  Top2 A[2], F;
  top2_init(A[0]);
  top2_init(A[1]);
  top2_init(F);
  int sample = INT_MAX;
  if (!defer) {
    const Tree& T = a.st;
    uint32_t stack[kStack];
    int sp = 0;
    const int top = T.nlevels - 1;
    for (int64_t j = 0; j < T.count[top]; ++j) stack[sp++] = pack_node(top, j);
    while (sp > 0) {
      const uint32_t nd = stack[--sp];
      const int lev = node_level(nd);
      const int64_t idx = node_index(nd);
      ++n_nodes;
      if (lev == 0) {
        const int64_t b = idx * kLeaf, e = min(b + kLeaf, a.n);
        n_items += uint64_t(e - b);
        for (int64_t j = b; j < e; ++j) {
          const float4 P = a.sph[j];
          const float dx = x - P.x, dy = y - P.y, dz = z - P.z;
          const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          if (d2 == 0.f) {
            const int o = a.sid[j];
            const D4 pj = a.sph64[o];
            if (pj.x == x64 && pj.y == y64 && pj.z == z64 && o < sample) sample = o;
          }
          const float r = fabsf(P.w);
          if (P.w != 0.f) {
            const int c = P.w < 0.f;
            if (!cov[c]) {
              const float4 Th = a.thr[j];
              if (d2 < Th.z) {
                cov[c] = true;
              } else if (d2 <= Th.w) {
                ++rechecks;
                cov[c] = ex_cov(x64, y64, z64, a.sph64[a.sid[j]], a.tol);
              }
            }
            const float t = r + top2_th(A[c], ea2);
            if (t > 0.f && d2 < t * t * grow) top2_push(A[c], __fsqrt_rn(d2) - r, int(j));
          }
          const float t2 = top2_th(F, ea2) - r;
          if (t2 > 0.f && d2 < t2 * t2 * grow) top2_push(F, __fsqrt_rn(d2) + r, int(j));
        }
      } else {
        const int64_t cb = idx * kFan, ce = min(cb + kFan, T.count[lev - 1]);
        const int64_t off = T.offset[lev - 1];
        float th0 = top2_th(A[0], ea2), th1 = top2_th(A[1], ea2);
        if (!cov[0]) th0 = fmaxf(th0, negtol);
        if (!cov[1]) th1 = fmaxf(th1, negtol);
        const float thf = top2_th(F, ea2);
        int best = -1;
        float bestd = INFINITY;
        uint32_t pend[kFan];
        int np = 0;
        for (int64_t c = cb; c < ce; ++c) {
          const float4 L = T.lo[off + c], H = T.hi[off + c];
          const float d2 = box_d2(x, y, z, L, H);
          bool need = inside_box(x, y, z, L, H);
          if (!need) {
            const float4 B = T.bp[off + c];
            const float t = fmaf(th0 + B.w, grow, bc.eprune);
            need = t > 0.f && ball_d2(x, y, z, B) < t * t;
          }
          if (!need) {
            const float4 B = T.bn[off + c];
            const float t = fmaf(th1 + B.w, grow, bc.eprune);
            need = t > 0.f && ball_d2(x, y, z, B) < t * t;
          }
          if (!need) {
            const float4 B = T.bf[off + c];
            const float t = fmaf(thf + B.w, grow, bc.eprune);
            need = t > 0.f && ball_d2(x, y, z, B) < t * t;
          }
          if (!need) continue;
          if (d2 < bestd) {
            if (best >= 0) pend[np++] = pack_node(lev - 1, best);
            best = int(c);
            bestd = d2;
          } else {
            pend[np++] = pack_node(lev - 1, c);
          }
        }
        for (int t = 0; t < np; ++t) stack[sp++] = pend[t];
        if (best >= 0) stack[sp++] = pack_node(lev - 1, best);
      }
    }
  }
  int code = -1;
  double value = 0.0;
  int64_t arg = -1;
  int flags = 0;
  if (!defer) {
    if (sample != INT_MAX) {
      code = GFS_CODE_SAMPLE;
      value = a.sph64[sample].w;
      arg = sample;
    } else if (cov[0] && cov[1]) {
      code = GFS_CODE_INVALID;
      value = __longlong_as_double(0x7ff8000000000000LL);
    } else if (!cov[0] && !cov[1]) {
      code = GFS_CODE_OUTSIDE;
    }
    if (code >= 0) flags = code;
  }
  if (!defer && code < 0) {
    const int cs = cov[0] ? 0 : 1, co = 1 - cs;
    // ---- pass over the survivors of x's sign -----------------------------
    float bd = INFINITY, sd = INFINITY;
    uint32_t gbest = 0xffffffffu;
    auto band = [&](float D) { return bc.ed_lin * __fsqrt_rn(D) + bc.ed_quad * D + 1e-30f; };
    if (a.vt[cs].nlevels > 0) {
      const Tree& T = a.vt[cs];
      const float4* items = a.surv[cs];
      float th = INFINITY, thn = INFINITY;  // threshold on d^2, and widened for nodes
      uint32_t stack[kStack];
      int sp = 0;
      const int top = T.nlevels - 1;
      for (int64_t j = 0; j < T.count[top]; ++j) stack[sp++] = pack_node(top, j);
      while (sp > 0) {
        const uint32_t nd = stack[--sp];
        const int lev = node_level(nd);
        const int64_t idx = node_index(nd);
        ++n_snodes;
        if (lev == 0) {
          const int64_t b = idx * kLeaf, e = min(b + kLeaf, T.nitems);
          n_sitems += uint64_t(e - b);
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
        } else {
          const int64_t cb = idx * kFan, ce = min(cb + kFan, T.count[lev - 1]);
          const int64_t off = T.offset[lev - 1];
          int best = -1;
          float bestd = INFINITY;
          uint32_t pend[kFan];
          int np = 0;
          for (int64_t c = cb; c < ce; ++c) {
            const float d2 = box_d2(x, y, z, T.lo[off + c], T.hi[off + c]);
            if (!(d2 < thn)) continue;
            if (d2 < bestd) {
              if (best >= 0) pend[np++] = pack_node(lev - 1, best);
              best = int(c);
              bestd = d2;
            } else {
              pend[np++] = pack_node(lev - 1, c);
            }
          }
          for (int t = 0; t < np; ++t) stack[sp++] = pend[t];
          if (best >= 0) stack[sp++] = pack_node(lev - 1, best);
        }
      }
    }
    const bool have_s = gbest != 0xffffffffu, have_u = A[co].idx >= 0;
    // exact nearest survivor: direct when no other survivor lies in the
    // error band, else an FP64 pass over the band
    double ds = INFINITY;
    if (have_s) {
      if (sd >= bd + 2.f * band(bd)) {
        double qx, qy, qz;
        surv_pos64(a, gbest, qx, qy, qz);
        ds = __dsqrt_rn(ex_d2(x64, y64, z64, qx, qy, qz));
      } else {
        ++n_band;
        ds = __dsqrt_rn(band_surv(a, bc, cs, x64, y64, z64, x, y, z, bd + 2.f * band(bd), gbest));
      }
    }
    // exact nearest opposite tangent point
    double ub = INFINITY;
    int uj = -1;
    if (have_u) {
      if (A[co].sec >= A[co].best + ea2) {
        uj = a.sid[A[co].idx];
        const D4 pj = a.sph64[uj];
        ub = __dsub_rn(__dsqrt_rn(ex_d2(x64, y64, z64, pj.x, pj.y, pj.z)), fabs(pj.w));
      } else {
        ++n_band;
        ub = band_sphere(a, bc, x64, y64, z64, x, y, z, 0, co, A[co].best + ea2, uj);
      }
    }
    // exact lower bound LB (max over x's class of r - |x-p|) on demand
    double lb = 0.0;
    int lj = -1;
    bool have_lb = false;
    auto exact_lb = [&]() {
      if (have_lb) return;
      have_lb = true;
      if (A[cs].sec >= A[cs].best + ea2) {
        lj = a.sid[A[cs].idx];
        const D4 pl = a.sph64[lj];
        lb = __dsub_rn(fabs(pl.w), __dsqrt_rn(ex_d2(x64, y64, z64, pl.x, pl.y, pl.z)));
      } else {
        ++n_band;
        lb = -band_sphere(a, bc, x64, y64, z64, x, y, z, 0, cs, A[cs].best + ea2, lj);
      }
    };
    double m;
    if (have_s && (!a.clamp_opp || ds <= ub)) {
      code = GFS_CODE_SURVIVOR;
      m = ds;
      arg = int64_t(gbest);
    } else if (a.clamp_opp && have_u) {
      code = GFS_CODE_OPPOSITE;
      m = ub;
      arg = uj;
    } else {
      exact_lb();
      code = GFS_CODE_LOWER;
      m = lb;
      arg = lj;
    }
    if (m < 0.0) m = 0.0;
    flags = code;
    const double E = double(bc.ea) * 1.01 + 1e-15;
    // LB_VIOL: m < LB - tol
    const double lbt = -double(A[cs].best) - a.tol;
    if (m < lbt - E) {
      flags |= GFS_FLAG_LB_VIOL;
    } else if (!(m > lbt + E)) {
      exact_lb();
      if (m < __dsub_rn(lb, a.tol)) flags |= GFS_FLAG_LB_VIOL;
    }
    // FAR_VIOL: m > FAR + tol
    const double ft = double(F.best) + a.tol;
    if (m > ft + E) {
      flags |= GFS_FLAG_FAR_VIOL;
    } else if (!(m < ft - E)) {
      double far;
      if (F.sec >= F.best + ea2) {
        const D4 pf = a.sph64[a.sid[F.idx]];
        far = __dadd_rn(__dsqrt_rn(ex_d2(x64, y64, z64, pf.x, pf.y, pf.z)), fabs(pf.w));
      } else {
        ++n_band;
        int fj;
        far = band_sphere(a, bc, x64, y64, z64, x, y, z, 1, 0, F.best + ea2, fj);
      }
      if (m > __dadd_rn(far, a.tol)) flags |= GFS_FLAG_FAR_VIOL;
    }
    if (have_u && ub < __dsub_rn(m, a.tol)) flags |= GFS_FLAG_OPP_VIOL;
    value = cs == 0 ? m : -m;
  }
  warp_count(&a.cnt->query_rechecks, rechecks);
  warp_count(&a.cnt->q_sphere_nodes, n_nodes);
  warp_count(&a.cnt->q_sphere_items, n_items);
  warp_count(&a.cnt->q_surv_nodes, n_snodes);
  warp_count(&a.cnt->q_band_passes, n_band);
  warp_count(&a.cnt->q_surv_items, n_sitems);
  if (!defer) {
    write_result(a, q, value, arg, flags);
    return;
  }
  // outside the coordinate range the error bounds assume: FP64 path
  const unsigned int slot = atomicAdd(&a.cnt->ndefer, 1u);
  if (slot < a.defer_cap) a.defer[slot] = uint32_t(q);
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
          const float4 Bs[2] = {T.bp[off + c], T.bn[off + c]};
          for (int cl = 0; cl < 2 && !need; ++cl) {
            if (!(Bs[cl].w > -INFINITY)) continue;
            double th = bestA[cl];
            if (!cov[cl]) th = fmax(th, -tol);
            const double t = (th + double(Bs[cl].w)) * (1.0 + 1e-12) + 1e-12;
            need = t > 0.0 && ball_d2_64(x, y, z, Bs[cl]) <= t * t;
          }
          if (!need) {
            const float4 B = T.bf[off + c];
            const double t = (bestF + double(B.w)) * (1.0 + 1e-12) + 1e-12;
            need = t > 0.0 && ball_d2_64(x, y, z, B) <= t * t;
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

cudaError_t launch_build_tree(const float4* items, int is_sphere, float A, Tree& T, cudaStream_t st) {
  if (T.nlevels == 0) return cudaSuccess;
  if (is_sphere) {
    k_sphere_leaves<<<nblk(T.count[0], 128), 128, 0, st>>>(items, T.nitems, A, T.lo, T.hi, T.bp, T.bn, T.bf,
                                                           T.count[0]);
    ++g_launches;
    for (int l = 1; l < T.nlevels; ++l) {
      k_sphere_level<<<nblk(T.count[l], 128), 128, 0, st>>>(T.lo, T.hi, T.bp, T.bn, T.bf, A, T.offset[l - 1],
                                                            T.count[l - 1], T.offset[l], T.count[l]);
      ++g_launches;
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
  dim3 grid(nblk(a.n, 128), unsigned(a.K));
  k_cull<<<grid, 128, 0, st>>>(a);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t launch_query_fast(const QueryArgs& a, cudaStream_t st) {
  if (a.m == 0) return cudaSuccess;
  k_query_fast<<<nblk(a.m, 128), 128, 0, st>>>(a);
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
