// Same-sign tangent augmentation, one warp per point (device code only).
//
// The steps and every FP64 expression are those of tangent_one in
// gfs_tangent.cuh (the host build checks that routine against the oracle);
// here the 32 lanes of a warp walk the sphere hierarchy for one point
// together: each round they take up to 32 nodes off a shared stack
// (warp_walk_until), every lane screens and evaluates its own nodes and
// leaves, and between rounds the lanes merge what they found.  The results
// are minima with fixed tie rules (the class distance with the lowest
// index, the far bound, the tangent point with the lowest id) and a
// containment OR, so they do not depend on which lane found what or in
// which round; the thresholds a round prunes with are the merged results
// of the rounds before it, which only ever prunes what cannot change them.
#pragma once

#include "gfs_tangent.cuh"
#include "gfs_warp.cuh"

namespace gfs {
namespace tangent {

constexpr unsigned kLanes = 0xffffffffu;
constexpr int kWarpStack = 512;  // per-warp walk stack entries (plus a reserve of kFan)

// lexicographic minimum of (v, i) over the warp, on every lane
__device__ __forceinline__ void warp_min_vi(double& v, int& i) {
  for (int o = 16; o > 0; o >>= 1) {
    const double v2 = __shfl_xor_sync(kLanes, v, o);
    const int i2 = __shfl_xor_sync(kLanes, i, o);
    if (v2 < v || (v2 == v && i2 < i)) {
      v = v2;
      i = i2;
    }
  }
}

__device__ __forceinline__ void warp_min_vl(double& v, int64_t& i) {
  for (int o = 16; o > 0; o >>= 1) {
    const double v2 = __shfl_xor_sync(kLanes, v, o);
    const long long i2 = __shfl_xor_sync(kLanes, (long long)i, o);
    // id -1 (nothing found) sorts last
    const bool better = v2 < v || (v2 == v && i2 >= 0 && (i < 0 || i2 < i));
    if (better) {
      v = v2;
      i = i2;
    }
  }
}

// sphere_bounds over the warp; every lane receives the result.  stk: the
// warp's stack (kWarpStack + kFan entries).
__device__ inline void warp_sphere_bounds(const QueryArgs& a, double x, double y, double z, uint32_t* stk, int lane,
                                          SphereBounds& R) {
  const double tol = a.tol;
  R.cov[0] = R.cov[1] = false;
  R.bestA[0] = R.bestA[1] = INFINITY;
  R.idxA[0] = R.idxA[1] = INT_MAX;
  R.bestF = INFINITY;
  const float x32 = float(x), y32 = float(y), z32 = float(z), ax = amax3(x32, y32, z32);
  float thF = INFINITY, thA[2] = {INFINITY, INFINITY};
  const Tree& T = a.st;
  if (T.nlevels == 0) return;
  auto item = [&](int64_t j) {
    const float4 S = a.sph[j];
    const float d32 = dist32(x32, y32, z32, S), r32 = fabsf(S.w);
    const float er = err32(ax, S, d32, r32);
    bool need = d32 + r32 - er <= thF;
    if (S.w != 0.f) need = need || d32 - r32 - er <= thA[S.w < 0.f];
    if (!need) return;
    const int o = a.sid[j];
    const D4 P = a.sph64[o];
    const double d2 = ex_d2(x, y, z, P.x, P.y, P.z);
    const double dl = __dsqrt_rn(d2);
    const double r = fabs(P.w);
    if (P.w != 0.0) {
      const int c = P.w < 0.0;
      if (!R.cov[c] && r > tol) {
        const double rt = __dsub_rn(r, tol);
        if (d2 < __dmul_rn(rt, rt)) R.cov[c] = true;
      }
      const double av = __dsub_rn(dl, r);
      if (av < R.bestA[c] || (av == R.bestA[c] && o < R.idxA[c])) {
        R.bestA[c] = av;
        R.idxA[c] = o;
      }
      // this lane's thresholds tighten at once, the warp's at the next merge
      thA[c] = fminf(thA[c], f_up(R.cov[c] ? R.bestA[c] : fmax(R.bestA[c], -tol)));
    }
    const double f = __dadd_rn(dl, r);
    if (f < R.bestF) {
      R.bestF = f;
      thF = fminf(thF, f_up(f));
    }
  };
  auto merge = [&]() {
    R.cov[0] = __any_sync(kLanes, R.cov[0]);
    R.cov[1] = __any_sync(kLanes, R.cov[1]);
    warp_min_vi(R.bestA[0], R.idxA[0]);
    warp_min_vi(R.bestA[1], R.idxA[1]);
    for (int o = 16; o > 0; o >>= 1) R.bestF = fmin(R.bestF, __shfl_xor_sync(kLanes, R.bestF, o));
    // FP32 copies (rounded up) of the thresholds a sphere must reach to
    // matter (per class at least -tol while the class has no containing ball)
    thF = f_up(R.bestF);
    for (int c = 0; c < 2; ++c) thA[c] = f_up(R.cov[c] ? R.bestA[c] : fmax(R.bestA[c], -tol));
  };
  // seed: the leaf whose balls reach nearest to x (the same greedy descent
  // on every lane), its items split over the lanes
  {
    const int top = T.nlevels - 1;
    int64_t best = 0;
    float bk = INFINITY;
    for (int64_t j = 0; j < T.count[top]; ++j) {
      const float4 B = T.na[T.offset[top] + j];
      const float k = dist32(x32, y32, z32, B) - B.w;
      if (k < bk) {
        bk = k;
        best = j;
      }
    }
    for (int lev = top; lev > 0; --lev) {
      const int64_t cb = best * kFan, ce = imin64(cb + kFan, T.count[lev - 1]);
      const int64_t off = T.offset[lev - 1];
      bk = INFINITY;
      for (int64_t c = cb; c < ce; ++c) {
        const float4 B = T.na[off + c];
        const float k = dist32(x32, y32, z32, B) - B.w;
        if (k < bk || c == cb) {
          bk = k;
          best = c;
        }
      }
    }
    const int64_t j = best * kLeaf + lane;
    if (lane < kLeaf && j < a.n) item(j);
    merge();
  }
  warp_walk_until(
      T, stk, kWarpStack, lane, &a.cnt->walk_err,
      [&]() {
        merge();
        return true;
      },
      [&](int64_t node) {
        const float4 B = T.na[node], W = T.nb[node], Fb = T.nf[node];
        const float dF = dist32(x32, y32, z32, Fb);
        if (dF - err32(ax, Fb, dF, Fb.w) - Fb.w <= thF) return true;
        const float dC = dist32(x32, y32, z32, B);
        for (int cl = 0; cl < 2; ++cl) {
          const float w = cl == 0 ? W.x : W.y;
          if (!(w > -INFINITY)) continue;
          if (dC - err32(ax, B, dC, w) - w <= thA[cl]) return true;
        }
        return false;
      },
      [&](int64_t idx) {
        const int64_t b = idx * kLeaf, e = imin64(b + kLeaf, a.n);
        for (int64_t j = b; j < e; ++j) item(j);
      });
  merge();
}

// tangent_search over the warp; every lane receives the result.
__device__ inline void warp_tangent_search(const QueryArgs& a, int box_cull, double x, double y, double z, int cs,
                                           int mode, double lim, double lo, uint32_t* stk, int lane, TanBest& B) {
  const Tree& T = a.st;
  const double lim_d = mode == kBelowSurvivor ? sqrt(lim) : (mode == kWithinOpposite ? lim : INFINITY);
  const float x32 = float(x), y32 = float(y), z32 = float(z), ax = amax3(x32, y32, z32);
  const float lo_f = f_dn(lo);
  float hi_f = INFINITY;
  int hint = -1;  // the ball that covered this lane's last tangent point
  auto merge = [&]() {
    warp_min_vl(B.d2, B.id);
    // distances beyond hi cannot change the result
    const double hi = (B.id >= 0 ? fmin(lim_d, sqrt(B.d2)) : lim_d) * kRel + kAbs;
    hi_f = f_up(hi);
  };
  merge();
  warp_walk_until(
      T, stk, kWarpStack, lane, &a.cnt->walk_err,
      [&]() {
        merge();
        return true;
      },
      [&](int64_t node) {
        const float4 W = T.nb[node];
        const float w = cs == 0 ? W.x : W.y;
        if (!(w > -INFINITY)) return false;
        const float4 Cb = T.na[node], Fb = T.nf[node];
        const float dc = dist32(x32, y32, z32, Cb), df = dist32(x32, y32, z32, Fb);
        const float ec = err32(ax, Cb, dc, w), ef = err32(ax, Fb, df, Fb.w);
        const float near_lo = dc - w - ec, near_hi = fmaxf(w - dc + ec, df + Fb.w + ef);
        const float far_lo = df - Fb.w - ef, far_hi = dc + w + ec;
        return (near_lo <= hi_f && near_hi >= lo_f) || (far_lo <= hi_f && far_hi >= lo_f);
      },
      [&](int64_t idx) {
        const int64_t b = idx * kLeaf, e = imin64(b + kLeaf, a.n);
        for (int64_t j = b; j < e; ++j) {
          const float4 S = a.sph[j];
          if (S.w == 0.f || int(S.w < 0.f) != cs) continue;
          const float d32 = dist32(x32, y32, z32, S), r32 = fabsf(S.w);
          const float er = err32(ax, S, d32, r32);
          const float an32 = fabsf(d32 - r32), af32 = d32 + r32;
          const bool try_near = an32 + er >= lo_f && an32 - er <= hi_f;
          const bool try_far = af32 + er >= lo_f && af32 - er <= hi_f;
          if (!try_near && !try_far) continue;
          const int o = a.sid[j];
          const D4 P = a.sph64[o];
          const double r = fabs(P.w);
          const double vx = __dsub_rn(x, P.x), vy = __dsub_rn(y, P.y), vz = __dsub_rn(z, P.z);
          const double dv =
              __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)), __dmul_rn(vz, vz)));
          if (!(dv > 0.0)) continue;
          const double ux = __ddiv_rn(vx, dv), uy = __ddiv_rn(vy, dv), uz = __ddiv_rn(vz, dv);
          for (int side = 0; side < 2; ++side) {
            if (!(side == 0 ? try_near : try_far)) continue;
            const double sr = side == 0 ? r : -r;
            const double tx = __dadd_rn(P.x, __dmul_rn(sr, ux));
            const double ty = __dadd_rn(P.y, __dmul_rn(sr, uy));
            const double tz = __dadd_rn(P.z, __dmul_rn(sr, uz));
            if (box_cull && !ex_inbox(tx, ty, tz)) continue;
            const double d2 = ex_d2(x, y, z, tx, ty, tz);
            const bool within =
                mode == kBelowSurvivor ? d2 < lim : (mode == kWithinOpposite ? __dsqrt_rn(d2) <= lim : true);
            if (!within) continue;
            const int64_t id = 2 * int64_t(o) + side;
            if (B.id >= 0 && (d2 > B.d2 || (d2 == B.d2 && id > B.id))) continue;
            if (hint >= 0 && hint != o && ex_cov(tx, ty, tz, a.sph64[hint], a.tol)) continue;
            const int k = covered_by_other(a, tx, ty, tz, o);
            if (k >= 0) {
              hint = k;
              continue;
            }
            B.d2 = d2;
            B.id = id;
          }
        }
      });
  merge();
}

// tangent_one over the warp (lane 0 writes the outputs).
__device__ inline void warp_tangent_one(const QueryArgs& a, int box_cull, int64_t q, uint32_t* stk, int lane) {
  const int code = a.fl_out[q] & 15;
  if (code != GFS_CODE_SURVIVOR && code != GFS_CODE_OPPOSITE && code != GFS_CODE_LOWER) return;
  double x, y, z;
  load_point(a, q, x, y, z);
  SphereBounds S;
  warp_sphere_bounds(a, x, y, z, stk, lane, S);
  if (S.cov[0] == S.cov[1]) return;  // OUTSIDE / INVALID: not refined
  const int cs = S.cov[0] ? 0 : 1, co = 1 - cs;
  const bool have_u = S.idxA[co] != INT_MAX;
  const double ub = have_u ? S.bestA[co] : INFINITY;
  int mode = kUnlimited;
  double lim = INFINITY;
  if (code == GFS_CODE_SURVIVOR) {
    double qx, qy, qz;
    if (!survivor_pos(a, a.arg_out[q], qx, qy, qz)) return;  // not this state's query output
    mode = kBelowSurvivor;
    lim = ex_d2(x, y, z, qx, qy, qz);
  } else if (code == GFS_CODE_OPPOSITE) {
    mode = kWithinOpposite;
    lim = ub;
  }
  const double lbv = -S.bestA[cs];
  const double lo = lbv - a.tol - 1e-9 - 1e-12 * fabs(lbv);
  TanBest B;
  B.d2 = INFINITY;
  B.id = -1;
  __syncwarp();
  warp_tangent_search(a, box_cull, x, y, z, cs, mode, lim, lo, stk, lane, B);
  if (B.id < 0 || lane != 0) return;
  const double m = __dsqrt_rn(B.d2);
  if (a.clamp_opp && !(m <= ub)) return;  // the opposite tangent point stays the value
  const double lb = -S.bestA[cs];
  int flags = GFS_CODE_TANGENT;
  if (m < __dsub_rn(lb, a.tol)) flags |= GFS_FLAG_LB_VIOL;
  if (m > __dadd_rn(S.bestF, a.tol)) flags |= GFS_FLAG_FAR_VIOL;
  if (have_u && ub < __dsub_rn(m, a.tol)) flags |= GFS_FLAG_OPP_VIOL;
  const double v = cs == 0 ? m : -m;
  if (a.s_out) a.s_out[q] = float(v);
  if (a.s64_out) a.s64_out[q] = v;
  a.arg_out[q] = B.id;
  a.fl_out[q] = uint16_t(flags);
}

}  // namespace tangent
}  // namespace gfs
