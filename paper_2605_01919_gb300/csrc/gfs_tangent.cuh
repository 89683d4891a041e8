// Same-sign tangent augmentation of the query: device routines.
//
// Def. 1 counts among the grow-to points T the tangent points of the
// spheres in the direction of the query point, and the exact procedure of
// Sec. 6 (min_valid_radius) takes them as candidates next to the contour
// points U and D.  The discrete query keeps only icosphere vertices on each
// sphere; this pass adds, for a point x of sign class sigma, the near and far
// tangent points of every sphere j of that class (|s_j| > 0, x != p_j),
//   side 0 (near): t = p_j + |s_j| (x - p_j) / |x - p_j|
//   side 1 (far):  t = p_j - |s_j| (x - p_j) / |x - p_j|
// kept when no other ball shrunk by tol contains t and, with the box cull,
// t lies in [-1,1]^3.  The nearest candidate over survivors and kept tangent
// points (squared distances; a survivor wins a tie, then the lowest id
// 2j + side) sets the value, clamped by the nearest opposite tangent point
// exactly as in the plain query; a tangent winner has code TANGENT and
// argmin 2j + side.
//
// Every value that decides anything is computed in FP64 with each operation
// rounded on its own, in the order written, so the decisions are those of a
// plain IEEE-754 evaluation.  Node tests and per-sphere screens run in FP32
// on the FP32 copies of the positions, widened by a bound on their rounding
// error (err32), so they only skip nodes and spheres that cannot decide
// anything; what passes them is evaluated in FP64.
//
// Also here, shared with the other exact passes: the screened coverage walk
// (covered_except: is a point inside a shrunk ball other than up to three
// given ones) and the point q* behind a query value (argmin_point).
#pragma once

#include <climits>
#include <cmath>

#include "gfs_kernels.h"

namespace gfs {
namespace tangent {

constexpr double kRel = 1.0 + 1e-12;  // widening of FP32 node radii in FP64 tests
constexpr double kAbs = 1e-12;

__device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }


// |x - q| in FP32, x rounded from FP64, q an FP32 point (node centre, or a
// sphere centre rounded from FP64)
__device__ __forceinline__ float dist32(float x, float y, float z, const float4& q) {
  const float dx = x - q.x, dy = y - q.y, dz = z - q.z;
  return sqrtf(dx * dx + dy * dy + dz * dz);
}

__device__ __forceinline__ float amax3(float x, float y, float z) { return fmaxf(fabsf(x), fmaxf(fabsf(y), fabsf(z))); }

// Bound on the error of dist32, and of an FP32 expression dist32 +- r +- this
// bound for a value r (a radius rounded from FP64, or an exact node radius),
// against the exact values of the FP64 points: the roundings of the
// coordinates (u |x| + u |q| per axis, sqrt 3 of that in the norm), of the
// FP32 norm (about 2.5 u d) and of the sums (a few u (d + r)), u = 2^-24,
// taken four times over.
__device__ __forceinline__ float err32(float ax, const float4& q, float d, float r) {
  return 16.f * 5.9604645e-8f * (ax + amax3(q.x, q.y, q.z) + d + fabsf(r)) + 1e-30f;
}

// FP32 values on the safe side of an FP64 threshold (one FP32 rounding of
// relative size <= u, covered twice)
__device__ __forceinline__ float f_up(double v) {
  const float f = float(v);
  return f + fabsf(f) * 2.4e-7f + 1e-37f;
}
__device__ __forceinline__ float f_dn(double v) {
  const float f = float(v);
  return f - fabsf(f) * 2.4e-7f - 1e-37f;
}

__device__ __forceinline__ void load_point(const QueryArgs& a, int64_t q, double& x, double& y, double& z) {
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

// Sec. 4.3 quantities at x over all spheres: containment per sign class
// (class 0 positive, 1 negative), the smallest |x - p_j| - r_j per class with
// its lowest input index (UB_opp for the opposite class, -LB for x's own),
// and the smallest |x - p_j| + r_j (the far bound).
struct SphereBounds {
  bool cov[2];
  double bestA[2];
  int idxA[2];
  double bestF;
};

__device__ inline void sphere_bounds(const QueryArgs& a, double x, double y, double z, SphereBounds& R) {
  const double tol = a.tol;
  R.cov[0] = R.cov[1] = false;
  R.bestA[0] = R.bestA[1] = INFINITY;
  R.idxA[0] = R.idxA[1] = INT_MAX;
  R.bestF = INFINITY;
  const float x32 = float(x), y32 = float(y), z32 = float(z), ax = amax3(x32, y32, z32);
  // FP32 copies (rounded up) of the thresholds a sphere must reach to matter:
  // the far bound, and per class the best |x - p| - r (at least -tol while
  // the class has no containing ball)
  float thF = INFINITY, thA[2] = {INFINITY, INFINITY};
  const Tree& T = a.st;
  uint32_t stack[kStack];
  int sp = 0;
  const int top = T.nlevels - 1;
  // seed: descend first to the leaf whose balls reach nearest to x (least
  // |x - C| - w at every level), so that the thresholds are tight before
  // the full walk; that leaf is visited again by the walk, which changes
  // nothing (minima with index ties are idempotent)
  {
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
    // the whole hierarchy, then the seed leaf on top of the stack (popped first)
    for (int64_t j = 0; j < T.count[top]; ++j) stack[sp++] = pack_node(top, j);
    stack[sp++] = pack_node(0, best);
  }
  while (sp > 0) {
    const uint32_t nd = stack[--sp];
    const int lev = node_level(nd);
    const int64_t idx = node_index(nd);
    if (lev == 0) {
      const int64_t b = idx * kLeaf, e = imin64(b + kLeaf, a.n);
      for (int64_t j = b; j < e; ++j) {
        // screen: the sphere can only matter if it may lower the far bound,
        // lower (or tie) its class's |x - p| - r, or contain x
        const float4 S = a.sph[j];
        const float d32 = dist32(x32, y32, z32, S), r32 = fabsf(S.w);
        const float er = err32(ax, S, d32, r32);
        bool need = d32 + r32 - er <= thF;
        if (S.w != 0.f) need = need || d32 - r32 - er <= thA[S.w < 0.f];
        if (!need) continue;
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
          thA[c] = f_up(R.cov[c] ? R.bestA[c] : fmax(R.bestA[c], -tol));
        }
        const double f = __dadd_rn(dl, r);
        if (f < R.bestF) {
          R.bestF = f;
          thF = f_up(f);
        }
      }
    } else {
      const int64_t cb = idx * kFan, ce = imin64(cb + kFan, T.count[lev - 1]);
      const int64_t off = T.offset[lev - 1];
      for (int64_t c = cb; c < ce; ++c) {
        const float4 B = T.na[off + c], W = T.nb[off + c], Fb = T.nf[off + c];
        // far bound: |x - p_j| + r_j >= |x - F| - wf
        const float dF = dist32(x32, y32, z32, Fb);
        bool need = dF - err32(ax, Fb, dF, Fb.w) - Fb.w <= thF;
        // near bound per class: |x - p_j| - r_j >= |x - C| - w_class; a class
        // without containment yet also needs every ball that could hold x
        if (!need) {
          const float dC = dist32(x32, y32, z32, B);
          for (int cl = 0; cl < 2 && !need; ++cl) {
            const float w = cl == 0 ? W.x : W.y;
            if (!(w > -INFINITY)) continue;
            need = dC - err32(ax, B, dC, w) - w <= thA[cl];
          }
        }
        if (need) stack[sp++] = pack_node(lev - 1, c);
      }
    }
  }
}

// A ball other than spheres skip0..skip2 (input indices; -1 for none) that,
// shrunk by tol, contains t (Sec. 3.1: the open balls; App. B tolerance), or
// -1.  A ball of the node with centre C and radius bound w can only contain t
// when |t - C| < w.
// The walk on a stack of kStack entries that the caller provides.
__device__ inline int covered_except_on(uint32_t* stack, const QueryArgs& a, double tx, double ty, double tz,
                                        int skip0, int skip1, int skip2) {
  const float x32 = float(tx), y32 = float(ty), z32 = float(tz), ax = amax3(x32, y32, z32);
  const float ntol = -f_dn(a.tol);  // >= -tol
  const Tree& T = a.st;
  int sp = 0;
  const int top = T.nlevels - 1;
  for (int64_t j = 0; j < T.count[top]; ++j) stack[sp++] = pack_node(top, j);
  // seed: the leaf reached by always entering the child ball that holds t
  // most deeply (least |t - C| - w) is tested first; a covered point usually
  // lies in one of its balls
  {
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
    stack[sp++] = pack_node(0, best);
  }
  while (sp > 0) {
    const uint32_t nd = stack[--sp];
    const int lev = node_level(nd);
    const int64_t idx = node_index(nd);
    if (lev == 0) {
      const int64_t b = idx * kLeaf, e = imin64(b + kLeaf, a.n);
      for (int64_t j = b; j < e; ++j) {
        // screen: containment needs |t - p| < r - tol
        const float4 S = a.sph[j];
        if (S.w == 0.f) continue;
        const float d32 = dist32(x32, y32, z32, S), r32 = fabsf(S.w);
        if (d32 - r32 - err32(ax, S, d32, r32) >= ntol) continue;
        const int o = a.sid[j];
        if (o == skip0 || o == skip1 || o == skip2) continue;
        if (ex_cov(tx, ty, tz, a.sph64[o], a.tol)) return o;
      }
    } else {
      const int64_t cb = idx * kFan, ce = imin64(cb + kFan, T.count[lev - 1]);
      const int64_t off = T.offset[lev - 1];
      // push the children that may hold a covering ball, the one holding t
      // most deeply last (popped first)
      const int base = sp;
      float key[kFan];
      for (int64_t c = cb; c < ce; ++c) {
        const float4 B = T.na[off + c];
        if (!(B.w > 0.f)) continue;
        const float dC = dist32(x32, y32, z32, B);
        if (!(dC - err32(ax, B, dC, B.w) < B.w)) continue;
        const float k = dC - B.w;
        int u = sp++;
        while (u > base && key[u - 1 - base] < k) {
          stack[u] = stack[u - 1];
          key[u - base] = key[u - 1 - base];
          --u;
        }
        stack[u] = pack_node(lev - 1, c);
        key[u - base] = k;
      }
    }
  }
  return -1;
}

__device__ inline int covered_except(const QueryArgs& a, double tx, double ty, double tz, int skip0, int skip1,
                                     int skip2) {
  uint32_t stack[kStack];
  return covered_except_on(stack, a, tx, ty, tz, skip0, skip1, skip2);
}

__device__ __forceinline__ int covered_by_other(const QueryArgs& a, double tx, double ty, double tz, int skip) {
  return covered_except(a, tx, ty, tz, skip, -1, -1);
}

// How far a tangent point may lie from x and still change the result.
enum Limit {
  kBelowSurvivor = 0,  // squared distance < lim (the nearest survivor's, a survivor wins ties)
  kWithinOpposite = 1, // distance <= lim (UB_opp, the clamp keeps a tangent point that ties it)
  kUnlimited = 2       // no candidate at all so far
};

struct TanBest {
  double d2;   // squared distance of the best kept tangent point
  int64_t id;  // 2j + side, or -1
};

// The nearest kept tangent point of class cs within the limit, ties to the
// lowest id.  A tangent point of sphere j lies on sphere j, inside the node
// ball (C, w_cs), so it is at least |x - C| - w_cs and at most |x - C| + w_cs
// away from x.
//
// lo: tangent points nearer to x than lo are known to be covered.  With A the
// containing sphere of x's class that attains LB = r_A - |x - p_A| (Sec. 4.3),
// a point t with |t - x| <= LB - tol - delta has |t - p_A| <= r_A - tol - delta
// (triangle inequality), so A's shrunk ball holds it with a margin delta that
// no FP64 rounding of the coverage test can undo; A's own tangent points are
// at least LB away, so t is never one of them.  Such points are skipped
// without a coverage walk, which is what keeps the pass affordable at points
// deep inside many balls.
__device__ inline void tangent_search(const QueryArgs& a, int box_cull, double x, double y, double z, int cs,
                                      int mode, double lim, double lo, TanBest& B) {
  const Tree& T = a.st;
  uint32_t stack[kStack];
  int sp = 0;
  const int top = T.nlevels - 1;
  for (int64_t j = 0; j < T.count[top]; ++j) stack[sp++] = pack_node(top, j);
  const double lim_d = mode == kBelowSurvivor ? sqrt(lim) : (mode == kWithinOpposite ? lim : INFINITY);
  const float x32 = float(x), y32 = float(y), z32 = float(z), ax = amax3(x32, y32, z32);
  int hint = -1;  // the ball that covered the last tangent point tested: neighbours often share it
  while (sp > 0) {
    const uint32_t nd = stack[--sp];
    const int lev = node_level(nd);
    const int64_t idx = node_index(nd);
    // distances beyond hi cannot change the result
    const double hi = (B.id >= 0 ? fmin(lim_d, sqrt(B.d2)) : lim_d) * kRel + kAbs;
    const float hi_f = f_up(hi), lo_f = f_dn(lo);
    if (lev == 0) {
      const int64_t b = idx * kLeaf, e = imin64(b + kLeaf, a.n);
      for (int64_t j = b; j < e; ++j) {
        const float4 S = a.sph[j];
        if (S.w == 0.f || int(S.w < 0.f) != cs) continue;
        // screen: |x - t| is |d - r| (near) or d + r (far)
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
        const double dv = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)), __dmul_rn(vz, vz)));
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
          const bool within = mode == kBelowSurvivor ? d2 < lim
                                                     : (mode == kWithinOpposite ? __dsqrt_rn(d2) <= lim : true);
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
    } else {
      const int64_t cb = idx * kFan, ce = imin64(cb + kFan, T.count[lev - 1]);
      const int64_t off = T.offset[lev - 1];
      for (int64_t c = cb; c < ce; ++c) {
        const float4 W = T.nb[off + c];
        const float w = cs == 0 ? W.x : W.y;
        if (!(w > -INFINITY)) continue;
        const float4 Cb = T.na[off + c], Fb = T.nf[off + c];
        const float dc = dist32(x32, y32, z32, Cb), df = dist32(x32, y32, z32, Fb);
        const float ec = err32(ax, Cb, dc, w), ef = err32(ax, Fb, df, Fb.w);
        // bounds over the node's spheres j of class cs, with d = |x - p_j|:
        //   near |d - r_j|: >= d - r_j >= dc - w;  r_j - d <= w - dc;
        //                   d - r_j <= df + |p_j - F| - r_j <= df + wf
        //   far d + r_j:    <= dc + w;  >= df - (|p_j - F| - r_j) >= df - wf
        const float near_lo = dc - w - ec, near_hi = fmaxf(w - dc + ec, df + Fb.w + ef);
        const float far_lo = df - Fb.w - ef, far_hi = dc + w + ec;
        if ((near_lo <= hi_f && near_hi >= lo_f) || (far_lo <= hi_f && far_hi >= lo_f))
          stack[sp++] = pack_node(lev - 1, c);
      }
    }
  }
}

// FP64 position of survivor g (icosphere vertex, or an inserted sphere's
// witness in slot K); false for an id that names no candidate of this state
__device__ __forceinline__ bool survivor_pos(const QueryArgs& a, int64_t g, double& qx, double& qy, double& qz) {
  if (g < 0) return false;
  const int64_t i = g / a.KS, k = g % a.KS;
  if (i >= a.n) return false;
  if (k < a.K) {
    ex_cand(a.sph64[i], a.U64[3 * k], a.U64[3 * k + 1], a.U64[3 * k + 2], qx, qy, qz);
    return true;
  }
  if (!a.witness64) return false;
  const double* w = a.witness64 + 3 * i;
  qx = w[0];
  qy = w[1];
  qz = w[2];
  return true;
}

// Refine one query's result in place (the outputs of the plain query).
__device__ inline void tangent_one(const QueryArgs& a, int box_cull, int64_t q) {
  const int code = a.fl_out[q] & 15;
  if (code != GFS_CODE_SURVIVOR && code != GFS_CODE_OPPOSITE && code != GFS_CODE_LOWER) return;
  double x, y, z;
  load_point(a, q, x, y, z);
  SphereBounds S;
  sphere_bounds(a, x, y, z, S);
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
  // points nearer than the deepest containing ball's reach, less tol and a
  // margin far above FP64 rounding, are covered by that ball
  const double lbv = -S.bestA[cs];
  const double lo = lbv - a.tol - 1e-9 - 1e-12 * fabs(lbv);
  TanBest B;
  B.d2 = INFINITY;
  B.id = -1;
  tangent_search(a, box_cull, x, y, z, cs, mode, lim, lo, B);
  if (B.id < 0) return;
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

// The point q* that sets a query's value, from its argmin g and code:
// SURVIVOR: the candidate (or witness); OPPOSITE / LOWER j: the near tangent
// point of sphere j; TANGENT 2j + side: that tangent point; OUTSIDE, and
// OPPOSITE / LOWER with no sphere: x; SAMPLE, INVALID, an undefined
// direction (x = p_j) or an id this state does not hold: NaN.
__device__ inline void argmin_point(const QueryArgs& a, double x, double y, double z, int code, int64_t g,
                                    double* o) {
  o[0] = o[1] = o[2] = NAN;
  if (code == GFS_CODE_SURVIVOR) {
    double qx, qy, qz;
    if (survivor_pos(a, g, qx, qy, qz)) {
      o[0] = qx;
      o[1] = qy;
      o[2] = qz;
    }
  } else if (code == GFS_CODE_OUTSIDE || ((code == GFS_CODE_LOWER || code == GFS_CODE_OPPOSITE) && g < 0)) {
    o[0] = x;
    o[1] = y;
    o[2] = z;
  } else if (code == GFS_CODE_OPPOSITE || code == GFS_CODE_LOWER || code == GFS_CODE_TANGENT) {
    const int64_t j = code == GFS_CODE_TANGENT ? g / 2 : g;
    if (j < 0 || j >= a.n) return;
    const D4 P = a.sph64[j];
    const double r = fabs(P.w);
    const double sr = (code == GFS_CODE_TANGENT && g % 2 == 1) ? -r : r;
    const double vx = __dsub_rn(x, P.x), vy = __dsub_rn(y, P.y), vz = __dsub_rn(z, P.z);
    const double dv = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)), __dmul_rn(vz, vz)));
    if (!(dv > 0.0)) return;
    o[0] = __dadd_rn(P.x, __dmul_rn(sr, __ddiv_rn(vx, dv)));
    o[1] = __dadd_rn(P.y, __dmul_rn(sr, __ddiv_rn(vy, dv)));
    o[2] = __dadd_rn(P.z, __dmul_rn(sr, __ddiv_rn(vz, dv)));
  }
}

}  // namespace tangent
}  // namespace gfs
