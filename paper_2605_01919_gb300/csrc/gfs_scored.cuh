// Scored value of the query (Sec. 3.3: score_for_radius, interpolate_sdf_to):
// device routines (the kernel and its launcher are in gfs_scored.cu).
//
// The paper does not return the minimum valid radius at a new point but the
// best-scoring valid one: every grow-to point q, with the input sphere i it
// lies on, gives the radius r = |x - q| for both signs; the type score ranks
// tangency points whose normals agree highest, then intersection points that
// agree, intersection points that disagree, tangency points that disagree;
// within a type the sign score prefers large radii, negative ones twice as
// much; the first valid value in that order is returned.  Here the grow-to
// points are the survivors S_tau (for the intersection points U, D) and the
// near and far tangent points of every sphere that no other shrunk ball
// covers (T of Def. 1); a value is valid when
//   (V1) it intersects no ball of the opposite sign (not UB < r - tol),
//   (V2) no sphere other than i loses all its survivors to the new ball
//        shrunk by tol (sphere i keeps q, on the new sphere),
//   (V3) no sphere lies strictly inside the new ball (not r > FAR + tol).
// normals_agree: sign * (x - q) and sign(s_i) * (p_i - q) have a positive dot
// product; ties go to the lower candidate key (survivor id g; tangent points
// after every survivor, 2j + side), then to the negative sign.  Points where
// no candidate is valid keep the plain query's result, flagged
// GFS_FLAG_SCORE_FALLBACK; SAMPLE and INVALID results are kept.
//
// One thread per point (Morton order), every decision in FP64 with each
// operation rounded on its own in the order written; node and item screens in
// FP32 with a bound on their rounding error only skip what cannot matter.
#pragma once

#include <climits>
#include <cstdint>

#include "gfs.h"
#include "gfs_tangent.cuh"

namespace gfs {
namespace scored {

using tangent::amax3;
using tangent::dist32;
using tangent::err32;
using tangent::f_up;
using tangent::imin64;

struct Best {
  int cls;      // type class 0..3, -1 none
  double sr;    // sign score * r
  int64_t key;  // survivor id, or kTanKey + 2j + side
  int sign;     // +1 / -1
  double r;
};

constexpr int64_t kTanKey = int64_t(1) << 40;

__device__ __forceinline__ bool better(int cls, double sr, int64_t key, int sign, const Best& b) {
  if (b.cls < 0) return true;
  if (cls != b.cls) return cls > b.cls;
  if (sr != b.sr) return sr > b.sr;
  if (key != b.key) return key < b.key;
  return sign < b.sign;
}

// dot product (x - q) . (p - q), summed left to right
__device__ __forceinline__ double dot_xq_pq(double x, double y, double z, double qx, double qy, double qz, const D4& P) {
  const double a0 = __dmul_rn(__dsub_rn(x, qx), __dsub_rn(P.x, qx));
  const double a1 = __dmul_rn(__dsub_rn(y, qy), __dsub_rn(P.y, qy));
  const double a2 = __dmul_rn(__dsub_rn(z, qz), __dsub_rn(P.z, qz));
  return __dadd_rn(__dadd_rn(a0, a1), a2);
}

struct Frame {
  double x, y, z;
  float x32, y32, z32, ax;
  int sig;             // allowed sign: +1, -1, or 0 (both)
  double ub[2];        // [0]: bound for positive values (negative spheres), [1]: for negative values
  double far;          // FAR
  double m1, m2;       // two least squared distances to the farthest survivor of a sphere
  int64_t j1, j2;      // their spheres
};

// Work budget of one point: every node pop, item and list entry costs one
// unit; a point that runs out (corrupted state; the walks are bounded by the
// hierarchy sizes otherwise) stops, keeps the plain query's result and
// records the phase in the status word (bit 0: survivor walks, bit 1: the
// per-sphere survivor lists, bit 2: tangent walk).
constexpr unsigned kScoreBudget = 1u << 24;

struct Budget {
  unsigned used = 0;
  unsigned failed = 0;
  __device__ __forceinline__ bool spend(unsigned phase) {
    if (++used <= kScoreBudget) return true;
    failed |= phase;
    return false;
  }
};

// Try candidate q (on sphere i) for both allowed signs against the best.
// tan: tangency point; key: its candidate key.  Returns whether it became
// the best (so the caller may run a coverage test only when needed).
template <class Accept>
__device__ __forceinline__ void try_candidate(const QueryArgs& a, const Frame& F, double qx, double qy, double qz,
                                              int64_t i, bool tan, int64_t key, Best& B, Accept accept) {
  const double tol = a.tol;
  const double r = __dsqrt_rn(ex_d2(F.x, F.y, F.z, qx, qy, qz));
  const D4 P = a.sph64[i];
  const double dn = dot_xq_pq(F.x, F.y, F.z, qx, qy, qz, P);
  const int si = P.w > 0.0 ? 1 : (P.w < 0.0 ? -1 : 0);
  for (int sgi = 0; sgi < 2; ++sgi) {
    const int sign = sgi == 0 ? 1 : -1;
    if (F.sig != 0 && sign != F.sig) continue;
    if (F.ub[sgi] < __dsub_rn(r, tol)) continue;  // V1
    if (r > __dadd_rn(F.far, tol)) continue;      // V3
    if (r > tol) {                                // V2
      const double rt = __dsub_rn(r, tol);
      const double eff = (i == F.j1) ? F.m2 : F.m1;
      if (eff < __dmul_rn(rt, rt)) continue;
    }
    const bool agree = double(sign * si) * dn > 0.0;
    const int cls = tan ? (agree ? 3 : 0) : (agree ? 2 : 1);
    const double sr = sign > 0 ? r : 2.0 * r;
    if (better(cls, sr, key, sign, B) && accept()) {
      B.cls = cls;
      B.sr = sr;
      B.key = key;
      B.sign = sign;
      B.r = r;
    }
  }
}

// Walk one survivor hierarchy: every item whose FP32 screen allows an exact
// distance <= R (per item the callback decides exactly).
template <class Item>
__device__ inline void walk_survivors(const QueryArgs& a, const Frame& F, int cls, double R, Budget& Bu, Item item) {
  const Tree& T = a.vt[cls];
  if (T.nlevels == 0) return;
  const float R32 = f_up(R);
  const float4* items = a.surv[cls];
  uint32_t stack[kStack];
  int sp = 0;
  const int top = T.nlevels - 1;
  for (int64_t j = 0; j < T.count[top] && sp < kStack; ++j) stack[sp++] = pack_node(top, j);
  while (sp > 0) {
    if (!Bu.spend(1u)) return;
    const uint32_t nd = stack[--sp];
    const int lev = node_level(nd);
    const int64_t idx = node_index(nd);
    if (lev == 0) {
      const int64_t b = idx * kLeaf, e = imin64(b + kLeaf, T.nitems);
      for (int64_t j = b; j < e; ++j) {
        if (!Bu.spend(1u)) return;
        const float4 S = items[j];
        const float d32 = dist32(F.x32, F.y32, F.z32, S);
        // the FP32 position is within the candidate error bound of the exact one
        if (d32 - err32(F.ax, S, d32, 0.f) - 4.f * a.bc->eq > R32) continue;
        item(__float_as_uint(S.w));
      }
    } else {
      const int64_t cb = idx * kFan, ce = imin64(cb + kFan, T.count[lev - 1]);
      const int64_t off = T.offset[lev - 1];
      for (int64_t c = cb; c < ce; ++c) {
        const float bd = sqrtf(box_d2(F.x32, F.y32, F.z32, T.lo[off + c], T.hi[off + c]));
        if (bd * (1.f - 1e-6f) - 4.f * a.bc->eq <= R32) {
          if (sp >= kStack) {  // cannot happen for a well-formed hierarchy
            Bu.failed |= 1u;
            Bu.used = kScoreBudget;
            return;
          }
          stack[sp++] = pack_node(lev - 1, c);
        }
      }
    }
  }
}

__device__ inline void scored_one(const QueryArgs& a, int box_cull, const uint32_t* __restrict__ csr_ids,
                                  const int64_t* __restrict__ csr_off, int64_t q, unsigned* status) {
  const int code = a.fl_out[q] & 15;
  if (code == GFS_CODE_SAMPLE || code == GFS_CODE_INVALID) return;
  const double tol = a.tol;
  Frame F;
  tangent::load_point(a, q, F.x, F.y, F.z);
  F.x32 = float(F.x);
  F.y32 = float(F.y);
  F.z32 = float(F.z);
  F.ax = amax3(F.x32, F.y32, F.z32);
  tangent::SphereBounds SB;
  tangent::sphere_bounds(a, F.x, F.y, F.z, SB);
  if (SB.cov[0] && SB.cov[1]) return;  // INVALID (the plain query says so too)
  F.sig = SB.cov[0] ? 1 : (SB.cov[1] ? -1 : 0);
  F.ub[0] = SB.bestA[1];
  F.ub[1] = SB.bestA[0];
  F.far = SB.bestF;
  const double R = __dadd_rn(F.far, tol);  // no valid radius exceeds it (V3)
  // (V2) spheres with a survivor within R: their farthest survivor, from the
  // per-sphere survivor lists; a sphere without one has every survivor
  // farther than any valid radius
  F.m1 = F.m2 = INFINITY;
  F.j1 = F.j2 = -1;
  // spheres already measured (a sphere's survivors come in runs of the
  // Morton order): a small ring of the latest, to avoid most repeats
  int64_t seen[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
  Budget Bu;
  int seen_at = 0;
  auto v2_sphere = [&](uint32_t g) {
    const int64_t i = int64_t(g) / a.KS;
    if (i == F.j1 || i == F.j2) return;
    for (int u = 0; u < 8; ++u)
      if (seen[u] == i) return;
    seen[seen_at] = i;
    seen_at = (seen_at + 1) & 7;
    double md = -1.0;
    const int64_t u0 = csr_off[i], u1 = imin64(csr_off[i + 1], u0 + a.KS);  // at most KS per sphere
    for (int64_t u = u0; u < u1; ++u) {
      if (!Bu.spend(2u)) return;
      double qx, qy, qz;
      tangent::survivor_pos(a, int64_t(csr_ids[u]), qx, qy, qz);
      const double d2 = ex_d2(F.x, F.y, F.z, qx, qy, qz);
      if (d2 > md) md = d2;
    }
    if (md < 0.0) return;
    if (md < F.m1) {
      F.m2 = F.m1;
      F.j2 = F.j1;
      F.m1 = md;
      F.j1 = i;
    } else if (md < F.m2) {
      F.m2 = md;
      F.j2 = i;
    }
  };
  walk_survivors(a, F, 0, R, Bu, v2_sphere);
  walk_survivors(a, F, 1, R, Bu, v2_sphere);
  Best B;
  B.cls = -1;
  // survivors (intersection points)
  auto surv_cand = [&](uint32_t g) {
    double qx, qy, qz;
    tangent::survivor_pos(a, int64_t(g), qx, qy, qz);
    try_candidate(a, F, qx, qy, qz, int64_t(g) / a.KS, false, int64_t(g), B, []() { return true; });
  };
  walk_survivors(a, F, 0, R, Bu, surv_cand);
  walk_survivors(a, F, 1, R, Bu, [&](uint32_t g) {
    // a zero sample's survivors are in both lists: once is enough
    if (a.sph64[int64_t(g) / a.KS].w == 0.0) return;
    surv_cand(g);
  });
  // tangent points: spheres whose near or far tangent point may lie within R
  {
    const Tree& T = a.st;
    const float R32 = f_up(R);
    // one array holds this walk's stack and, above it, the stack of the
    // coverage walks it runs: with an array of their own the compiler gave
    // both the same local memory, and each coverage walk overwrote this one
    uint32_t stack[2 * kStack];
    uint32_t* const cstack = stack + kStack;
    int sp = 0;
    // the balls that covered the latest tangent points: neighbouring
    // tangent points are mostly covered by the same few large balls, so
    // these are tested before a walk (a ball found here is one the walk
    // could have returned: the decision is the same)
    int hint[4] = {-1, -1, -1, -1};
    float4 hintf[4];  // their centres in FP32 and radius - tol rounded down
    int hint_at = 0;
    auto uncovered_tan = [&](double tx, double ty, double tz, int j) -> bool {
      for (int u = 0; u < 4; ++u) {
        const int c = hint[u];
        if (c >= 0 && c != j && ex_cov(tx, ty, tz, a.sph64[c], a.tol)) return false;
      }
      const int o = tangent::covered_except_on(cstack, a, tx, ty, tz, j, -1, -1);
      if (o < 0) return true;
      const D4 Q = a.sph64[o];
      hint[hint_at] = o;
      hintf[hint_at] = make_float4(float(Q.x), float(Q.y), float(Q.z), tangent::f_dn(__dsub_rn(fabs(Q.w), tol)));
      hint_at = (hint_at + 1) & 3;
      return false;
    };
    // Is the tangent point p + sr (x - p)/d of sphere j (FP32 copy S) surely
    // inside a cached ball other than j?  t32 is within mt of the exact
    // point (roundings of x, p, the direction and the sum, taken four
    // times over); the distance test keeps err32's margin on top.
    auto surely_covered = [&](const float4& S, float d32, float sr, int j) -> bool {
      const float ap = amax3(S.x, S.y, S.z), r = fabsf(sr);
      if (!(d32 > 1e-3f * (F.ax + ap + r))) return false;
      const float inv = 1.f / d32;
      const float tx = S.x + sr * ((F.x32 - S.x) * inv), ty = S.y + sr * ((F.y32 - S.y) * inv),
                  tz = S.z + sr * ((F.z32 - S.z) * inv);
      const float mt = 64.f * 5.9604645e-8f * (F.ax + ap + r) * (1.f + r * inv);
      const float at = amax3(tx, ty, tz);
      for (int u = 0; u < 4; ++u) {
        if (hint[u] < 0 || hint[u] == j) continue;
        const float4 H = hintf[u];
        const float dd = dist32(tx, ty, tz, H);
        if (dd + mt + err32(at, H, dd, 0.f) < H.w) return true;
      }
      return false;
    };
    const int top = T.nlevels - 1;
    for (int64_t j = 0; j < T.count[top] && sp < kStack; ++j) stack[sp++] = pack_node(top, j);
    while (sp > 0 && Bu.spend(4u)) {
      const uint32_t nd = stack[--sp];
      const int lev = node_level(nd);
      const int64_t idx = node_index(nd);
      if (lev == 0) {
        const int64_t b = idx * kLeaf, e = imin64(b + kLeaf, a.n);
        for (int64_t jj = b; jj < e; ++jj) {
          if (!Bu.spend(4u)) break;
          const float4 S = a.sph[jj];
          if (S.w == 0.f) continue;
          const float d32 = dist32(F.x32, F.y32, F.z32, S), r32 = fabsf(S.w);
          const float er = err32(F.ax, S, d32, r32);
          bool near_ok = fabsf(d32 - r32) - er <= R32, far_ok = d32 + r32 - er <= R32;
          if (!near_ok && !far_ok) continue;
          const int j = a.sid[jj];
          // FP32 screen against the best so far: a side whose radius (within
          // er of r32 +- d32) and type class cannot beat it for any allowed
          // sign, or that intersects an opposite ball for every allowed sign
          // (V1), needs no FP64 evaluation (the FP64 test would reject it)
          {
            const int si = S.w > 0.f ? 1 : -1;
            for (int side = 0; side < 2; ++side) {
              bool& ok = side == 0 ? near_ok : far_ok;
              if (!ok) continue;
              const float rr = side == 0 ? fabsf(d32 - r32) : d32 + r32;
              const float r_hi = rr + er, r_lo = rr - er;
              // near point: the normals agree when sign * si * sign(d - r) < 0;
              // far point: when sign * si > 0 (undecided near d = r)
              const int dr = side == 1 ? 0 : (d32 - r32 > er ? 1 : (r32 - d32 > er ? -1 : 2));
              bool any = false;
              for (int sgi = 0; sgi < 2 && !any; ++sgi) {
                const int sign = sgi == 0 ? 1 : -1;
                if (F.sig != 0 && sign != F.sig) continue;
                if (double(r_lo) - tol > F.ub[sgi]) continue;  // V1 fails for sure
                if (B.cls < 0) {
                  any = true;
                  break;
                }
                int cls;
                if (side == 1) cls = sign * si > 0 ? 3 : 0;
                else if (dr == 2) cls = 3;  // undecided: the highest it could be
                else cls = sign * si * dr < 0 ? 3 : 0;
                const double sr_hi = double(r_hi) * (sign > 0 ? 1.0 : 2.0);
                if (cls > B.cls || (cls == B.cls && sr_hi >= B.sr)) any = true;
              }
              if (!any) ok = false;
              // a tangent point inside another ball is no grow-to point
              else if (surely_covered(S, d32, side == 0 ? r32 : -r32, j)) ok = false;
            }
            if (!near_ok && !far_ok) continue;
          }
          const D4 P = a.sph64[j];
          const double r = fabs(P.w);
          const double vx = __dsub_rn(F.x, P.x), vy = __dsub_rn(F.y, P.y), vz = __dsub_rn(F.z, P.z);
          const double dv =
              __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)), __dmul_rn(vz, vz)));
          if (!(dv > 0.0)) continue;
          for (int side = 0; side < 2; ++side) {
            if (side == 0 ? !near_ok : !far_ok) continue;
            const double sr = side == 0 ? r : -r;
            const double tx = __dadd_rn(P.x, __dmul_rn(sr, __ddiv_rn(vx, dv)));
            const double ty = __dadd_rn(P.y, __dmul_rn(sr, __ddiv_rn(vy, dv)));
            const double tz = __dadd_rn(P.z, __dmul_rn(sr, __ddiv_rn(vz, dv)));
            if (box_cull && !ex_inbox(tx, ty, tz)) continue;
            // the coverage walk runs only for a point that would become the best
            try_candidate(a, F, tx, ty, tz, int64_t(j), true, kTanKey + 2 * int64_t(j) + side, B, [&]() {
              return Bu.spend(4u) && uncovered_tan(tx, ty, tz, j);
            });
          }
        }
      } else {
        const int64_t cb = idx * kFan, ce = imin64(cb + kFan, T.count[lev - 1]);
        const int64_t off = T.offset[lev - 1];
        for (int64_t c = cb; c < ce; ++c) {
          // a near tangent point of a sphere that does not hold x lies
          // >= |x - C| - w away; one that holds x lies within the node ball;
          // a far one >= |x - F| - wf
          const float4 Bc = T.na[off + c], Fb = T.nf[off + c];
          const float dC = dist32(F.x32, F.y32, F.z32, Bc), dF = dist32(F.x32, F.y32, F.z32, Fb);
          const bool need = dC - err32(F.ax, Bc, dC, Bc.w) - Bc.w <= R32 ||
                            dF - err32(F.ax, Fb, dF, Fb.w) - Fb.w <= R32;
          if (need) {
            if (sp >= kStack) {  // cannot happen for a well-formed hierarchy
              Bu.failed |= 4u;
              Bu.used = kScoreBudget;
              break;
            }
            stack[sp++] = pack_node(lev - 1, c);
          }
        }
      }
    }
  }
  if (Bu.failed) {
    atomicOr(status, Bu.failed);
    return;
  }
  if (B.cls < 0) {
    a.fl_out[q] = uint16_t(a.fl_out[q] | GFS_FLAG_SCORE_FALLBACK);
    return;
  }
  const bool tan = B.key >= kTanKey;
  const double v = B.sign > 0 ? B.r : -B.r;
  int flags = tan ? GFS_CODE_TANGENT : GFS_CODE_SURVIVOR;
  const int c = B.sign > 0 ? 0 : 1;
  if (SB.cov[c] && B.r < __dsub_rn(-SB.bestA[c], tol)) flags |= GFS_FLAG_LB_VIOL;
  if (a.s_out) a.s_out[q] = float(v);
  if (a.s64_out) a.s64_out[q] = v;
  a.arg_out[q] = tan ? B.key - kTanKey : B.key;
  a.fl_out[q] = uint16_t(flags);
}

}  // namespace scored
}  // namespace gfs
