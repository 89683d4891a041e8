// Exact uncovered test per sphere (Prop. 1 (ii)), device routines.
//
// Sphere i keeps a point outside every other ball shrunk by tol exactly when
// one of these points is outside every ball but i and the spheres it was
// built from (N_i: the spheres k != i with rho_k = |s_k| - tol > 0 whose
// shrunk open ball meets sphere i, | |p_i - p_k| - |s_i| | < rho_k):
//  - any point, when N_i is empty;
//  - the two points of each circle C_k = S_i with the sphere (p_k, rho_k)
//    nearest and farthest from the reference point p_i + (|s_i| + 1) e,
//    e = (0.36, 0.48, 0.8) -- an uncovered circle is wholly uncovered;
//  - the two points shared by S_i and the spheres (p_k, rho_k),
//    (p_m, rho_m), k < m in N_i -- the ends of the uncovered arcs of a
//    partly covered circle (the D points of Def. 1).
// The uncovered set, if not empty, is a closed proper subset of the sphere,
// so its boundary holds one of these points.  A sample with s_i = 0 is the
// point p_i.  Every value is computed in FP64 with each operation rounded on
// its own, in the order written (the circle and triple constructions of the
// exact grow-to points), so the decisions are those of a plain IEEE-754
// evaluation.
#pragma once

#include "gfs_tangent.cuh"

namespace gfs {
namespace exact {

constexpr int kMaxMeet = 512;  // balls meeting one sphere that a thread can hold

__device__ __forceinline__ double dot(const double* a, const double* b) {
  return __dadd_rn(__dadd_rn(__dmul_rn(a[0], b[0]), __dmul_rn(a[1], b[1])), __dmul_rn(a[2], b[2]));
}
__device__ __forceinline__ double norm(const double* v) { return __dsqrt_rn(dot(v, v)); }

// the points of the circle S(p1, r1) with S(p2, r2) nearest to and farthest
// from x; false when the spheres do not cross in a circle
__device__ inline bool circle_points(const double* p1, double r1, const double* p2, double r2, const double* x,
                                     double* out) {
  double mu[3] = {__dsub_rn(p2[0], p1[0]), __dsub_rn(p2[1], p1[1]), __dsub_rn(p2[2], p1[2])};
  const double d = norm(mu);
  if (!(d > 1e-12) || d >= __dadd_rn(r1, r2) || d <= fabs(__dsub_rn(r1, r2))) return false;
  for (int c = 0; c < 3; ++c) mu[c] = __ddiv_rn(mu[c], d);
  const double a = __ddiv_rn(__dsub_rn(__dadd_rn(__dmul_rn(d, d), __dmul_rn(r1, r1)), __dmul_rn(r2, r2)),
                             __dmul_rn(2.0, d));
  const double rho2 = __dsub_rn(__dmul_rn(r1, r1), __dmul_rn(a, a));
  if (!(rho2 > 0.0)) return false;
  const double rho = __dsqrt_rn(rho2);
  double zeta[3], v[3];
  for (int c = 0; c < 3; ++c) {
    zeta[c] = __dadd_rn(p1[c], __dmul_rn(a, mu[c]));
    v[c] = __dsub_rn(x[c], zeta[c]);
  }
  const double vm = dot(v, mu);
  double t[3];
  for (int c = 0; c < 3; ++c) t[c] = __dsub_rn(v[c], __dmul_rn(vm, mu[c]));
  double nt = norm(t);
  if (!(nt > 1e-12)) {  // x on the axis: every circle point is as near
    double e[3] = {1.0, 0.0, 0.0};
    if (fabs(mu[0]) > 0.9) {
      e[0] = 0.0;
      e[1] = 1.0;
    }
    const double em = dot(e, mu);
    for (int c = 0; c < 3; ++c) t[c] = __dsub_rn(e[c], __dmul_rn(em, mu[c]));
    nt = norm(t);
  }
  for (int c = 0; c < 3; ++c) {
    const double step = __ddiv_rn(__dmul_rn(rho, t[c]), nt);
    out[c] = __dadd_rn(zeta[c], step);
    out[3 + c] = __dsub_rn(zeta[c], step);
  }
  return true;
}

// the two points shared by three spheres (trilateration in the frame of the
// first two centres); false when there are none
__device__ inline bool triple_points(const double* p1, double r1, const double* p2, double r2, const double* p3,
                                     double r3, double* out) {
  double ex[3] = {__dsub_rn(p2[0], p1[0]), __dsub_rn(p2[1], p1[1]), __dsub_rn(p2[2], p1[2])};
  const double d = norm(ex);
  if (!(d > 1e-12)) return false;
  for (int c = 0; c < 3; ++c) ex[c] = __ddiv_rn(ex[c], d);
  const double t13[3] = {__dsub_rn(p3[0], p1[0]), __dsub_rn(p3[1], p1[1]), __dsub_rn(p3[2], p1[2])};
  const double i = dot(ex, t13);
  double ey[3];
  for (int c = 0; c < 3; ++c) ey[c] = __dsub_rn(t13[c], __dmul_rn(i, ex[c]));
  const double ny = norm(ey);
  if (!(ny > 1e-12)) return false;
  for (int c = 0; c < 3; ++c) ey[c] = __ddiv_rn(ey[c], ny);
  const double ez[3] = {__dsub_rn(__dmul_rn(ex[1], ey[2]), __dmul_rn(ex[2], ey[1])),
                        __dsub_rn(__dmul_rn(ex[2], ey[0]), __dmul_rn(ex[0], ey[2])),
                        __dsub_rn(__dmul_rn(ex[0], ey[1]), __dmul_rn(ex[1], ey[0]))};
  const double j = dot(ey, t13);
  const double r1s = __dmul_rn(r1, r1);
  const double X = __ddiv_rn(__dadd_rn(__dsub_rn(r1s, __dmul_rn(r2, r2)), __dmul_rn(d, d)), __dmul_rn(2.0, d));
  const double Y = __dsub_rn(
      __ddiv_rn(__dadd_rn(__dadd_rn(__dsub_rn(r1s, __dmul_rn(r3, r3)), __dmul_rn(i, i)), __dmul_rn(j, j)),
                __dmul_rn(2.0, j)),
      __dmul_rn(__ddiv_rn(i, j), X));
  const double z2 = __dsub_rn(__dsub_rn(r1s, __dmul_rn(X, X)), __dmul_rn(Y, Y));
  if (z2 < 0.0) return false;
  const double Z = __dsqrt_rn(z2);
  for (int c = 0; c < 3; ++c) {
    const double base = __dadd_rn(__dadd_rn(p1[c], __dmul_rn(X, ex[c])), __dmul_rn(Y, ey[c]));
    out[c] = __dadd_rn(base, __dmul_rn(Z, ez[c]));
    out[3 + c] = __dsub_rn(base, __dmul_rn(Z, ez[c]));
  }
  return true;
}

// N_i of sphere i (input index) into meet[0, kMaxMeet), gathered by a walk
// over the hierarchy: a ball of a node with centre C and radius bound w can
// meet sphere i only if |p_i - C| < r_i + w.  Returns the count, or -1 when
// more than kMaxMeet balls meet the sphere.
__device__ inline int gather_meet(const QueryArgs& a, int i, int* meet) {
  const D4 P = a.sph64[i];
  const double ri = fabs(P.w);
  int nn = 0;
  const float x32 = float(P.x), y32 = float(P.y), z32 = float(P.z), ax = tangent::amax3(x32, y32, z32);
  const float ri32 = tangent::f_up(ri);
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
      const int64_t b = idx * kLeaf, e = tangent::imin64(b + kLeaf, a.n);
      for (int64_t j = b; j < e; ++j) {
        const int k = a.sid[j];
        if (k == i) continue;
        const D4 Q = a.sph64[k];
        const double rho = __dsub_rn(fabs(Q.w), a.tol);
        if (!(rho > 0.0)) continue;
        const double d = __dsqrt_rn(ex_d2(P.x, P.y, P.z, Q.x, Q.y, Q.z));
        if (!(fabs(__dsub_rn(d, ri)) < rho)) continue;
        if (nn == kMaxMeet) return -1;
        meet[nn++] = k;
      }
    } else {
      const int64_t cb = idx * kFan, ce = tangent::imin64(cb + kFan, T.count[lev - 1]);
      const int64_t off = T.offset[lev - 1];
      for (int64_t c = cb; c < ce; ++c) {
        const float4 B = T.na[off + c];
        if (!(B.w > 0.f)) continue;
        const float dC = tangent::dist32(x32, y32, z32, B);
        if (dC - tangent::err32(ax, B, dC, B.w + ri32) < B.w + ri32) stack[sp++] = pack_node(lev - 1, c);
      }
    }
  }
  return nn;
}

// Does one of the test points handled by `lane` of `nlanes` lie outside every
// ball but the ones it was built from?  The lane takes the circles of
// meet[c] with c = lane mod nlanes and the pairs whose running number is
// lane mod nlanes; it stops early once *found (another lane's success, may
// be null) is set.  Which lane finds a point does not matter: sphere i is
// uncovered when any lane does.
__device__ inline bool lane_candidates(const QueryArgs& a, int i, const int* meet, int nn, int lane, int nlanes,
                                       const volatile int* found) {
  const D4 P = a.sph64[i];
  const double pi[3] = {P.x, P.y, P.z};
  const double ri = fabs(P.w);
  const double e_ref[3] = {0.36, 0.48, 0.8};
  double ref[3];
  for (int c = 0; c < 3; ++c) ref[c] = __dadd_rn(pi[c], __dmul_rn(__dadd_rn(ri, 1.0), e_ref[c]));
  double pts[6];
  int64_t pair = 0;
  for (int u = 0; u < nn; ++u) {
    if (found && *found) return false;
    const int k = meet[u];
    const D4 Q = a.sph64[k];
    const double pk[3] = {Q.x, Q.y, Q.z};
    const double rk = __dsub_rn(fabs(Q.w), a.tol);
    if (u % nlanes == lane && circle_points(pi, ri, pk, rk, ref, pts)) {
      if (tangent::covered_except(a, pts[0], pts[1], pts[2], i, k, -1) < 0) return true;
      if (tangent::covered_except(a, pts[3], pts[4], pts[5], i, k, -1) < 0) return true;
    }
    for (int v = u + 1; v < nn; ++v, ++pair) {
      if (pair % nlanes != lane) continue;
      if (found && *found) return false;
      const int m = meet[v];
      const D4 R = a.sph64[m];
      const double pm[3] = {R.x, R.y, R.z};
      const double rm = __dsub_rn(fabs(R.w), a.tol);
      // the oracle takes the pair in increasing index order
      const bool km = k < m;
      if (triple_points(pi, ri, km ? pk : pm, km ? rk : rm, km ? pm : pk, km ? rm : rk, pts)) {
        if (tangent::covered_except(a, pts[0], pts[1], pts[2], i, k, m) < 0) return true;
        if (tangent::covered_except(a, pts[3], pts[4], pts[5], i, k, m) < 0) return true;
      }
    }
  }
  return false;
}

// The cases decided before any test point: 1 for a zero sample outside the
// other balls or a sphere no ball meets, 0 for a covered zero sample, 2 for
// more than kMaxMeet meeting balls; -1 when the test points decide.
__device__ inline int trivial_case(const QueryArgs& a, int i, int nn) {
  const D4 P = a.sph64[i];
  if (fabs(P.w) == 0.0) return tangent::covered_except(a, P.x, P.y, P.z, i, -1, -1) < 0 ? 1 : 0;
  if (nn < 0) return 2;
  if (nn == 0) return 1;
  return -1;
}

// 1: sphere i (input index) keeps an uncovered point; 0: it does not;
// 2: undecided (more than kMaxMeet balls meet it).  One thread.
__device__ inline int sphere_uncovered(const QueryArgs& a, int i) {
  int meet[kMaxMeet];
  const int nn = fabs(a.sph64[i].w) == 0.0 ? 0 : gather_meet(a, i, meet);
  const int t = trivial_case(a, i, nn);
  if (t >= 0) return t;
  return lane_candidates(a, i, meet, nn, 0, 1, nullptr) ? 1 : 0;
}

}  // namespace exact
}  // namespace gfs
