// Exact uncovered test per sphere (Prop. 1 (ii)), device routines.
//
// Sphere i keeps a point outside every other ball shrunk by tol exactly when
// one of these test points is outside every ball but i and the spheres it
// was built from (N_i: the spheres k != i with rho_k = |s_k| - tol > 0 whose
// shrunk open ball meets sphere i, | |p_i - p_k| - |s_i| | < rho_k):
//  - any point, when N_i is empty;
//  - the two points of each circle C_k = S_i with the sphere (p_k, rho_k)
//    nearest and farthest from the reference point p_i + (|s_i| + 1) e,
//    e = (0.36, 0.48, 0.8) -- an uncovered circle is wholly uncovered;
//  - the two points shared by S_i and the spheres (p_k, rho_k),
//    (p_m, rho_m), k < m in N_i -- the ends of the uncovered arcs of a
//    partly covered circle (the D points of Def. 1).
// The uncovered set, if not empty, is a closed proper subset of the sphere,
// so its boundary holds one of these points.  The argument holds for the
// caps of any subset S of N_i: if every test point built from S lies in the
// cap of another member of S, the caps of S cover the sphere.
//
// So instead of all |N_i|^2 test points (|N_i| reaches millions for a deep
// sphere of a 128^3 grid) the routine grows a certificate S: it starts from
// the balls that hold six probe points of the sphere, and tests the points
// of S's circles and pairs in the order the members joined.  A point that a
// member of S holds is covered; otherwise a walk over the sphere hierarchy
// tests it against every ball but the ones it was built from: if none holds
// it, it is an uncovered test point of N_i (the same point and the same test
// as the full enumeration) and the sphere is uncovered; if a ball of N_i
// holds it, that ball joins S.  When every point of S is covered, the sphere
// is covered.  A sample with s_i = 0 is the point p_i.  Every value is
// computed in FP64 with each operation rounded on its own, in the order
// written (the circle and triple constructions of the exact grow-to points),
// so the decisions are those of a plain IEEE-754 evaluation.
#pragma once

#include "gfs_exact.h"
#include "gfs_tangent.cuh"

namespace gfs {
namespace exact {

constexpr int kMaxSet = 512;  // members of one sphere's certificate

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

// Is sphere k in N_i (same arithmetic as the full enumeration)?
__device__ __forceinline__ bool meets(const QueryArgs& a, const D4& P, double ri, int k) {
  const D4 Q = a.sph64[k];
  const double rho = __dsub_rn(fabs(Q.w), a.tol);
  if (!(rho > 0.0)) return false;
  const double d = __dsqrt_rn(ex_d2(P.x, P.y, P.z, Q.x, Q.y, Q.z));
  return fabs(__dsub_rn(d, ri)) < rho;
}

// The first ball of N_i in hierarchy order, or -1 when N_i is empty: a ball
// of a node with centre C and radius bound w can meet sphere i only if
// |p_i - C| < r_i + w.
__device__ inline int first_member(const QueryArgs& a, int i, uint32_t* stack) {
  const D4 P = a.sph64[i];
  const double ri = fabs(P.w);
  const float x32 = float(P.x), y32 = float(P.y), z32 = float(P.z), ax = tangent::amax3(x32, y32, z32);
  const float ri32 = tangent::f_up(ri);
  const Tree& T = a.st;
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
        if (k != i && meets(a, P, ri, k)) return k;
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
  return -1;
}

// The test points of certificate entry (n, u), u <= n: for u < n the two
// points S_i shares with the shrunk spheres of members S[u] and S[n] (taken
// in increasing index order, as the full enumeration does), for u = n the
// two points of S[n]'s circle nearest to and farthest from ref.  k and m
// receive the members the points were built from (m = -1 for a circle).
__device__ inline bool entry_points(const QueryArgs& a, const double* pi, double ri, const double* ref, const int* S,
                                    int n, int u, double* pts, int& k, int& m) {
  k = S[n];
  m = u < n ? S[u] : -1;
  const D4 Q = a.sph64[k];
  const double pk[3] = {Q.x, Q.y, Q.z};
  const double rk = __dsub_rn(fabs(Q.w), a.tol);
  if (m < 0) return circle_points(pi, ri, pk, rk, ref, pts);
  const D4 R = a.sph64[m];
  const double pm[3] = {R.x, R.y, R.z};
  const double rm = __dsub_rn(fabs(R.w), a.tol);
  const bool km = k < m;
  return triple_points(pi, ri, km ? pk : pm, km ? rk : rm, km ? pm : pk, km ? rm : rk, pts);
}

// Is t held by a member of S[0, ns) other than k and m?  last: the member
// that held the previous point (tested first; updated).
__device__ inline bool held_by_member(const QueryArgs& a, const double* t, const int* S, int ns, int k, int m,
                                      int& last) {
  if (last >= 0) {
    const int o = S[last];
    if (o != k && o != m && ex_cov(t[0], t[1], t[2], a.sph64[o], a.tol)) return true;
  }
  for (int u = 0; u < ns; ++u) {
    const int o = S[u];
    if (u == last || o == k || o == m) continue;
    if (ex_cov(t[0], t[1], t[2], a.sph64[o], a.tol)) {
      last = u;
      return true;
    }
  }
  return false;
}

// The reference point of sphere i's circles: p_i + (|s_i| + 1) e.
__device__ inline void circle_ref(const double* pi, double ri, double* ref) {
  const double e_ref[3] = {0.36, 0.48, 0.8};
  for (int c = 0; c < 3; ++c) ref[c] = __dadd_rn(pi[c], __dmul_rn(__dadd_rn(ri, 1.0), e_ref[c]));
}

// The certificate: members in the order they joined.
struct Cert {
  int* S;
  int ns;
  uint32_t* stack;  // kStack entries for the hierarchy walks
  int last;         // the member that held the latest covered point (tested first)
};

// Add ball j (found to hold a point of sphere i) to the certificate when it
// is in N_i and not yet a member.  False when the certificate is full.
__device__ inline bool join(const QueryArgs& a, const D4& P, double ri, int j, Cert& C) {
  for (int u = 0; u < C.ns; ++u)
    if (C.S[u] == j) return true;
  if (!meets(a, P, ri, j)) return true;  // holds the point, but no circle of N_i
  if (C.ns == kMaxSet) return false;
  C.S[C.ns++] = j;
  return true;
}

// Test point t built from i, k and m (m = -1 for a circle point): 1 when no
// ball but those holds it; 0 when one does (joining the certificate if it is
// not a member); -1 when the certificate is full.
__device__ inline int test_point(const QueryArgs& a, const D4& P, double ri, int i, const double* t, int k, int m,
                                 Cert& C) {
  // neighbouring test points are mostly held by the same member
  if (held_by_member(a, t, C.S, C.ns, k, m, C.last)) return 0;
  const int j = tangent::covered_except_on(C.stack, a, t[0], t[1], t[2], i, k, m);
  if (j < 0) return 1;
  return join(a, P, ri, j, C) ? 0 : -1;
}

// 1: sphere i (input index) keeps an uncovered point (witness, when not
// null, receives it: a test point, or p_i for a zero sample); 0: every point
// is covered; 2: undecided (the certificate outgrew kMaxSet members).
// S: kMaxSet entries; stack: kStack entries.  One thread; the GPU kernel
// runs the same steps with the 32 lanes of a warp sharing one certificate.
__device__ inline int sphere_uncovered(const QueryArgs& a, int i, int* S, uint32_t* stack, double* witness) {
  const D4 P = a.sph64[i];
  const double pi[3] = {P.x, P.y, P.z};
  const double ri = fabs(P.w);
  if (ri == 0.0) {
    if (tangent::covered_except_on(stack, a, P.x, P.y, P.z, i, -1, -1) >= 0) return 0;
    if (witness)
      for (int c = 0; c < 3; ++c) witness[c] = pi[c];
    return 1;
  }
  Cert C{S, 0, stack, -1};
  // probe points p_i +- r_i e_c: the balls that hold them start the
  // certificate (they are not test points: an uncovered probe decides nothing)
  for (int c = 0; c < 6; ++c) {
    double t[3] = {pi[0], pi[1], pi[2]};
    t[c >> 1] = __dadd_rn(pi[c >> 1], (c & 1) ? -ri : ri);
    const int j = tangent::covered_except_on(stack, a, t[0], t[1], t[2], i, -1, -1);
    if (j >= 0) join(a, P, ri, j, C);
  }
  if (C.ns == 0) {
    const int k = first_member(a, i, stack);
    if (k < 0) {  // N_i is empty: every point is uncovered
      if (witness)
        for (int c = 0; c < 3; ++c) witness[c] = c == 0 ? __dadd_rn(pi[0], ri) : pi[c];
      return 1;
    }
    S[C.ns++] = k;
  }
  double ref[3];
  circle_ref(pi, ri, ref);
  double pts[6];
  for (int n = 0; n < C.ns; ++n) {
    // the pairs of member n with the members before it, then its circle
    for (int u = 0; u <= n; ++u) {
      int k, m;
      if (!entry_points(a, pi, ri, ref, S, n, u, pts, k, m)) continue;
      for (int h = 0; h < 2; ++h) {
        const int r = test_point(a, P, ri, i, pts + 3 * h, k, m, C);
        if (r < 0) return 2;
        if (r == 1) {
          if (witness)
            for (int c = 0; c < 3; ++c) witness[c] = pts[3 * h + c];
          return 1;
        }
      }
    }
  }
  return 0;
}

// ---------------------------------------------------------------------------
// Uncovered intersection circles and points (Def. 1 U and the circles of D;
// the U and D precomputation of Sec. 4.1).
//
// For spheres S_i = (p_i, |s_i|), |s_i| > 0, i < j: the circle C_ij where
// S_i and S_j cut is uncovered when some point of it lies in no ball but i
// and j shrunk by tol.  Its uncovered part is closed; if it is not empty
// and not the whole circle its ends lie where C_ij crosses a shrunk sphere
// (p_m, |s_m| - tol).  The test points are C_ij's points nearest to and
// farthest from p_i + (|s_i| + 1) e and its crossings with every such
// sphere, each tested against every ball but i, j and the m it was built
// from.  As for a whole sphere, a circle grows a certificate M instead of
// taking every m: the balls that hold the two extreme points start it, the
// crossings of its members are tested against M and then against all
// balls, a ball that holds a crossing joins M, and a point that no ball
// holds decides "uncovered" (the full enumeration's own decision on one of
// its points).  A ball that holds a point but whose shrunk sphere does not
// cross the circle holds the whole circle: covered.  The uncovered points U
// on an uncovered circle C_ij are the points shared by S_i, S_j and S_m,
// m > j, in no ball but i, j, m shrunk by tol; a covered circle has none,
// and neither has a circle on a sphere that the other balls cover, so the
// kernel starts from the uncovered spheres only.
// ---------------------------------------------------------------------------

// Circle C_ij (extreme points q): 1 uncovered, 0 covered, -1 certificate full.
// M: kMaxSet entries; stack: kStack entries.
__device__ inline int circle_uncovered(const QueryArgs& a, int i, int j, const double* pi, double ri,
                                       const double* pj, double rj, const double* q, int* M, uint32_t* stack) {
  int nm = 0, last = -1;
  // ball b holds a point of C_ij: joins M; 2 when it holds the whole circle
  auto join = [&](int b) -> int {
    for (int u = 0; u < nm; ++u)
      if (M[u] == b) return 1;
    const D4 B = a.sph64[b];
    const double pb[3] = {B.x, B.y, B.z};
    double t[6];
    if (!triple_points(pi, ri, pj, rj, pb, __dsub_rn(fabs(B.w), a.tol), t)) return 2;
    if (nm == kMaxSet) return -1;
    M[nm++] = b;
    return 1;
  };
  // 1: no ball holds t; 0: held; 2: held by a ball that holds the circle; -1: full
  auto test = [&](const double* t, int m) -> int {
    if (last >= 0 && M[last] != m && ex_cov(t[0], t[1], t[2], a.sph64[M[last]], a.tol)) return 0;
    for (int u = 0; u < nm; ++u) {
      const int o = M[u];
      if (u == last || o == m) continue;
      if (ex_cov(t[0], t[1], t[2], a.sph64[o], a.tol)) {
        last = u;
        return 0;
      }
    }
    const int b = tangent::covered_except_on(stack, a, t[0], t[1], t[2], i, j, m);
    if (b < 0) return 1;
    const int r = join(b);
    return r == 1 ? 0 : r;
  };
  for (int h = 0; h < 2; ++h) {
    const int r = test(q + 3 * h, -1);
    if (r == 1 || r == -1) return r;
    if (r == 2) return 0;
  }
  for (int n = 0; n < nm; ++n) {
    const int m = M[n];
    const D4 B = a.sph64[m];
    const double pm[3] = {B.x, B.y, B.z};
    double t[6];
    if (!triple_points(pi, ri, pj, rj, pm, __dsub_rn(fabs(B.w), a.tol), t)) continue;
    for (int h = 0; h < 2; ++h) {
      const int r = test(t + 3 * h, m);
      if (r == 1 || r == -1) return r;
      if (r == 2) return 0;
    }
  }
  return 0;
}

__device__ inline void ud_record_circle(const UDOut& o, int i, int j) {
  const unsigned long long k = atomicAdd(o.cnt, 1ull);
  if (k < (unsigned long long)o.cap_c) {
    o.circ[2 * k] = i;
    o.circ[2 * k + 1] = j;
  }
}

__device__ inline void ud_record_point(const UDOut& o, int i, int j, int m, int side, const double* t) {
  const unsigned long long k = atomicAdd(o.cnt + 1, 1ull);
  if (k < (unsigned long long)o.cap_p) {
    o.quad[4 * k] = i;
    o.quad[4 * k + 1] = j;
    o.quad[4 * k + 2] = m;
    o.quad[4 * k + 3] = side;
    for (int c = 0; c < 3; ++c) o.pts[3 * k + c] = t[c];
  }
}

// The uncovered points of circle C_ij: spheres m > j whose sphere may cross
// the circle (centre zeta, radius rc): ||p_m - zeta| - r_m| <= rc, node
// bound |C - zeta| - w <= rc.
__device__ inline void circle_points_u(const QueryArgs& a, int i, int j, const double* pi, double ri,
                                       const double* pj, double rj, uint32_t* stack, uint32_t* cstack,
                                       const UDOut& o) {
  double mu[3] = {__dsub_rn(pj[0], pi[0]), __dsub_rn(pj[1], pi[1]), __dsub_rn(pj[2], pi[2])};
  const double d = norm(mu);
  const double al = (d * d + ri * ri - rj * rj) / (2.0 * d);
  const double rc = sqrt(fmax(ri * ri - al * al, 0.0));
  double zeta[3];
  for (int c = 0; c < 3; ++c) zeta[c] = pi[c] + al * mu[c] / d;
  const float zx = float(zeta[0]), zy = float(zeta[1]), zz = float(zeta[2]);
  const float az = tangent::amax3(zx, zy, zz);
  // rounding of zeta and rc in FP64 is far below the FP32 screens' margins
  const float rc32 = tangent::f_up(rc) + 1e-6f * (1.f + az);
  const Tree& T = a.st;
  int sp = 0;
  const int top = T.nlevels - 1;
  for (int64_t u = 0; u < T.count[top]; ++u) stack[sp++] = pack_node(top, u);
  while (sp > 0) {
    const uint32_t nd = stack[--sp];
    const int lev = node_level(nd);
    const int64_t idx = node_index(nd);
    if (lev == 0) {
      const int64_t b = idx * kLeaf, e = tangent::imin64(b + kLeaf, a.n);
      for (int64_t u = b; u < e; ++u) {
        const int m = a.sid[u];
        if (m <= j) continue;
        const float4 S = a.sph[u];
        if (S.w == 0.f) continue;
        const float dm = tangent::dist32(zx, zy, zz, S), rm32 = fabsf(S.w);
        if (fabsf(dm - rm32) - tangent::err32(az, S, dm, rm32) > rc32) continue;
        const D4 Q = a.sph64[m];
        const double rm = fabs(Q.w);
        if (!(rm > 0.0)) continue;
        const double pm[3] = {Q.x, Q.y, Q.z};
        double t[6];
        if (!triple_points(pi, ri, pj, rj, pm, rm, t)) continue;
        for (int h = 0; h < 2; ++h)
          if (tangent::covered_except_on(cstack, a, t[3 * h], t[3 * h + 1], t[3 * h + 2], i, j, m) < 0)
            ud_record_point(o, i, j, m, h, t + 3 * h);
      }
    } else {
      const int64_t cb = idx * kFan, ce = tangent::imin64(cb + kFan, T.count[lev - 1]);
      const int64_t off = T.offset[lev - 1];
      for (int64_t c = cb; c < ce; ++c) {
        const float4 B = T.na[off + c];
        if (!(B.w > 0.f)) continue;
        const float dC = tangent::dist32(zx, zy, zz, B);
        if (dC - tangent::err32(az, B, dC, B.w) - B.w <= rc32) stack[sp++] = pack_node(lev - 1, c);
      }
    }
  }
}

// The circles of sphere i (input index) with the spheres after it: every
// j > i with uncov[j] != 0 whose sphere cuts sphere i in a circle (the
// construction of circle_points), passed to emit(j).  stack: kStack entries.
template <class Emit>
__device__ inline void sphere_pairs(const QueryArgs& a, int i, const uint8_t* uncov, uint32_t* stack, Emit emit) {
  const D4 P = a.sph64[i];
  const double ri = fabs(P.w);
  if (!(ri > 0.0)) return;
  const double pi[3] = {P.x, P.y, P.z};
  const double e_ref[3] = {0.36, 0.48, 0.8};
  double ref[3];
  for (int c = 0; c < 3; ++c) ref[c] = __dadd_rn(pi[c], __dmul_rn(__dadd_rn(ri, 1.0), e_ref[c]));
  const float x32 = float(P.x), y32 = float(P.y), z32 = float(P.z), ax = tangent::amax3(x32, y32, z32);
  const float ri32 = tangent::f_up(ri);
  const Tree& T = a.st;
  int sp = 0;
  const int top = T.nlevels - 1;
  for (int64_t u = 0; u < T.count[top]; ++u) stack[sp++] = pack_node(top, u);
  while (sp > 0) {
    const uint32_t nd = stack[--sp];
    const int lev = node_level(nd);
    const int64_t idx = node_index(nd);
    if (lev == 0) {
      const int64_t b = idx * kLeaf, e = tangent::imin64(b + kLeaf, a.n);
      for (int64_t u = b; u < e; ++u) {
        const int j = a.sid[u];
        if (j <= i || uncov[j] == 0) continue;
        const D4 Q = a.sph64[j];
        const double rj = fabs(Q.w);
        if (!(rj > 0.0)) continue;
        const double pj[3] = {Q.x, Q.y, Q.z};
        double q[6];
        if (circle_points(pi, ri, pj, rj, ref, q)) emit(j);
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
}

// Circle C_ij (i < j, both spheres cut in a circle): its certificate, and on
// an uncovered circle its uncovered points.  stacks: 2 kStack entries (the
// certificate's and the point walk's, the point tests'); M: kMaxSet entries.
__device__ inline void circle_intersections(const QueryArgs& a, int i, int j, int* M, uint32_t* stacks,
                                            const UDOut& o) {
  const D4 P = a.sph64[i], Q = a.sph64[j];
  const double ri = fabs(P.w), rj = fabs(Q.w);
  const double pi[3] = {P.x, P.y, P.z}, pj[3] = {Q.x, Q.y, Q.z};
  const double e_ref[3] = {0.36, 0.48, 0.8};
  double ref[3];
  for (int c = 0; c < 3; ++c) ref[c] = __dadd_rn(pi[c], __dmul_rn(__dadd_rn(ri, 1.0), e_ref[c]));
  double q[6];
  if (!circle_points(pi, ri, pj, rj, ref, q)) return;
  int r = circle_uncovered(a, i, j, pi, ri, pj, rj, q, M, stacks);
  if (r < 0) {
    atomicOr(o.status, 1u);
    r = 1;
  }
  if (r == 0) return;
  ud_record_circle(o, i, j);
  circle_points_u(a, i, j, pi, ri, pj, rj, stacks, stacks + kStack, o);
}

// ---------------------------------------------------------------------------
// Exact minimum valid radius for a known sign (Sec. 6,
// min_valid_radius_for_known_sign; Def. 1 P = T u U u D): the least distance
// from x to a grow-to point that no other ball, shrunk by tol, holds:
//  - U: the points shared by three spheres none of whose signs is opposite
//    to sigma -- the precomputed uncovered points (tested there against
//    every ball but their three);
//  - D: the points of each circle of two such spheres nearest to and
//    farthest from x -- on the precomputed uncovered circles (a circle that
//    other balls cover entirely has no uncovered point), tested against
//    every ball but the two;
//  - T: the near and far tangent points p_i -+ r_i (x - p_i)/|x - p_i| of
//    every sphere (either sign), tested against every ball but i;
// in the box when the context culls by it.  Every point and distance is
// computed in FP64 in the order written (the oracle's constructions), so
// the minimum is the oracle's bit for bit.  INFINITY when there is no
// candidate.  A point is coverage-tested only when it is nearer than the
// best so far (the minimum does not depend on the order).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int sgn64(double v) { return v > 0.0 ? 1 : (v < 0.0 ? -1 : 0); }

// Candidates lane, lane + stride, ... of each set (lane 0, stride 1: all);
// returns min(best, the nearest uncovered one).  phase: 0 U, 1 D, 2 T.
__device__ inline double rmin_phase(const QueryArgs& a, int box_cull, const UDLists& L, const double* x, int sigma,
                                    int phase, int64_t lane, int64_t stride, double best, uint32_t* stack) {
  if (phase == 0) {
    for (int64_t u = lane; u < L.np; u += stride) {
      const int64_t* qd = L.quad + 4 * u;
      if (sigma * sgn64(a.sph64[qd[0]].w) < 0 || sigma * sgn64(a.sph64[qd[1]].w) < 0 ||
          sigma * sgn64(a.sph64[qd[2]].w) < 0)
        continue;
      const double* q = L.pts + 3 * u;
      if (box_cull && !ex_inbox(q[0], q[1], q[2])) continue;
      const double dd = __dsqrt_rn(ex_d2(x[0], x[1], x[2], q[0], q[1], q[2]));
      if (dd < best) best = dd;
    }
  } else if (phase == 1) {
    for (int64_t u = lane; u < L.nc; u += stride) {
      const int i = int(L.circ[2 * u]), j = int(L.circ[2 * u + 1]);
      const D4 P = a.sph64[i], Q = a.sph64[j];
      if (sigma * sgn64(P.w) < 0 || sigma * sgn64(Q.w) < 0) continue;
      const double pi[3] = {P.x, P.y, P.z}, pj[3] = {Q.x, Q.y, Q.z};
      double q[6];
      if (!circle_points(pi, fabs(P.w), pj, fabs(Q.w), x, q)) continue;
      for (int h = 0; h < 2; ++h) {
        const double* t = q + 3 * h;
        if (box_cull && !ex_inbox(t[0], t[1], t[2])) continue;
        const double dd = __dsqrt_rn(ex_d2(x[0], x[1], x[2], t[0], t[1], t[2]));
        if (!(dd < best)) continue;
        if (tangent::covered_except_on(stack, a, t[0], t[1], t[2], i, j, -1) >= 0) continue;
        best = dd;
      }
    }
  } else {
    for (int64_t i = lane; i < a.n; i += stride) {
      const D4 P = a.sph64[i];
      const double w[3] = {__dsub_rn(x[0], P.x), __dsub_rn(x[1], P.y), __dsub_rn(x[2], P.z)};
      const double d = norm(w);
      if (!(d > 0.0)) continue;
      const double r = fabs(P.w);
      // the two points lie |d -+ r| from x (up to rounding): skip the pair
      // when both are clearly beyond the best
      const double lo = fabs(__dsub_rn(d, r));
      if (lo > best + 1e-12 * (d + r + best)) continue;
      for (int c = -1; c <= 1; c += 2) {
        const double cr = c * r;
        const double t[3] = {__dadd_rn(P.x, __ddiv_rn(__dmul_rn(cr, w[0]), d)),
                             __dadd_rn(P.y, __ddiv_rn(__dmul_rn(cr, w[1]), d)),
                             __dadd_rn(P.z, __ddiv_rn(__dmul_rn(cr, w[2]), d))};
        if (box_cull && !ex_inbox(t[0], t[1], t[2])) continue;
        const double dd = __dsqrt_rn(ex_d2(x[0], x[1], x[2], t[0], t[1], t[2]));
        if (!(dd < best)) continue;
        if (tangent::covered_except_on(stack, a, t[0], t[1], t[2], int(i), -1, -1) >= 0) continue;
        best = dd;
      }
    }
  }
  return best;
}

}  // namespace exact
}  // namespace gfs
