// Test harness: runs device routines of the library on the CPU over a
// sphere hierarchy built here: the tangent pass (tangent_one), refining the
// oracle's plain query results in place, the scored value (scored_one, over
// survivor hierarchies built here too), the cell coverage count of the
// refinement order (cell_cover_count) and the exact uncovered test per
// sphere (sphere_uncovered).  The hierarchy has the library's layout (implicit 8-ary
// tree over sorted items) with bounding balls computed directly in FP64 and
// rounded outwards to FP32, so every bound the routines rely on holds.
// Item order: Morton order of the FP32 centres (order_seed = 0, as the
// library sorts) or a seeded shuffle (other seeds: loose, overlapping nodes).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <random>
#include <utility>
#include <vector>

#include "gfs_exact.cuh"
#include "gfs_order.cuh"
#include "gfs_scored.cuh"

using namespace gfs;

namespace {

float round_out(double v) {  // an FP32 value >= v
  if (!(v > -INFINITY)) return -INFINITY;
  float f = float(v);
  if (double(f) < v) f = std::nextafter(f, INFINITY);
  return f * (f > 0 ? 1.000001f : 0.999999f) + 1e-7f;
}

struct HostTree {
  std::vector<D4> sph;
  std::vector<float4> sph32;  // sorted FP32 copies, as the library stores them
  std::vector<int> sid;
  std::vector<float4> na, nb, nf, lo, hi;
  Tree T{};
};

// the hierarchy over (p, s) in the library's layout; false if too deep
bool build_tree(const double* p, const double* s, int64_t n, unsigned order_seed, HostTree& H) {
  H.sph.resize(n);
  for (int64_t i = 0; i < n; ++i) H.sph[i] = D4{p[3 * i], p[3 * i + 1], p[3 * i + 2], s[i]};
  H.sid.resize(n);
  for (int64_t i = 0; i < n; ++i) H.sid[i] = int(i);
  if (order_seed == 0) {
    std::vector<uint32_t> key(n);
    for (int64_t i = 0; i < n; ++i) key[i] = morton3(float(p[3 * i]), float(p[3 * i + 1]), float(p[3 * i + 2]));
    std::stable_sort(H.sid.begin(), H.sid.end(), [&](int a, int b) { return key[a] < key[b]; });
  } else {
    std::mt19937 rng(order_seed);
    std::shuffle(H.sid.begin(), H.sid.end(), rng);
  }
  H.sph32.resize(n);
  for (int64_t j = 0; j < n; ++j) {
    const D4& P = H.sph[H.sid[j]];
    float w = float(P.w);
    if (w == 0.f && P.w != 0.0) w = std::copysign(1.4e-45f, float(P.w));  // keep the sign class
    H.sph32[j] = float4{float(P.x), float(P.y), float(P.z), w};
  }
  Tree& T = H.T;
  T.nitems = n;
  int64_t cnt = (n + kLeaf - 1) / kLeaf, total = 0;
  int L = 0;
  while (true) {
    if (L >= kMaxLevels) return false;
    T.count[L] = cnt;
    T.offset[L] = total;
    total += cnt;
    ++L;
    if (cnt <= kFan) break;
    cnt = (cnt + kFan - 1) / kFan;
  }
  T.nlevels = L;
  H.na.resize(total);
  H.nb.resize(total);
  H.nf.resize(total);
  H.lo.resize(total);
  H.hi.resize(total);
  const std::vector<D4>& sph = H.sph;
  const std::vector<int>& sid = H.sid;
  int64_t span = kLeaf;
  for (int l = 0; l < L; ++l, span *= kFan) {
    for (int64_t j = 0; j < T.count[l]; ++j) {
      const int64_t b = j * span, e = std::min<int64_t>(b + span, n);
      double cx = 0, cy = 0, cz = 0;
      for (int64_t t = b; t < e; ++t) {
        cx += sph[sid[t]].x;
        cy += sph[sid[t]].y;
        cz += sph[sid[t]].z;
      }
      const float4 C{float(cx / double(e - b)), float(cy / double(e - b)), float(cz / double(e - b)), 0};
      double wp = -INFINITY, wn = -INFINITY, w0 = 0, wf = -INFINITY;
      float4 L4{INFINITY, INFINITY, INFINITY, 0}, H4{-INFINITY, -INFINITY, -INFINITY, 0};
      for (int64_t t = b; t < e; ++t) {
        const D4& P = sph[sid[t]];
        const double d = std::sqrt((P.x - C.x) * (P.x - C.x) + (P.y - C.y) * (P.y - C.y) + (P.z - C.z) * (P.z - C.z));
        const double r = std::fabs(P.w);
        if (P.w > 0) wp = std::max(wp, d + r);
        if (P.w < 0) wn = std::max(wn, d + r);
        w0 = std::max(w0, d);
        wf = std::max(wf, d - r);
        L4 = float4{std::min(L4.x, std::nextafter(float(P.x), -INFINITY)),
                    std::min(L4.y, std::nextafter(float(P.y), -INFINITY)),
                    std::min(L4.z, std::nextafter(float(P.z), -INFINITY)), 0};
        H4 = float4{std::max(H4.x, std::nextafter(float(P.x), INFINITY)),
                    std::max(H4.y, std::nextafter(float(P.y), INFINITY)),
                    std::max(H4.z, std::nextafter(float(P.z), INFINITY)), 0};
      }
      const int64_t k = T.offset[l] + j;
      H.na[k] = float4{C.x, C.y, C.z, round_out(std::max(wp, wn))};
      H.nb[k] = float4{round_out(wp), round_out(wn), round_out(w0), 0};
      H.nf[k] = float4{C.x, C.y, C.z, round_out(wf)};
      H.lo[k] = L4;
      H.hi[k] = H4;
    }
  }
  T.na = H.na.data();
  T.nb = H.nb.data();
  T.nf = H.nf.data();
  T.lo = H.lo.data();
  T.hi = H.hi.data();
  return true;
}

QueryArgs args_for(const HostTree& H, int64_t n, double tol) {
  QueryArgs a{};
  a.sph = H.sph32.data();
  a.sid = H.sid.data();
  a.sph64 = H.sph.data();
  a.st = H.T;
  a.n = n;
  a.tol = tol;
  return a;
}

}  // namespace

extern "C" int tangent_host(const double* p, const double* s, int64_t n, const double* U, int K, double tol,
                            int clamp_opp, int box_cull, const double* x, int64_t m, double* value,
                            int64_t* argmin, uint16_t* flags, unsigned order_seed) {
  HostTree H;
  if (!build_tree(p, s, n, order_seed, H)) return -1;
  QueryArgs a = args_for(H, n, tol);
  a.U64 = U;
  a.K = K;
  a.KS = K + 1;
  a.clamp_opp = clamp_opp;
  a.x64 = x;
  a.m = m;
  a.s64_out = value;
  a.arg_out = argmin;
  a.fl_out = flags;
  for (int64_t q = 0; q < m; ++q) tangent::tangent_one(a, box_cull, q);
  return 0;
}

extern "C" int coverage_host(const double* p, const double* s, int64_t n, double tol, const int32_t* cells,
                             int64_t ncells, const double* origin, double h, int sub, uint32_t* counts,
                             unsigned order_seed) {
  HostTree H;
  if (!build_tree(p, s, n, order_seed, H)) return -1;
  const QueryArgs a = args_for(H, n, tol);
  for (int64_t c = 0; c < ncells; ++c) {
    counts[c] = order::cell_cover_count(a, cells + 3 * c, origin[0], origin[1], origin[2], h, sub, 0, 1);
    // the warp kernel's split: lane l takes the points l, l + 32, ...
    unsigned warp = 0;
    for (int lane = 0; lane < 32; ++lane)
      warp += order::cell_cover_count(a, cells + 3 * c, origin[0], origin[1], origin[2], h, sub, lane, 32);
    if (warp != counts[c]) return -2;
  }
  return 0;
}

extern "C" int uncovered_host(const double* p, const double* s, int64_t n, double tol, uint8_t* out,
                              double* witness, unsigned order_seed) {
  HostTree H;
  if (!build_tree(p, s, n, order_seed, H)) return -1;
  const QueryArgs a = args_for(H, n, tol);
  std::vector<int> S(exact::kMaxSet);
  std::vector<uint32_t> stack(kStack);
  for (int64_t i = 0; i < n; ++i)
    out[i] = uint8_t(exact::sphere_uncovered(a, int(i), S.data(), stack.data(), witness + 3 * i));
  return 0;
}

// uncovered intersection circles and points: the per-sphere test, then the
// intersections routine for every uncovered sphere (in hierarchy order);
// outputs unsorted, counts in cnt[0..1], status in *status
extern "C" int intersections_host(const double* p, const double* s, int64_t n, double tol, int64_t cap_c,
                                  int64_t* circ, int64_t cap_p, int64_t* quad, double* pts,
                                  unsigned long long* cnt, unsigned* status, unsigned order_seed) {
  HostTree H;
  if (!build_tree(p, s, n, order_seed, H)) return -1;
  const QueryArgs a = args_for(H, n, tol);
  std::vector<int> S(exact::kMaxSet);
  std::vector<uint32_t> stacks(3 * kStack);
  std::vector<uint8_t> uncov(size_t(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) uncov[i] = uint8_t(exact::sphere_uncovered(a, int(i), S.data(), stacks.data(), nullptr));
  cnt[0] = cnt[1] = 0;
  *status = 0;
  const exact::UDOut o{cnt, cap_c, cap_p, circ, quad, pts, status};
  // the pair list of the first kernel, then one circle at a time
  std::vector<std::pair<int, int>> pairs;
  for (int64_t u = 0; u < n; ++u) {
    const int i = a.sid[u];
    if (uncov[i] != 0)
      exact::sphere_pairs(a, i, uncov.data(), stacks.data() + 2 * kStack, [&](int j) { pairs.emplace_back(i, j); });
  }
  for (const auto& pr : pairs) exact::circle_intersections(a, pr.first, pr.second, S.data(), stacks.data(), o);
  return 0;
}

// exact minimum valid radius at each point for its sign: the uncovered
// circles and points as above, then the three candidate sets in turn
extern "C" int exact_rmin_host(const double* p, const double* s, int64_t n, double tol, int box_cull, const double* x,
                               const int8_t* sigma, int64_t m, double* out, unsigned order_seed) {
  HostTree H;
  if (!build_tree(p, s, n, order_seed, H)) return -1;
  const QueryArgs a = args_for(H, n, tol);
  std::vector<int> S(exact::kMaxSet);
  std::vector<uint32_t> stacks(3 * kStack);
  std::vector<uint8_t> uncov(size_t(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) uncov[i] = uint8_t(exact::sphere_uncovered(a, int(i), S.data(), stacks.data(), nullptr));
  const int64_t cap = 1 << 20;
  std::vector<int64_t> circ(2 * cap), quad(4 * cap);
  std::vector<double> pts(3 * cap);
  unsigned long long cnt[2] = {0, 0};
  unsigned status = 0;
  const exact::UDOut o{cnt, cap, cap, circ.data(), quad.data(), pts.data(), &status};
  for (int64_t u = 0; u < n; ++u) {
    const int i = a.sid[u];
    if (uncov[i] != 0)
      exact::sphere_pairs(a, i, uncov.data(), stacks.data() + 2 * kStack,
                          [&](int j) { exact::circle_intersections(a, i, j, S.data(), stacks.data(), o); });
  }
  if (cnt[0] > (unsigned long long)cap || cnt[1] > (unsigned long long)cap) return -2;
  const exact::UDLists L{quad.data(), pts.data(), int64_t(cnt[1]), circ.data(), int64_t(cnt[0])};
  for (int64_t q = 0; q < m; ++q) {
    double best = INFINITY;
    for (int phase = 0; phase < 3; ++phase)
      best = exact::rmin_phase(a, box_cull, L, x + 3 * q, sigma[q], phase, 0, 1, best, stacks.data());
    out[q] = best;
  }
  return 0;
}

// q* of each point from the argmin and flags (argmin_point)
extern "C" int points_host(const double* p, const double* s, int64_t n, const double* U, int K, const double* x,
                           int64_t m, const int64_t* argmin, const uint16_t* flags, double* out) {
  HostTree H;
  if (!build_tree(p, s, n, 0, H)) return -1;
  QueryArgs a = args_for(H, n, 1e-6);
  a.U64 = U;
  a.K = K;
  a.KS = K + 1;
  for (int64_t q = 0; q < m; ++q)
    tangent::argmin_point(a, x[3 * q], x[3 * q + 1], x[3 * q + 2], flags[q] & 15, argmin[q], out + 3 * q);
  return 0;
}

namespace {

// A survivor hierarchy in the library's layout: FP32 items (x, y, z, id
// bits) in Morton order, leaves of kLeaf, boxes over the FP32 positions
// widened by one ulp.
struct HostPoints {
  std::vector<float4> items, lo, hi;
  Tree T{};
};

void build_points(const std::vector<float4>& in, HostPoints& H) {
  const int64_t n = int64_t(in.size());
  std::vector<int64_t> ord(n);
  for (int64_t i = 0; i < n; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) {
    return morton3(in[a].x, in[a].y, in[a].z) < morton3(in[b].x, in[b].y, in[b].z);
  });
  H.items.resize(n);
  for (int64_t i = 0; i < n; ++i) H.items[i] = in[ord[i]];
  Tree& T = H.T;
  T = Tree{};
  T.nitems = n;
  if (n == 0) return;
  int64_t cnt = (n + kLeaf - 1) / kLeaf, total = 0;
  int L = 0;
  while (true) {
    T.count[L] = cnt;
    T.offset[L] = total;
    total += cnt;
    ++L;
    if (cnt <= kFan || L == kMaxLevels) break;
    cnt = (cnt + kFan - 1) / kFan;
  }
  T.nlevels = L;
  H.lo.resize(total);
  H.hi.resize(total);
  int64_t span = kLeaf;
  for (int l = 0; l < L; ++l, span *= kFan)
    for (int64_t j = 0; j < T.count[l]; ++j) {
      const int64_t b = j * span, e = std::min<int64_t>(b + span, n);
      float4 L4{INFINITY, INFINITY, INFINITY, 0}, H4{-INFINITY, -INFINITY, -INFINITY, 0};
      for (int64_t t = b; t < e; ++t) {
        const float4& P = H.items[t];
        L4 = float4{std::min(L4.x, std::nextafter(P.x, -INFINITY)), std::min(L4.y, std::nextafter(P.y, -INFINITY)),
                    std::min(L4.z, std::nextafter(P.z, -INFINITY)), 0};
        H4 = float4{std::max(H4.x, std::nextafter(P.x, INFINITY)), std::max(H4.y, std::nextafter(P.y, INFINITY)),
                    std::max(H4.z, std::nextafter(P.z, INFINITY)), 0};
      }
      H.lo[T.offset[l] + j] = L4;
      H.hi[T.offset[l] + j] = H4;
    }
  T.lo = H.lo.data();
  T.hi = H.hi.data();
  T.na = T.nb = T.nf = nullptr;
}

}  // namespace

// Scored value (scored_one) refining the oracle's plain query results in
// place; survivors given as the oracle's list (ids g, their spheres, FP64
// positions).
extern "C" int scored_host(const double* p, const double* s, int64_t n, const double* U, int K, double tol,
                           int box_cull, const int64_t* sg, const int64_t* ssph, const double* sq, int64_t ns,
                           const double* x, int64_t m, double* value, int64_t* argmin, uint16_t* flags,
                           unsigned order_seed) {
  HostTree H;
  if (!build_tree(p, s, n, order_seed, H)) return -1;
  QueryArgs a = args_for(H, n, tol);
  a.U64 = U;
  a.K = K;
  a.KS = K + 1;
  a.clamp_opp = 1;
  a.x64 = x;
  a.m = m;
  a.s64_out = value;
  a.arg_out = argmin;
  a.fl_out = flags;
  // survivor lists per class (a zero sample's survivors in both)
  std::vector<float4> cls[2];
  for (int64_t g = 0; g < ns; ++g) {
    const float4 it{float(sq[3 * g]), float(sq[3 * g + 1]), float(sq[3 * g + 2]), __uint_as_float(uint32_t(sg[g]))};
    const double sv = s[ssph[g]];
    if (!(sv < 0.0)) cls[0].push_back(it);
    if (!(sv > 0.0)) cls[1].push_back(it);
  }
  HostPoints V[2];
  for (int k = 0; k < 2; ++k) {
    build_points(cls[k], V[k]);
    a.surv[k] = V[k].items.data();
    a.vt[k] = V[k].T;
  }
  // the candidate error bound of the build constants (FP32 vs FP64 survivor
  // positions), as the library derives it from the data bounds
  double A = 1.0, R = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    A = std::max(A, std::max(std::fabs(p[3 * i]), std::max(std::fabs(p[3 * i + 1]), std::fabs(p[3 * i + 2]))));
    R = std::max(R, std::fabs(s[i]));
  }
  BuildConsts bc{};
  bc.eq = float(5.9604645e-8 * (2.0 * A + 2.0 * R + 0.01) * 1.01 + 1e-12);
  a.bc = &bc;
  // per-sphere sorted survivor ids
  std::vector<uint32_t> ids(ns);
  for (int64_t g = 0; g < ns; ++g) ids[g] = uint32_t(sg[g]);
  std::sort(ids.begin(), ids.end());
  std::vector<int64_t> off(n + 1);
  for (int64_t i = 0; i <= n; ++i)
    off[i] = std::lower_bound(ids.begin(), ids.end(), uint32_t(uint64_t(i) * uint64_t(K + 1))) - ids.begin();
  unsigned status = 0;
  for (int64_t q = 0; q < m; ++q) scored::scored_one(a, box_cull, ids.data(), off.data(), q, &status);
  return status ? -3 : 0;
}
