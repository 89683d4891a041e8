// Greedy sequential insertion (Sec. 4: every new value is consistent with
// the inputs and with all values generated before it).
//
// State between hierarchy rebuilds:
//   spheres    [0, n_static) in the sphere hierarchy, [n_static, n_total)
//              inserted since the last rebuild (scanned linearly);
//   survivors  the per-class survivor hierarchies (with a tombstone bit per
//              sorted slot) plus per-class lists of survivors added since
//              the last rebuild (with a tombstone byte each).
// One insertion step = two launches:
//   k_ins_query  -- one block evaluates the value at y_t exactly (the
//                   oracle's FP64 expressions and tie rules) with a
//                   block-parallel walk of the hierarchies (256 nodes per
//                   round), FP32 filters in front of every FP64 evaluation;
//   k_ins_update -- culls the new sphere's K candidates and its witness
//                   against every other sphere, and tombstones the survivors
//                   the new ball covers (raising LOST_WITNESS when a sphere
//                   loses its last survivor).
#include <cooperative_groups.h>

#include "gfs_internal.cuh"
#include "gfs_kernels.h"

namespace cg = cooperative_groups;

namespace gfs {

namespace {

constexpr unsigned kAll = 0xffffffffu;

__device__ __forceinline__ void surv64(const InsertArgs& a, uint32_t g, double& qx, double& qy, double& qz) {
  const uint32_t i = g / uint32_t(a.KS), k = g % uint32_t(a.KS);
  if (int(k) < a.K) {
    ex_cand(a.sph64[i], a.U64[3 * k], a.U64[3 * k + 1], a.U64[3 * k + 2], qx, qy, qz);
  } else {
    qx = a.witness64[3 * int64_t(i)];
    qy = a.witness64[3 * int64_t(i) + 1];
    qz = a.witness64[3 * int64_t(i) + 2];
  }
}

__device__ __forceinline__ bool tombed(const uint32_t* bits, int64_t slot) {
  return (bits[slot >> 5] >> (slot & 31)) & 1u;
}

__device__ __forceinline__ void warp_min_vu(double& v, uint32_t& idx) {
  for (int o = 16; o > 0; o >>= 1) {
    const double v2 = __shfl_xor_sync(kAll, v, o);
    const uint32_t i2 = __shfl_xor_sync(kAll, idx, o);
    if (v2 < v || (v2 == v && i2 < idx)) {
      v = v2;
      idx = i2;
    }
  }
}

// ---------------------------------------------------------------------------
// Step query: one block of kQT threads.  Every node and item test runs first
// in FP32 with an error margin that makes it conservative (it never drops a
// node or an item that the exact FP64 comparison could keep); only the items
// that pass are evaluated in FP64 with the oracle's expressions and tie
// rules.  GB300 issues FP64 at a small fraction of the FP32 rate, so the
// filter, not the exact arithmetic, carries the walk.
// ---------------------------------------------------------------------------
constexpr int kQT = 256;
constexpr int kQW = kQT / 32;
constexpr int kQStack = 8192;
constexpr float kRel = 1e-6f;  // ~16 ulp: relative margin of the FP32 filters

struct QShared {
  uint32_t stk[kQStack];
  double rd[4][kQW];
  uint32_t ri[4][kQW];
  int scan[kQW];
};

// block-wide lexicographic (value, index) minimum of NV pairs; every thread
// receives the result
template <int NV>
__device__ void block_argmin(double (&v)[NV], uint32_t (&idx)[NV], QShared& S) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) warp_min_vu(v[i], idx[i]);
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      S.rd[i][w] = v[i];
      S.ri[i][w] = idx[i];
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    v[i] = S.rd[i][0];
    idx[i] = S.ri[i][0];
    for (int k = 1; k < kQW; ++k) {
      const double v2 = S.rd[i][k];
      const uint32_t i2 = S.ri[i][k];
      if (v2 < v[i] || (v2 == v[i] && i2 < idx[i])) {
        v[i] = v2;
        idx[i] = i2;
      }
    }
  }
  __syncthreads();
}

// exclusive block prefix sum of cnt; total receives the block sum
__device__ int block_excl_scan(int cnt, int& total, QShared& S) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int pre = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(kAll, pre, o);
    if (lane >= o) pre += v;
  }
  if (lane == 31) S.scan[w] = pre;
  __syncthreads();
  int base = 0;
  total = 0;
  for (int k = 0; k < kQW; ++k) {
    const int s = S.scan[k];
    if (k < w) base += s;
    total += s;
  }
  __syncthreads();
  return base + pre - cnt;
}

// Block-parallel walk: each round pops up to kQT nodes (one per thread),
// refreshes the shared thresholds, expands the nodes and pushes the children
// the caller marks.  Every thread of the block must call it.
template <class Refresh, class NeedChild, class Leaf>
__device__ void block_walk(const Tree& T, QShared& S, unsigned* err, Refresh refresh, NeedChild need_child,
                           Leaf leaf) {
  if (T.nlevels == 0) return;
  const int tid = threadIdx.x;
  const int top = T.nlevels - 1;
  int sp = int(T.count[top]);
  for (int i = tid; i < sp; i += kQT) S.stk[i] = pack_node(top, i);
  __syncthreads();
  while (sp > 0) {
    const int take = min(sp, kQT);
    const uint32_t nd = tid < take ? S.stk[sp - 1 - tid] : 0xffffffffu;
    sp -= take;
    refresh();
    unsigned mask = 0;
    int64_t cb = 0;
    int lev = -1;
    if (nd != 0xffffffffu) {
      lev = node_level(nd);
      const int64_t idx = node_index(nd);
      if (lev == 0) {
        leaf(idx);
      } else {
        cb = idx * kFan;
        const int64_t ce = min(cb + kFan, T.count[lev - 1]);
        const int64_t off = T.offset[lev - 1];
        for (int64_t c = cb; c < ce; ++c)
          if (need_child(off + c)) mask |= 1u << unsigned(c - cb);
      }
    }
    const int cnt = __popc(mask);
    int total;
    const int pre = block_excl_scan(cnt, total, S);
    if (sp + total > kQStack) {
      if (tid == 0) atomicOr(err, 1u);
      return;
    }
    int w = sp + pre;
    for (int c = 0; c < kFan; ++c)
      if ((mask >> c) & 1u) S.stk[w++] = pack_node(lev - 1, cb + c);
    sp += total;
    __syncthreads();
  }
}

// Greedy descent run by a group of 8 lanes (all 32 lanes of the warp call
// it, each group with its own score): at every level the lanes score the
// children, the lowest score (lowest index on ties) is followed.  Returns the
// leaf reached, uniform across the group.
template <class Score>
__device__ int64_t group_descend(const Tree& T, int sub, Score score) {
  int lev = T.nlevels - 1;
  int64_t cb = 0, ce = T.count[lev];
  for (;;) {
    const int64_t c = cb + sub;
    float v = c < ce ? score(T.offset[lev] + c) : INFINITY;
    int64_t bi = c < ce ? c : cb;
    for (int o = 4; o > 0; o >>= 1) {
      const float v2 = __shfl_xor_sync(kAll, v, o);
      const int64_t i2 = __shfl_xor_sync(kAll, bi, o);
      if (v2 < v || (v2 == v && i2 < bi)) {
        v = v2;
        bi = i2;
      }
    }
    if (lev == 0) return bi;
    cb = bi * kFan;
    ce = min(cb + kFan, T.count[lev - 1]);
    --lev;
  }
}

__device__ __forceinline__ float absmax3(float a, float b, float c) { return fmaxf(fmaxf(fabsf(a), fabsf(b)), fabsf(c)); }

// FP32 upper / lower bounds of an FP64 threshold: the filters compare FP32
// values against these, so no FP64 instruction runs per tested item or node
__device__ __forceinline__ float f_up(double v) { return __double2float_ru(v); }
__device__ __forceinline__ float f_dn(double v) { return __double2float_rd(v); }
// upper bound of sqrt(v) in FP32 (v >= 0; the FP64 root is correctly
// rounded, the factor covers its half ulp)
__device__ __forceinline__ float f_up_sqrt(double v) { return f_up(__dsqrt_rn(v) * (1.0 + 1e-15)); }

}  // namespace

__global__ void __launch_bounds__(kQT) k_ins_query(InsertArgs a, int64_t t) {
  __shared__ QShared S;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const double x = a.y[3 * t], y = a.y[3 * t + 1], z = a.y[3 * t + 2];
  const float xf = float(x), yf = float(y), zf = float(z);
  const float Ax = absmax3(xf, yf, zf);
  const double tol = a.tol;
  const int n_total = *a.n_total;
  // ---- spheres: sample, containment, nearest tangent per class, far bound
  // exact per-thread state (FP64, the oracle's expressions)
  bool cov0 = false, cov1 = false;
  double bA0 = INFINITY, bA1 = INFINITY, bF = INFINITY;
  uint32_t iA0 = 0xffffffffu, iA1 = 0xffffffffu;
  int sample = INT_MAX;
  // block-wide thresholds of the last refresh
  double tA0 = INFINITY, tA1 = INFINITY, tF = INFINITY;
  bool cw0 = false, cw1 = false;
  // FP32 upper bounds of min(block threshold, own best), for the filters
  float fA0 = INFINITY, fA1 = INFINITY, fF = INFINITY;
  const float ntol_up = f_up(-tol);
  auto sphere_exact = [&](int o) {
    const D4 P = a.sph64[o];
    if (P.x == x && P.y == y && P.z == z && o < sample) sample = o;
    const double d2 = ex_d2(x, y, z, P.x, P.y, P.z);
    const double dl = __dsqrt_rn(d2);
    const double r = fabs(P.w);
    if (P.w != 0.0) {
      const bool neg = P.w < 0.0;
      bool& cv = neg ? cov1 : cov0;
      if (!cv && r > tol) {
        const double rt = __dsub_rn(r, tol);
        if (d2 < __dmul_rn(rt, rt)) cv = true;
      }
      const double av = __dsub_rn(dl, r);
      double& bA = neg ? bA1 : bA0;
      uint32_t& iA = neg ? iA1 : iA0;
      if (av < bA || (av == bA && uint32_t(o) < iA)) {
        bA = av;
        iA = uint32_t(o);
        float& fA = neg ? fA1 : fA0;
        fA = fminf(fA, f_up(av));
      }
    }
    const double f = __dadd_rn(dl, r);
    if (f < bF) {
      bF = f;
      fF = fminf(fF, f_up(f));
    }
  };
  // FP32 filter of one sphere (float copy Pf of sphere o): evaluates it
  // exactly unless it provably cannot be the sample, a covering ball, a
  // tangent minimum of its class or the far minimum.  E bounds the rounding
  // of x and p to FP32 (sqrt3 u (|x| + |p|)), of the FP32 distance (3 u d)
  // and of r (u r), with a 5x margin.
  auto sphere_filtered = [&](const float4& Pf, int o) {
    const float dx = xf - Pf.x, dy = yf - Pf.y, dz = zf - Pf.z;
    const float df = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    const float r = fabsf(Pf.w);
    const float E = kRel * (df + r + Ax + absmax3(Pf.x, Pf.y, Pf.z)) + 1e-30f;
    bool need = df <= E;
    if (Pf.w != 0.f) {
      const bool neg = Pf.w < 0.f;
      const bool cv = neg ? (cov1 || cw1) : (cov0 || cw0);
      const float lo = df - r - E;
      if (!cv && lo < ntol_up) need = true;
      if (lo <= (neg ? fA1 : fA0)) need = true;
    }
    if (df + r - E <= fF) need = true;
    if (need) sphere_exact(o);
  };
  auto refresh_spheres = [&]() {
    double v[3] = {bA0, bA1, bF};
    uint32_t id[3] = {0, 0, 0};
    block_argmin<3>(v, id, S);
    tA0 = v[0];
    tA1 = v[1];
    tF = v[2];
    fA0 = fminf(fA0, f_up(tA0));
    fA1 = fminf(fA1, f_up(tA1));
    fF = fminf(fF, f_up(tF));
    cw0 = __syncthreads_or(cov0) != 0;
    cw1 = __syncthreads_or(cov1) != 0;
  };
  // spheres inserted since the last rebuild (at most one per step)
  for (int o = a.n_static + tid; o < n_total; o += kQT) {
    const D4 P = a.sph64[o];
    float w = float(P.w);
    if (w == 0.f && P.w != 0.0) w = copysignf(1.4e-45f, float(P.w));
    sphere_filtered(make_float4(float(P.x), float(P.y), float(P.z), w), o);
  }
  // seed: warp 0 runs four greedy descents (nearest box, each class's
  // tangent bound, far bound); each group of 8 lanes evaluates the items of
  // the leaf it reached
  if (wid == 0 && a.st.nlevels > 0) {
    const int grp = lane >> 3, sub = lane & 7;
    const int64_t nl = group_descend(a.st, sub, [&](int64_t node) {
      if (grp == 0) return box_d2(xf, yf, zf, a.st.lo[node], a.st.hi[node]);
      if (grp == 3) {
        const float4 Fb = a.st.nf[node];
        return sqrtf(ball_d2(xf, yf, zf, Fb)) - Fb.w;
      }
      const float4 R = a.st.nb[node];
      const float w = grp == 1 ? R.x : R.y;
      if (!(w > -INFINITY)) return INFINITY;
      return sqrtf(ball_d2(xf, yf, zf, a.st.na[node])) - w;
    });
    const int64_t j = nl * kLeaf + sub;
    if (j < a.st.nitems) sphere_filtered(a.sph[j], a.sid[j]);
  }
  block_walk(
      a.st, S, a.err, refresh_spheres,
      [&](int64_t node) {
        // lower bounds over the node's spheres of |x-p| - r (per class),
        // |x-p| + r (far) and |x-p| (a sample at x): |x-C| - w, evaluated in
        // FP32 with margin
        const float4 R = a.st.nb[node], Fb = a.st.nf[node];
        const float dc = sqrtf(ball_d2(xf, yf, zf, a.st.na[node]));
        const float df = sqrtf(ball_d2(xf, yf, zf, Fb));
        auto below = [&](float d, float w, float th) {
          if (!(w > -INFINITY)) return false;
          const float E = kRel * (d + fabsf(w) + Ax) + 1e-30f;
          return d - w - E <= th;
        };
        const float th0 = cw0 ? fA0 : fmaxf(fA0, ntol_up);
        const float th1 = cw1 ? fA1 : fmaxf(fA1, ntol_up);
        return below(dc, R.z, 0.f) || below(dc, R.x, th0) || below(dc, R.y, th1) || below(df, Fb.w, fF);
      },
      [&](int64_t leaf) {
        const int64_t b = leaf * kLeaf, e = min(b + kLeaf, a.st.nitems);
        for (int64_t j = b; j < e; ++j) sphere_filtered(a.sph[j], a.sid[j]);
      });
  const bool c0 = __syncthreads_or(cov0) != 0, c1 = __syncthreads_or(cov1) != 0;
  {
    double v[4] = {bA0, bA1, bF, double(sample)};
    uint32_t id[4] = {iA0, iA1, 0, 0};
    block_argmin<4>(v, id, S);
    bA0 = v[0];
    bA1 = v[1];
    bF = v[2];
    iA0 = id[0];
    iA1 = id[1];
    sample = v[3] < double(INT_MAX) ? int(v[3]) : INT_MAX;
  }
  // a known value's sign fixes the class (Sec. 6 repair), else containment
  const double sk = a.known ? a.known[t] : 0.0;
  const int ks = sk > 0.0 ? 0 : (sk < 0.0 ? 1 : -1);
  int code = -1;
  double value = 0.0;
  int64_t arg = -1;
  if (sample != INT_MAX) {
    code = GFS_CODE_SAMPLE;
    value = a.sph64[sample].w;
    arg = sample;
  } else if (ks >= 0) {
    // class given: no OUTSIDE / INVALID outcome
  } else if (c0 && c1) {
    code = GFS_CODE_INVALID;
    value = __longlong_as_double(0x7ff8000000000000LL);
  } else if (!c0 && !c1) {
    code = GFS_CODE_OUTSIDE;
  }
  if (code >= 0) {
    if (tid == 0) {
      if (a.s_out) a.s_out[t] = value;
      if (a.arg_out) a.arg_out[t] = arg;
      if (a.fl_out) a.fl_out[t] = uint16_t(code);
      a.rec->insert = 0;
    }
    return;
  }
  const int cs = ks >= 0 ? ks : (c0 ? 0 : 1);
  const double bAs = cs == 0 ? bA0 : bA1, bAo = cs == 0 ? bA1 : bA0;
  const uint32_t iAs = cs == 0 ? iA0 : iA1, iAo = cs == 0 ? iA1 : iA0;
  // ---- nearest live survivor of x's class ----------------------------------
  double bd = INFINITY, td = INFINITY;  // squared distances: own best, block threshold
  float fd = INFINITY;                   // FP32 upper bound of sqrt(min(td, bd))
  uint32_t gbest = 0xffffffffu;
  const float eqt = float(a.bc->eq);
  auto surv_exact = [&](uint32_t g) {
    double qx, qy, qz;
    surv64(a, g, qx, qy, qz);
    const double d2 = ex_d2(x, y, z, qx, qy, qz);
    if (d2 < bd || (d2 == bd && g < gbest)) {
      bd = d2;
      gbest = g;
      fd = fminf(fd, f_up_sqrt(d2));
    }
  };
  // FP32 filter of one survivor: its FP32 position is within eq of the exact
  // one per coordinate (eq covers the FP32 candidate formula; a rounded FP64
  // point is within u |q| <= eq of it)
  auto surv_filtered = [&](const float4& P) {
    const float dx = xf - P.x, dy = yf - P.y, dz = zf - P.z;
    const float df = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    const float eqi = fmaxf(eqt, 1.2e-7f * absmax3(P.x, P.y, P.z));
    const float lo = df - (1.7320508f * eqi * 1.01f + kRel * (df + Ax) + 1e-30f);
    if (lo <= fd) surv_exact(__float_as_uint(P.w));
  };
  auto refresh_surv = [&]() {
    double v[1] = {bd};
    uint32_t id[1] = {0};
    block_argmin<1>(v, id, S);
    td = v[0];
    if (td < INFINITY) fd = fminf(fd, f_up_sqrt(td));
  };
  {
    const Tree& T = a.vt[cs];
    const float4* items = a.surv[cs];
    const uint32_t* tomb = a.tomb[cs];
    // survivors added since the rebuild (recent insertions lie nearby, so
    // this list gives the walk a tight threshold)
    const unsigned nd = a.dcount_start[cs];
    for (unsigned j = tid; j < nd; j += kQT)
      if (!a.dtomb[cs][j]) surv_filtered(a.dsurv[cs][j]);
    // seed: the leaf nearest by box and its three successors in Morton order
    if (wid == 0 && T.nlevels > 0) {
      const int grp = lane >> 3, sub = lane & 7;
      const int64_t nl = group_descend(T, sub, [&](int64_t node) { return box_d2(xf, yf, zf, T.lo[node], T.hi[node]); });
      const int64_t j = (nl + grp) * kLeaf + sub;
      if (j < T.nitems && !tombed(tomb, j)) surv_filtered(items[j]);
    }
    const float slack = f_up(2.0 * 1.7320508075688772 * double(a.bc->eq) + 1e-12);
    block_walk(
        T, S, a.err, refresh_surv,
        [&](int64_t node) {
          const float db = sqrtf(box_d2(xf, yf, zf, T.lo[node], T.hi[node]));
          return db - kRel * (db + Ax) - 1e-30f - slack <= fd;
        },
        [&](int64_t leaf) {
          const int64_t b = leaf * kLeaf, e = min(b + kLeaf, T.nitems);
          for (int64_t j = b; j < e; ++j)
            if (!tombed(tomb, j)) surv_filtered(items[j]);
        });
  }
  {
    double v[1] = {bd};
    uint32_t id[1] = {gbest};
    block_argmin<1>(v, id, S);
    bd = v[0];
    gbest = id[0];
  }
  if (tid != 0) return;
  const bool have_s = gbest != 0xffffffffu, have_u = iAo != 0xffffffffu;
  const double ds = have_s ? __dsqrt_rn(bd) : INFINITY;
  const double ub = have_u ? bAo : INFINITY;
  const double lb = -bAs;
  double m;
  if (have_s && (!a.clamp_opp || ds <= ub)) {
    code = GFS_CODE_SURVIVOR;
    m = ds;
    arg = int64_t(gbest);
  } else if (a.clamp_opp && have_u) {
    code = GFS_CODE_OPPOSITE;
    m = ub;
    arg = int64_t(iAo);
  } else {
    code = GFS_CODE_LOWER;
    m = lb;
    arg = iAs == 0xffffffffu ? int64_t(-1) : int64_t(iAs);
  }
  if (m < 0.0) m = 0.0;
  int flags = code;
  if (m < __dsub_rn(lb, tol)) flags |= GFS_FLAG_LB_VIOL;
  if (m > __dadd_rn(bF, tol)) flags |= GFS_FLAG_FAR_VIOL;
  if (have_u && ub < __dsub_rn(m, tol)) flags |= GFS_FLAG_OPP_VIOL;
  value = cs == 0 ? m : -m;
  if (ks >= 0 && fabs(value) < __dsub_rn(fabs(sk), tol)) flags |= GFS_FLAG_NONCONSERVATIVE;
  if (a.s_out) a.s_out[t] = value;
  if (a.arg_out) a.arg_out[t] = arg;
  if (a.fl_out) a.fl_out[t] = uint16_t(flags);
  // witness: the point that set the value
  double wx, wy, wz;
  if (code == GFS_CODE_SURVIVOR) {
    surv64(a, gbest, wx, wy, wz);
  } else if (arg < 0) {  // no sphere sets the value (value 0): the point itself
    wx = x;
    wy = y;
    wz = z;
  } else {
    const D4 pj = a.sph64[arg];
    const double rj = fabs(pj.w);
    const double dx = __dsub_rn(x, pj.x), dy = __dsub_rn(y, pj.y), dz = __dsub_rn(z, pj.z);
    const double d = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
    wx = __dadd_rn(pj.x, __dmul_rn(rj, __ddiv_rn(dx, d)));
    wy = __dadd_rn(pj.y, __dmul_rn(rj, __ddiv_rn(dy, d)));
    wz = __dadd_rn(pj.z, __dmul_rn(rj, __ddiv_rn(dz, d)));
  }
  const int jn = n_total;
  a.sph64[jn] = D4{x, y, z, value};
  a.witness64[3 * int64_t(jn)] = wx;
  a.witness64[3 * int64_t(jn) + 1] = wy;
  a.witness64[3 * int64_t(jn) + 2] = wz;
  a.counts[jn] = 0;
  *a.n_total = n_total + 1;
  a.rec->insert = 1;
}

// Cull the new sphere's candidates and witness; tombstone covered survivors.
// Blocks [0, nc) hold one warp per candidate (k = 0..K, k = K the witness):
// a warp-parallel walk of the sphere hierarchy that stops at the first
// covering ball (FP32 decisions where provably away from the boundary, FP64
// otherwise).  Block nc walks both survivor hierarchies with the new ball
// (warps 0, 1); the kDynBlocks blocks after it scan the survivor lists added
// since the rebuild.  The block that finishes last sets LOST_WITNESS and
// opens the next step.
constexpr int kUStack = 2048;
constexpr int kDynBlocks = 16;  // update blocks that scan the lists added since the rebuild

template <class Refresh, class NeedChild, class Leaf>
__device__ void warp_walk_until(const Tree& T, uint32_t* stk, int cap, int lane, unsigned* err, Refresh refresh,
                                NeedChild need_child, Leaf leaf) {
  if (T.nlevels == 0) return;
  const int top = T.nlevels - 1;
  int sp = int(T.count[top]);
  if (lane < sp) stk[lane] = pack_node(top, lane);
  __syncwarp();
  while (sp > 0) {
    if (!refresh()) return;
    const int take = min(sp, 32);
    const uint32_t nd = lane < take ? stk[sp - 1 - lane] : 0xffffffffu;
    sp -= take;
    __syncwarp();
    unsigned mask = 0;
    int64_t cb = 0;
    int lev = -1;
    if (nd != 0xffffffffu) {
      lev = node_level(nd);
      const int64_t idx = node_index(nd);
      if (lev == 0) {
        leaf(idx);
      } else {
        cb = idx * kFan;
        const int64_t ce = min(cb + kFan, T.count[lev - 1]);
        const int64_t off = T.offset[lev - 1];
        for (int64_t c = cb; c < ce; ++c)
          if (need_child(off + c)) mask |= 1u << unsigned(c - cb);
      }
    }
    const int cnt = __popc(mask);
    int pre = cnt;
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(kAll, pre, o);
      if (lane >= o) pre += v;
    }
    const int total = __shfl_sync(kAll, pre, 31);
    pre -= cnt;
    if (sp + total > cap) {
      if (lane == 0) atomicOr(err, 1u);
      return;
    }
    int w = sp + pre;
    for (int c = 0; c < kFan; ++c)
      if ((mask >> c) & 1u) stk[w++] = pack_node(lev - 1, cb + c);
    sp += total;
    __syncwarp();
  }
}

__global__ void __launch_bounds__(128) k_ins_update(InsertArgs a, int64_t t) {
  __shared__ uint32_t s_stk[4][kUStack];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint32_t* stk = s_stk[wib];
  const bool active = a.rec->insert != 0;
  const int jn = *a.n_total - 1;
  const int KS = a.KS;
  const int ncand_blocks = (KS + 3) / 4;
  if (active) {
    const D4 nw = a.sph64[jn];
    const double tol = a.tol;
    const float ntol_up = f_up(-tol), ntol_dn = f_dn(-tol);
    if (int(blockIdx.x) < ncand_blocks) {
      const int k = int(blockIdx.x) * 4 + wib;
      if (k < KS) {
        double qx, qy, qz;
        if (k < a.K) {
          ex_cand(nw, a.U64[3 * k], a.U64[3 * k + 1], a.U64[3 * k + 2], qx, qy, qz);
        } else {
          qx = a.witness64[3 * int64_t(jn)];
          qy = a.witness64[3 * int64_t(jn) + 1];
          qz = a.witness64[3 * int64_t(jn) + 2];
        }
        if (!a.box_cull || ex_inbox(qx, qy, qz)) {
          const float qxf = float(qx), qyf = float(qy), qzf = float(qz);
          const float Aq = absmax3(qxf, qyf, qzf);
          // FP32 filter of "q is in the ball of sphere o shrunk by tol":
          // decided in FP32 when |d - r| is provably away from tol (E bounds
          // the rounding of q and p to FP32, of the distance and of r), else
          // by the exact FP64 predicate
          auto covered_by = [&](const float4& Pf, int o) {
            const float dx = qxf - Pf.x, dy = qyf - Pf.y, dz = qzf - Pf.z;
            const float df = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
            const float r = fabsf(Pf.w);
            const float E = kRel * (df + r + Aq + absmax3(Pf.x, Pf.y, Pf.z)) + 1e-30f;
            if (df - r - E >= ntol_up) return false;
            if (df - r + E < ntol_dn) return true;
            return ex_cov(qx, qy, qz, a.sph64[o], tol);
          };
          bool covered = false;
          for (int o = a.n_static + lane; o < jn && !covered; o += 32) {
            const D4 P = a.sph64[o];
            if (covered_by(make_float4(float(P.x), float(P.y), float(P.z), float(P.w)), o)) covered = true;
          }
          warp_walk_until(
              a.st, stk, kUStack, lane, a.err, [&]() { return !__any_sync(kAll, covered); },
              [&](int64_t node) {
                // some sphere of the node has |q-p| - r < -tol only if
                // |q-C| - max(wp, wn) < -tol
                const float4 B = a.st.na[node];
                if (!(B.w > -INFINITY)) return false;
                const float dc = sqrtf(ball_d2(qxf, qyf, qzf, B));
                const float E = kRel * (dc + fabsf(B.w) + Aq) + 1e-30f;
                return dc - B.w - E < ntol_up;
              },
              [&](int64_t leaf) {
                const int64_t b = leaf * kLeaf, e = min(b + kLeaf, a.st.nitems);
                for (int64_t j = b; j < e && !covered; ++j)
                  if (covered_by(a.sph[j], a.sid[j])) covered = true;
              });
          covered = __any_sync(kAll, covered);
          if (!covered && lane == 0) {
            const uint32_t g = uint32_t(jn) * uint32_t(KS) + uint32_t(k);
            const float4 item = make_float4(qxf, qyf, qzf, __uint_as_float(g));
            for (int c = 0; c < 2; ++c) {
              const bool mine = c == 0 ? !(nw.w < 0.0) : !(nw.w > 0.0);
              if (!mine) continue;
              const unsigned slot = atomicAdd(a.dcount + c, 1u);
              if (slot < a.dcap) {
                a.dsurv[c][slot] = item;
                a.dtomb[c][slot] = 0;
              } else {
                atomicOr(a.err, 2u);
              }
            }
            atomicAdd(a.counts + jn, 1);
          }
        }
      }
    } else {
      // survivors the new ball covers
      const double rn = fabs(nw.w);
      const float nxf = float(nw.x), nyf = float(nw.y), nzf = float(nw.z);
      const float An = absmax3(nxf, nyf, nzf);
      const float eqt = float(a.bc->eq);
      const float reach = f_up(rn - tol + 2.0 * 1.7320508075688772 * double(eqt) + 1e-9);
      const float rkill = f_up(rn - tol);
      auto kill = [&](int cls, const float4& P, bool dyn, int64_t j) {
        // FP32 filter: the exact survivor lies within sqrt3 eqi of P
        const float dx = P.x - nxf, dy = P.y - nyf, dz = P.z - nzf;
        const float df = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        const float eqi = fmaxf(eqt, 1.2e-7f * absmax3(P.x, P.y, P.z));
        const float E = kRel * (df + An + absmax3(P.x, P.y, P.z)) + 1.7320508f * eqi * 1.01f + 1e-30f;
        if (df - E >= rkill) return;
        const uint32_t g = __float_as_uint(P.w);
        double qx, qy, qz;
        surv64(a, g, qx, qy, qz);
        if (!ex_cov(qx, qy, qz, nw, tol)) return;
        bool fresh;
        if (dyn) {
          fresh = atomicExch(a.dtomb[cls] + j, 1u) == 0u;
        } else {
          const uint32_t bit = 1u << unsigned(j & 31);
          fresh = !(atomicOr(a.tomb[cls] + (j >> 5), bit) & bit);
        }
        if (!fresh) return;
        // count each survivor once (a zero sample's survivors are in both lists)
        const int sph = int(g / uint32_t(KS));
        if (cls == 1 && a.sph64[sph].w == 0.0) return;
        if (atomicSub(a.counts + sph, 1) == 1) atomicOr(a.lost, 1u);
      };
      if (int(blockIdx.x) == ncand_blocks) {
        if (wib < 2) {
          const int cls = wib;
          const Tree& T = a.vt[cls];
          warp_walk_until(
              T, stk, kUStack, lane, a.err, [&]() { return true; },
              [&](int64_t node) {
                const float db = sqrtf(box_d2(nxf, nyf, nzf, T.lo[node], T.hi[node]));
                return db - kRel * (db + An) - 1e-30f < reach;
              },
              [&](int64_t leaf) {
                const int64_t b = leaf * kLeaf, e = min(b + kLeaf, T.nitems);
                for (int64_t j = b; j < e; ++j) kill(cls, a.surv[cls][j], false, j);
              });
        }
      } else {
        // lists added since the rebuild, spread over the scan blocks
        const unsigned n0 = a.dcount_start[0], n1 = a.dcount_start[1];
        const unsigned nthr = (gridDim.x - ncand_blocks - 1) * blockDim.x;
        for (unsigned j = (blockIdx.x - ncand_blocks - 1) * blockDim.x + threadIdx.x; j < n0 + n1; j += nthr) {
          if (j < n0) kill(0, a.dsurv[0][j], true, j);
          else kill(1, a.dsurv[1][j - n0], true, j - n0);
        }
      }
    }
  }
  // the last block to finish closes the step
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(a.done, 1u);
    s_last = done == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    if (active && *a.lost && a.fl_out) a.fl_out[t] = uint16_t(a.fl_out[t] | GFS_FLAG_LOST_WITNESS);
    *a.lost = 0;
    a.dcount_start[0] = a.dcount[0];
    a.dcount_start[1] = a.dcount[1];
    *a.done = 0;
  }
}

// per-sphere survivor counts from the survivor lists (after a build/rebuild)
__global__ void k_ins_counts(const float4* __restrict__ s0, unsigned n0, const float4* __restrict__ s1, unsigned n1,
                             const D4* __restrict__ sph64, int KS, int* __restrict__ counts) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n0) {
    atomicAdd(counts + __float_as_uint(s0[t].w) / unsigned(KS), 1);
  } else if (t < n0 + n1) {
    const unsigned sph = __float_as_uint(s1[t - n0].w) / unsigned(KS);
    if (sph64[sph].w != 0.0) atomicAdd(counts + sph, 1);
  }
}

// live survivors of one class into a fresh list (before a rebuild)
__global__ void k_ins_compact(const float4* __restrict__ ssurv, const uint32_t* __restrict__ tomb, unsigned ns,
                              const float4* __restrict__ dsurv, const uint32_t* __restrict__ dtomb, unsigned nd,
                              float4* __restrict__ out, unsigned* __restrict__ count) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  float4 v;
  bool live;
  if (t < ns) {
    v = ssurv[t];
    live = !((tomb[t >> 5] >> (t & 31)) & 1u);
  } else if (t < ns + nd) {
    v = dsurv[t - ns];
    live = !dtomb[t - ns];
  } else {
    return;
  }
  if (live) out[atomicAdd(count, 1u)] = v;
}

cudaError_t launch_ins_step(const InsertArgs& a, int64_t t, cudaStream_t st) {
  k_ins_query<<<1, kQT, 0, st>>>(a, t);
  k_ins_update<<<(a.KS + 3) / 4 + 1 + kDynBlocks, 128, 0, st>>>(a, t);
  return cudaGetLastError();
}

cudaError_t launch_ins_counts(const float4* s0, unsigned n0, const float4* s1, unsigned n1, const D4* sph64, int KS,
                              int* counts, cudaStream_t st) {
  if (n0 + n1 == 0) return cudaSuccess;
  k_ins_counts<<<(n0 + n1 + 255) / 256, 256, 0, st>>>(s0, n0, s1, n1, sph64, KS, counts);
  return cudaGetLastError();
}

cudaError_t launch_ins_compact(const float4* ssurv, const uint32_t* tomb, unsigned ns, const float4* dsurv,
                               const uint32_t* dtomb, unsigned nd, float4* out, unsigned* count, cudaStream_t st) {
  if (ns + nd == 0) return cudaSuccess;
  k_ins_compact<<<(ns + nd + 255) / 256, 256, 0, st>>>(ssurv, tomb, ns, dsurv, dtomb, nd, out, count);
  return cudaGetLastError();
}

}  // namespace gfs
