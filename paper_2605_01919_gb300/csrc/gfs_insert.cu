// Greedy sequential insertion (Sec. 4: every new value is consistent with
// the inputs and with all values generated before it), run as deterministic
// parallel rounds with the results of the sequential loop.
//
// A round takes a window of the first pending steps (in step order):
//   k_ins_query    -- one block per step evaluates its value exactly (the
//                     oracle's FP64 expressions and tie rules) against the
//                     state at the start of the round, with a
//                     block-parallel walk of the hierarchies (FP32 filters in
//                     front of every FP64 evaluation), and records a bound R
//                     on the step's value in any later state and the radius
//                     rho of the region that decides its result;
//   k_ins_conflict -- a step commits when no earlier pending step can reach
//                     it or be reached by it (disjoint balls B(y_t, R_t) and
//                     B(y_t', rho_t')), so its result is the sequential one;
//   k_ins_commit   -- committed results go out, their spheres join the state
//                     and the window is compacted and refilled;
// then the state update of the round's new spheres (covered survivors are
// tombstoned, the new candidates and witnesses culled and added).  The first
// pending step always commits, so every round makes progress.  Steps that
// commit out of step order use provisional sphere indices n0 + t (which order
// them as the sequential numbering does); the call renumbers the inserted
// spheres consecutively at the end.
//
// State between hierarchy rebuilds:
//   spheres    in the sphere hierarchy, plus a list of the ones inserted
//              since the last rebuild (scanned linearly);
//   survivors  the per-class survivor hierarchies (with a tombstone bit per
//              sorted slot) plus per-class lists of survivors added since
//              the last rebuild (with a tombstone word each).
#include <cub/cub.cuh>

#include "gfs_internal.cuh"
#include "gfs_warp.cuh"
#include "gfs_kernels.h"

namespace gfs {

static unsigned long long g_insert_launches = 0;
unsigned long long insert_launch_count() { return g_insert_launches; }

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
constexpr int kQStack = 8192;  // walk stack entries (plus a reserve of kFan)
constexpr float kRel = 1e-6f;  // ~16 ulp: relative margin of the FP32 filters

constexpr int kQCap = 288;     // per-warp queue of items awaiting their FP64 evaluation
static_assert(32 % kLeaf == 0, "a leaf's slots must share one tombstone word");

struct QShared {
  uint32_t stk[kQStack + kFan];
  double rd[4][kQW];
  uint32_t ri[4][kQW];
  int scan[kQW];
  // Survivors that pass a thread's FP32 screen are queued per warp with
  // their FP32 lower bound, while the thread's threshold already tightens to
  // their FP32 upper bounds; the queue is evaluated in FP64 after the next
  // block-wide threshold exchange, by all 32 lanes together, skipping every
  // item that the exchanged threshold rules out.  Evaluated where screened,
  // each thread would take one FP64 evaluation per new running minimum of its
  // own items (most of them far from the block's minimum), a few lanes at a
  // time.
  uint32_t q[kQW][kQCap];
  float qlo[kQW][kQCap];
  int qn[kQW];
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
// the caller marks.  A round pops at most (kQStack - sp) / kFan nodes (at
// least one), so the stack never outgrows kQStack + kFan - 1 entries: a wide
// frontier turns the walk depth-first instead of overflowing.  Each round
// and the end of the walk call refresh() and then post() (work the previous
// round queued) on every thread.  Every thread of the block must call it.
template <class Refresh, class NeedChild, class Leaf, class Post>
__device__ void block_walk(const Tree& T, QShared& S, unsigned* err, Refresh refresh, NeedChild need_child,
                           Leaf leaf, Post post) {
  if (T.nlevels == 0) return;
  const int tid = threadIdx.x;
  const int top = T.nlevels - 1;
  int sp = int(T.count[top]);
  for (int i = tid; i < sp; i += kQT) S.stk[i] = pack_node(top, i);
  __syncthreads();
  while (sp > 0) {
    const int take = min(min(sp, kQT), max(1, (kQStack - sp) / kFan));
    const uint32_t nd = tid < take ? S.stk[sp - 1 - tid] : 0xffffffffu;
    sp -= take;
    refresh();
    post();  // every thread: the work queued in the previous round
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
    if (sp + total > kQStack + kFan) {  // cannot happen (see above); kept as a guard
      if (tid == 0) atomicOr(err, 1u);
      return;
    }
    int w = sp + pre;
    for (int c = 0; c < kFan; ++c)
      if ((mask >> c) & 1u) S.stk[w++] = pack_node(lev - 1, cb + c);
    sp += total;
    __syncthreads();
  }
  refresh();
  post();
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

// Speculative step query: block `slot` evaluates the value of its pending
// step exactly (the oracle's FP64 expressions and tie rules) against the
// state at the start of the round, and records what the commit test needs.
__global__ void __launch_bounds__(kQT) k_ins_query(InsertArgs a) {
  __shared__ QShared S;
  const int slot = int(blockIdx.x);
  if (slot >= a.misc->npend) return;
  const int64_t t = a.slot_t[slot];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const double x = a.y[3 * t], y = a.y[3 * t + 1], z = a.y[3 * t + 2];
  const float xf = float(x), yf = float(y), zf = float(z);
  const float Ax = absmax3(xf, yf, zf);
  const double tol = a.tol;
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
  unsigned n_sph_exact = 0, n_sph_tested = 0, n_surv_exact = 0, n_surv_tested = 0;
  if (lane == 0) S.qn[wid] = 0;
  __syncwarp();
  // queue a survivor for the warp's next FP64 pass (at most 8 per lane
  // between passes; passes run at convergent points)
  auto enqueue = [&](uint32_t id, float lo) {
    const int k = atomicAdd(&S.qn[wid], 1);
    if (k < kQCap) {
      S.q[wid][k] = id;
      S.qlo[wid][k] = lo;
    } else {
      atomicOr(&a.misc->err, 1u);  // cannot happen with the passes placed as they are
    }
  };
  auto sphere_exact = [&](int o) {
    ++n_sph_exact;
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
  // FP32 filter of one sphere (float copy Pf): it needs its exact
  // evaluation unless it provably cannot be the sample, a covering ball, a
  // tangent minimum of its class or the far minimum.  E bounds the rounding
  // of x and p to FP32 (sqrt3 u (|x| + |p|)), of the FP32 distance (3 u d)
  // and of r (u r), with a 5x margin.  A ball that provably covers x sets its
  // class's containment without the FP64 test (the same decision), and the
  // FP32 upper bounds of its tangent and far distances tighten the
  // thresholds at once.
  const float ntol_dn = f_dn(-tol);
  auto sphere_need = [&](const float4& Pf, bool tighten) {
    const float dx = xf - Pf.x, dy = yf - Pf.y, dz = zf - Pf.z;
    const float df = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    const float r = fabsf(Pf.w);
    const float E = kRel * (df + r + Ax + absmax3(Pf.x, Pf.y, Pf.z)) + 1e-30f;
    bool need = df <= E;
    if (Pf.w != 0.f) {
      const bool neg = Pf.w < 0.f;
      bool& cvo = neg ? cov1 : cov0;
      const bool cv = cvo || (neg ? cw1 : cw0);
      const float lo = df - r - E;
      if (!cv && lo < ntol_up) {
        if (tighten && df - r + E < ntol_dn) cvo = true;
        else need = true;
      }
      float& fA = neg ? fA1 : fA0;
      if (lo <= fA) need = true;
      if (tighten) fA = fminf(fA, df - r + E);
    }
    if (df + r - E <= fF) need = true;
    if (tighten) fF = fminf(fF, df + r + E);
    return need;
  };
  // locator of a sphere's FP32 copy: sorted slot j of the hierarchy, or
  // (bit 31) slot j of the dynamic list
  auto sphere_at = [&](uint32_t loc, float4& Pf) {
    if (loc >> 31) {
      Pf = a.dyn_f4[loc & 0x7fffffffu];
      return a.dyn_ids[loc & 0x7fffffffu];
    }
    Pf = a.sph[loc];
    return a.sid[loc];
  };
  auto sphere_screen = [&](const float4& Pf, uint32_t loc) {
    ++n_sph_tested;
    if (sphere_need(Pf, true)) enqueue(loc, 0.f);
  };
  auto sphere_filtered = [&](uint32_t loc) {
    float4 Pf;
    sphere_at(loc, Pf);
    sphere_screen(Pf, loc);
  };
  // the warp's FP64 pass over its queued spheres, after a threshold
  // exchange: each is screened again with the warp's least thresholds (one
  // per lane, all lanes call it)
  auto drain_spheres = [&]() {
    __syncwarp();
    for (int o = 16; o > 0; o >>= 1) {
      fA0 = fminf(fA0, __shfl_xor_sync(kAll, fA0, o));
      fA1 = fminf(fA1, __shfl_xor_sync(kAll, fA1, o));
      fF = fminf(fF, __shfl_xor_sync(kAll, fF, o));
    }
    cw0 = cw0 || __any_sync(kAll, cov0);
    cw1 = cw1 || __any_sync(kAll, cov1);
    const int n = min(S.qn[wid], kQCap);
    for (int b = 0; b < n; b += 32)
      if (b + lane < n) {
        float4 Pf;
        const int o = sphere_at(S.q[wid][b + lane], Pf);
        if (sphere_need(Pf, false)) sphere_exact(o);
      }
    __syncwarp();
    if (lane == 0) S.qn[wid] = 0;
    __syncwarp();
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
    if (j < a.st.nitems) sphere_filtered(uint32_t(j));
  }
  // the seeds' bounds, block-wide, before the spheres inserted since the
  // last rebuild (FP32 copies, the sign class kept) are screened with them
  refresh_spheres();
  drain_spheres();
  const int ndyn = a.misc->ndyn;
  for (int base = 0; base < ndyn; base += kQT) {
    if (base + tid < ndyn) sphere_filtered(0x80000000u | uint32_t(base + tid));
    drain_spheres();
  }
  block_walk(
      a.st, S, &a.misc->err, refresh_spheres,
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
        // all of the leaf's loads first, then the screens
        float4 P[kLeaf];
#pragma unroll
        for (int k = 0; k < kLeaf; ++k)
          if (b + k < e) P[k] = a.sph[b + k];
#pragma unroll
        for (int k = 0; k < kLeaf; ++k)
          if (b + k < e) sphere_screen(P[k], uint32_t(b + k));
      },
      drain_spheres);
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
  auto flush_counts = [&]() {
    const unsigned v[4] = {n_sph_exact, n_sph_tested, n_surv_exact, n_surv_tested};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const unsigned w = __reduce_add_sync(kAll, v[k]);
      if (lane == 0 && w) atomicAdd(&a.misc->work[k], (unsigned long long)w);
    }
  };
  if (code >= 0) {
    flush_counts();
    if (tid == 0) {
      InsSlot r;
      r.value = value;
      r.wx = r.wy = r.wz = 0.0;
      // SAMPLE and INVALID results never change (a lower-index sample stays;
      // containment only grows) and never insert; an OUTSIDE point may later
      // lie in a new ball of either class, with a value below that class's
      // nearest opposite tangent distance
      r.R = -1.0;
      if (code == GFS_CODE_OUTSIDE)
        r.R = a.clamp_opp ? fmax(fmax(bA0, bA1), 0.0) : INFINITY;
      r.rho = 0.0;
      r.arg = arg;
      r.t = int(t);
      r.flags = uint16_t(code);
      r.insert = 0;
      r.pad = 0;
      a.slots[slot] = r;
    }
    return;
  }
  const int cs = ks >= 0 ? ks : (c0 ? 0 : 1);
  const double bAs = cs == 0 ? bA0 : bA1, bAo = cs == 0 ? bA1 : bA0;
  const uint32_t iAs = cs == 0 ? iA0 : iA1, iAo = cs == 0 ? iA1 : iA0;
  // ---- nearest live survivor of x's class ----------------------------------
  double bd = INFINITY, td = INFINITY;  // squared distances: own best, block threshold
  // FP32 upper bound of sqrt(min(td, bd)); with the opposite clamp a survivor
  // farther than UB_opp never sets the value, so the search starts there
  float fd = (a.clamp_opp && iAo != 0xffffffffu) ? fmaxf(f_up(bAo), 0.f) : INFINITY;
  uint32_t gbest = 0xffffffffu;
  const float eqt = float(a.bc->eq);
  auto surv_exact = [&](uint32_t g) {
    ++n_surv_exact;
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
    ++n_surv_tested;
    const float dx = xf - P.x, dy = yf - P.y, dz = zf - P.z;
    const float df = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    const float eqi = fmaxf(eqt, 1.2e-7f * absmax3(P.x, P.y, P.z));
    const float mg = 1.7320508f * eqi * 1.01f + kRel * (df + Ax) + 1e-30f;
    const float lo = df - mg;
    if (lo <= fd) {
      enqueue(__float_as_uint(P.w), lo);
      // an upper bound of the distance of a live survivor bounds the minimum
      fd = fminf(fd, df + mg);
    }
  };
  // the warp's FP64 pass over its queue, after a threshold exchange: the
  // warp's least threshold first, then one item per lane (all lanes call it)
  auto drain_surv = [&]() {
    __syncwarp();
    float fw = fd;
    for (int o = 16; o > 0; o >>= 1) fw = fminf(fw, __shfl_xor_sync(kAll, fw, o));
    fd = fw;
    const int n = min(S.qn[wid], kQCap);
    for (int b = 0; b < n; b += 32)
      if (b + lane < n && S.qlo[wid][b + lane] <= fd) surv_exact(S.q[wid][b + lane]);
    __syncwarp();
    if (lane == 0) S.qn[wid] = 0;
    __syncwarp();
  };
  auto refresh_surv = [&]() {
    double v[2] = {bd, double(fd)};
    uint32_t id[2] = {0, 0};
    block_argmin<2>(v, id, S);
    td = v[0];
    fd = fminf(fd, float(v[1]));  // exact conversion: v[1] is a float
    if (td < INFINITY) fd = fminf(fd, f_up_sqrt(td));
  };
  {
    const Tree& T = a.vt[cs];
    const float4* items = a.surv[cs];
    const uint32_t* tomb = a.tomb[cs];
    // seed: the leaf nearest by box and its three successors in Morton order
    if (wid == 0 && T.nlevels > 0) {
      const int grp = lane >> 3, sub = lane & 7;
      const int64_t nl = group_descend(T, sub, [&](int64_t node) { return box_d2(xf, yf, zf, T.lo[node], T.hi[node]); });
      const int64_t j = (nl + grp) * kLeaf + sub;
      if (j < T.nitems && !tombed(tomb, j)) surv_filtered(items[j]);
    }
    refresh_surv();  // the seed's distance, block-wide, before the dynamic survivors are screened
    drain_surv();
    // survivors of the spheres inserted since the rebuild (recent insertions
    // lie nearby, so they give the walk a tight threshold): KS slots per
    // sphere; a sphere whose surface stays farther than the threshold is
    // skipped (its candidates and witness lie on it, within the FP32
    // rounding of a candidate), the slots of the others are scanned by the
    // whole block
    {
      const int nds = a.misc->ndyn;
      uint32_t* list = S.stk;  // the walk stack is not in use yet (capacity >= the dynamic list)
      if (tid == 0) S.scan[0] = 0;
      __syncthreads();
      for (int d = tid; d < nds; d += kQT) {
        const float4 P = a.dyn_f4[d];
        if (cs == 0 ? !(P.w < 0.f) : !(P.w > 0.f)) {
          const float px = P.x, py = P.y, pz = P.z, pr = fabsf(P.w);
          const float dx = xf - px, dy = yf - py, dz = zf - pz;
          const float df = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
          const float E = 2.f * kRel * (df + pr + Ax + absmax3(px, py, pz)) + 2.f * 1.7320508f * eqt + 1e-30f;
          if (fabsf(df - pr) - E <= fd) {
            const int k = atomicAdd(&S.scan[0], 1);
            if (k < kQStack) list[k] = uint32_t(d);
            else atomicOr(&a.misc->err, 2u);  // the dynamic list is capped below kQStack
          }
        }
      }
      __syncthreads();
      const int tot = min(S.scan[0], kQStack);
      __syncthreads();
      for (int base = 0; base < tot * a.KS; base += kQT) {
        const int i = base + tid;
        if (i < tot * a.KS) {
          const int64_t slot = int64_t(list[i / a.KS]) * a.KS + i % a.KS;
          if (!a.dtomb[cs][slot]) surv_filtered(a.dsurv[cs][slot]);
        }
        drain_surv();
      }
      __syncthreads();
    }
    const float slack = f_up(2.0 * 1.7320508075688772 * double(a.bc->eq) + 1e-12);
    block_walk(
        T, S, &a.misc->err, refresh_surv,
        [&](int64_t node) {
          const float db = sqrtf(box_d2(xf, yf, zf, T.lo[node], T.hi[node]));
          return db - kRel * (db + Ax) - 1e-30f - slack <= fd;
        },
        [&](int64_t leaf) {
          // a leaf's kLeaf (8) slots share one tombstone word; all loads first
          const int64_t b = leaf * kLeaf, e = min(b + kLeaf, T.nitems);
          const uint32_t tw = tomb[b >> 5] >> unsigned(b & 31);
          float4 P[kLeaf];
#pragma unroll
          for (int k = 0; k < kLeaf; ++k)
            if (b + k < e && !((tw >> k) & 1u)) P[k] = items[b + k];
#pragma unroll
          for (int k = 0; k < kLeaf; ++k)
            if (b + k < e && !((tw >> k) & 1u)) surv_filtered(P[k]);
        },
        drain_surv);
  }
  {
    double v[1] = {bd};
    uint32_t id[1] = {gbest};
    block_argmin<1>(v, id, S);
    bd = v[0];
    gbest = id[0];
  }
  flush_counts();
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
  InsSlot r;
  r.value = value;
  r.wx = wx;
  r.wy = wy;
  r.wz = wz;
  // the class stays (containment only grows; a second class makes the point
  // INVALID), so any later value is at most the nearest opposite tangent
  // distance of the class, which only falls as spheres are added
  r.R = (a.clamp_opp && have_u) ? fmax(ub, 0.0) : INFINITY;
  r.rho = code == GFS_CODE_LOWER ? INFINITY : m;
  r.arg = arg;
  r.t = int(t);
  r.flags = uint16_t(flags);
  r.insert = 1;
  r.pad = 0;
  a.slots[slot] = r;
}


// ---------------------------------------------------------------------------
// Commit test.  Step t' of the window commits when no earlier pending step t
// can change its result and it cannot change t's: the ball of t (radius at
// most R_t in any later state) and the region that decides t' (radius rho_t'
// around y_t') are disjoint with a margin.  Every interaction of two steps --
// containment, a tangent or far bound, a survivor t's ball removes, a
// candidate t adds, equal positions -- needs |y_t - y_t'| <= r_t + rho_t'.
// An earlier step that commits in the same round has its exact radius; the
// passes propagate that (pass 0 uses R for every earlier step, pass p the
// commits of pass p - 1; the committed set only grows and stays consistent).
// One warp per slot.
// ---------------------------------------------------------------------------
constexpr double kReachAbs = 1e-6;    // absolute margin of the commit test (covers tol-shifted comparisons)
constexpr double kReachRel = 1e-9;    // relative margin (FP64 rounding of the compared radii)

__global__ void __launch_bounds__(256) k_ins_conflict(InsertArgs a, int pass) {
  const int lane = threadIdx.x & 31;
  const int j = int(blockIdx.x) * 8 + (threadIdx.x >> 5);
  const int np = a.misc->npend;
  if (j >= np) return;
  const unsigned char* prev = a.cbuf + (pass & 1) * a.wcap;
  unsigned char* cur = a.cbuf + ((pass + 1) & 1) * a.wcap;
  const InsSlot& sj = a.slots[j];
  const double yx = a.y[3 * int64_t(sj.t)], yy = a.y[3 * int64_t(sj.t) + 1], yz = a.y[3 * int64_t(sj.t) + 2];
  const double rho = sj.rho;
  bool blocked = false;
  for (int i = lane; i < j && !blocked; i += 32) {
    const InsSlot& si = a.slots[i];
    double r;
    if (pass > 0 && prev[i]) r = si.insert ? fabs(si.value) : -1.0;  // committed: its exact radius
    else r = si.R;                                                   // pending: a bound
    if (r < 0.0) continue;                                           // never inserts
    if (!(rho < INFINITY) || !(r < INFINITY)) {
      blocked = true;
      continue;
    }
    const double* yi = a.y + 3 * int64_t(si.t);
    const double dx = yi[0] - yx, dy = yi[1] - yy, dz = yi[2] - yz;
    // decided in FP32 when the distance is clear of the threshold by far more
    // than the FP32 rounding (GB300 issues FP64 at a small fraction of the
    // FP32 rate), else in FP64
    const double lim = r + rho + kReachAbs;
    const float d2f = float(dx) * float(dx) + float(dy) * float(dy) + float(dz) * float(dz);
    const float limf = float(lim);
    if (d2f > 1.0001f * limf * limf + 1e-30f) continue;
    if (d2f < 0.9999f * limf * limf) {
      blocked = true;
      continue;
    }
    const double d = sqrt(dx * dx + dy * dy + dz * dz);
    if (d <= lim + kReachRel * (d + r + rho)) blocked = true;
  }
  blocked = __any_sync(0xffffffffu, blocked);
  if (lane == 0) cur[j] = blocked ? 0 : 1;
}

// Commit: results of the committed slots go to the outputs; the ones that
// insert get their sphere (provisional index n0 + t), witness and counters;
// the uncommitted slots are compacted in step order and the window is refilled
// with the next steps up to wnext slots.  One block of 1024 threads.
constexpr int kCT = 1024;
constexpr int kCPer = 4;  // slots per thread: window capacity <= kCT * kCPer

__global__ void __launch_bounds__(kCT) k_ins_commit(InsertArgs a, int passes, int wnext) {
  __shared__ int s_scan[kCT / 32];
  __shared__ int s_tot[2];
  InsMisc* M = a.misc;
  const int np = M->npend;
  const unsigned char* dec = a.cbuf + (passes & 1) * a.wcap;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  // per thread: kCPer consecutive slots
  int keep_cnt = 0, new_cnt = 0;
  int ts[kCPer];
  unsigned char cm[kCPer];
#pragma unroll
  for (int q = 0; q < kCPer; ++q) {
    const int j = tid * kCPer + q;
    cm[q] = 0;
    ts[q] = -1;
    if (j < np) {
      ts[q] = a.slot_t[j];
      cm[q] = dec[j];
      if (!cm[q]) ++keep_cnt;
      else if (a.slots[j].insert) ++new_cnt;
    }
  }
  // block exclusive scans of (kept, new)
  auto scan = [&](int v, int which) {
    int pre = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, pre, o);
      if (lane >= o) pre += u;
    }
    if (lane == 31) s_scan[w] = pre;
    __syncthreads();
    if (w == 0) {
      int x = lane < kCT / 32 ? s_scan[lane] : 0;
      int incl = x;
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
      }
      if (lane < kCT / 32) s_scan[lane] = incl - x;
      if (lane == 31) s_tot[which] = incl;
    }
    __syncthreads();
    const int base = s_scan[w] + pre - v;
    __syncthreads();
    return base;
  };
  int kb = scan(keep_cnt, 0);
  int nb = scan(new_cnt, 1);
  const int kept = s_tot[0], nnew = s_tot[1];
  const int ndyn = M->ndyn;
  // slots are rewritten below: read everything first
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kCPer; ++q) {
    const int j = tid * kCPer + q;
    if (j >= np) continue;
    if (!cm[q]) {
      a.slot_t[kb++] = ts[q];  // kb <= j: compaction never overtakes an unread slot of this thread
      continue;
    }
    const InsSlot r = a.slots[j];
    const int64_t t = r.t;
    if (a.s_out) a.s_out[t] = r.value;
    if (a.arg_out) a.arg_out[t] = r.arg;
    if (a.fl_out) a.fl_out[t] = r.flags;
    a.inserted[t] = r.insert;
    a.codes[t] = uint8_t(r.flags & 15);
    if (r.insert) {
      const int o = a.n0 + int(t);
      a.sph64[o] = D4{a.y[3 * t], a.y[3 * t + 1], a.y[3 * t + 2], r.value};
      a.witness64[3 * int64_t(o)] = r.wx;
      a.witness64[3 * int64_t(o) + 1] = r.wy;
      a.witness64[3 * int64_t(o) + 2] = r.wz;
      a.counts[o] = 0;
      a.maxrem[o] = -1;
      a.new_ids[nb] = o;
      a.dyn_ids_w[ndyn + nb] = o;
      float w32 = float(r.value);
      if (w32 == 0.f && r.value != 0.0) w32 = copysignf(1.4e-45f, float(r.value));  // keep the sign class
      a.dyn_f4[ndyn + nb] = make_float4(float(a.y[3 * t]), float(a.y[3 * t + 1]), float(a.y[3 * t + 2]), w32);
      ++nb;
    }
  }
  __syncthreads();
  // refill the window with the next steps, in order
  const int next = M->next;
  const int64_t room = int64_t(max(wnext, kept)) - kept;
  const int fill = int(min(room, a.T - int64_t(next)));
  for (int q = tid; q < fill; q += kCT) a.slot_t[kept + q] = next + q;
  if (tid == 0) {
    M->ncommit = np - kept;
    M->nnew = nnew;
    M->ndyn = ndyn + nnew;
    M->ninserted += nnew;
    M->npend = kept + fill;
    M->next = next + fill;
    M->ndyn_start = ndyn;
    M->nlost = 0;
  }
}

cudaError_t launch_ins_query(const InsertArgs& a, int nslots, cudaStream_t st) {
  if (nslots > 0) {
    k_ins_query<<<nslots, kQT, 0, st>>>(a);
    ++g_insert_launches;
  }
  return cudaGetLastError();
}

cudaError_t launch_ins_commit(const InsertArgs& a, int nslots, int passes, int wnext, cudaStream_t st) {
  if (nslots > 0) {
    for (int p = 0; p < passes; ++p) k_ins_conflict<<<(nslots + 7) / 8, 256, 0, st>>>(a, p);
    g_insert_launches += passes;
  }
  k_ins_commit<<<1, kCT, 0, st>>>(a, passes, wnext);
  ++g_insert_launches;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// State update for the spheres a round inserted.
// ---------------------------------------------------------------------------
constexpr int kUStack = 2048;  // per-warp walk stack entries (plus a reserve of kFan)
constexpr int kNear = 1024;    // per new sphere: dynamic-list spheres that reach it


// A survivor covered by a new ball: tombstone it (once), count it off its
// sphere, remember the largest step that removed one of the sphere's
// survivors and list the sphere when its last survivor goes.
__device__ void ins_kill(const InsertArgs& a, int cls, const float4& P, bool dyn, int64_t j, const D4& nw, int step,
                         float nxf, float nyf, float nzf, float An, float eqt, float rkill) {
  const double tol = a.tol;
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
  const int sph = int(g / uint32_t(a.KS));
  if (cls == 1 && a.sph64[sph].w == 0.0) return;
  atomicMax(a.maxrem + sph, step);
  if (atomicSub(a.counts + sph, 1) == 1) {
    const unsigned k = atomicAdd(&a.misc->nlost, 1u);
    a.lost_list[k] = sph;
  }
}

// Survivors in the hierarchies covered by a new ball: one block per new
// sphere, warps 0 and 1 walk the two class hierarchies.
__global__ void __launch_bounds__(64) k_ins_kill_static(InsertArgs a) {
  __shared__ uint32_t s_stk[2][kUStack + kFan];
  const int lane = threadIdx.x & 31, cls = threadIdx.x >> 5;
  const int o = a.new_ids[blockIdx.x];
  const D4 nw = a.sph64[o];
  const int step = o - a.n0;
  const double rn = fabs(nw.w);
  const float nxf = float(nw.x), nyf = float(nw.y), nzf = float(nw.z);
  const float An = absmax3(nxf, nyf, nzf);
  const float eqt = float(a.bc->eq);
  const float reach = f_up(rn - a.tol + 2.0 * 1.7320508075688772 * double(eqt) + 1e-9);
  const float rkill = f_up(rn - a.tol);
  const Tree& T = a.vt[cls];
  warp_walk_until(
      T, s_stk[cls], kUStack, lane, &a.misc->err, [&]() { return true; },
      [&](int64_t node) {
        const float db = sqrtf(box_d2(nxf, nyf, nzf, T.lo[node], T.hi[node]));
        return db - kRel * (db + An) - 1e-30f < reach;
      },
      [&](int64_t leaf) {
        const int64_t b = leaf * kLeaf, e = min(b + kLeaf, T.nitems);
        for (int64_t j = b; j < e; ++j)
          if (!tombed(a.tomb[cls], j)) ins_kill(a, cls, a.surv[cls][j], false, j, nw, step, nxf, nyf, nzf, An, eqt,
                                                rkill);
      });
}

// Survivors of the spheres inserted since the rebuild (before this round)
// covered by a new ball: one warp per such sphere, its KS slots scanned for
// every new ball that reaches its surface.
__global__ void __launch_bounds__(256) k_ins_kill_dynamic(InsertArgs a) {
  const int lane = threadIdx.x & 31;
  const int d = int(blockIdx.x) * 8 + (threadIdx.x >> 5);
  if (d >= a.misc->ndyn_start) return;
  const int nnew = a.misc->nnew, base = a.misc->ndyn_start;
  const float4 Pf = a.dyn_f4[d];
  const float eqt = float(a.bc->eq);
  for (int b = 0; b < nnew; ++b) {
    // a point of sphere d (or its witness) in the shrunk new ball needs
    // |p_new - p_d| < r_new + r_d; FP32 with a margin far above its rounding
    const float4 Nf = a.dyn_f4[base + b];
    const float dx = Nf.x - Pf.x, dy = Nf.y - Pf.y, dz = Nf.z - Pf.z;
    const float lim = (fabsf(Nf.w) + fabsf(Pf.w)) * 1.0001f + 1e-5f;
    if (!(dx * dx + dy * dy + dz * dz < lim * lim)) continue;
    const int o = a.new_ids[b];
    const D4 nw = a.sph64[o];
    const float nxf = float(nw.x), nyf = float(nw.y), nzf = float(nw.z);
    const float An = absmax3(nxf, nyf, nzf);
    const float rkill = f_up(fabs(nw.w) - a.tol);
    for (int cls = 0; cls < 2; ++cls) {
      if (!(cls == 0 ? !(Pf.w < 0.f) : !(Pf.w > 0.f))) continue;
      for (int k = lane; k < a.KS; k += 32) {
        const int64_t slot = int64_t(d) * a.KS + k;
        if (!a.dtomb[cls][slot])
          ins_kill(a, cls, a.dsurv[cls][slot], true, slot, nw, o - a.n0, nxf, nyf, nzf, An, eqt, rkill);
      }
    }
  }
}

// For each new sphere, the spheres of the dynamic list whose ball reaches its
// surface (the only ones of that list that can cover its candidates and
// witness): |p_d - p_new| < r_d + r_new, in FP32 with a margin far above its
// rounding.  One block per new sphere; more than kNear entries: the list is
// marked full (the cull then scans the whole dynamic list).
__global__ void __launch_bounds__(256) k_ins_dyn_near(InsertArgs a) {
  __shared__ int s_cnt;
  const int which = blockIdx.x;
  const int me = a.misc->ndyn_start + which;
  const float4 N = a.dyn_f4[me];
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  const int ndyn = a.misc->ndyn;
  int* L = a.near_list + int64_t(which) * kNear;
  for (int d = threadIdx.x; d < ndyn; d += blockDim.x) {
    if (d == me) continue;
    const float4 P = a.dyn_f4[d];
    const float dx = P.x - N.x, dy = P.y - N.y, dz = P.z - N.z;
    const float lim = (fabsf(P.w) + fabsf(N.w)) * 1.0001f + 1e-5f;
    if (dx * dx + dy * dy + dz * dz < lim * lim) {
      const int k = atomicAdd(&s_cnt, 1);
      if (k < kNear) L[k] = d;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) a.near_cnt[which] = s_cnt;
}

// The new spheres' candidates and witnesses, culled against every other
// sphere: one warp per (new sphere, candidate), a warp-parallel walk of the
// sphere hierarchy that stops at the first covering ball (FP32 decisions
// where provably away from the boundary, FP64 otherwise), then the spheres
// inserted since the rebuild.  Survivors join the dynamic lists.
__global__ void __launch_bounds__(128) k_ins_cull_new(InsertArgs a) {
  __shared__ uint32_t s_stk[4][kUStack + kFan];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint32_t* stk = s_stk[wib];
  const int KS = a.KS;
  const int per = (KS + 3) / 4;
  const int which = int(blockIdx.x) / per;
  const int k = (int(blockIdx.x) % per) * 4 + wib;
  if (k >= KS) return;
  const int jn = a.new_ids[which];
  const D4 nw = a.sph64[jn];
  const int64_t slot = int64_t(a.misc->ndyn_start + which) * KS + k;
  const double tol = a.tol;
  const float ntol_up = f_up(-tol), ntol_dn = f_dn(-tol);
  double qx, qy, qz;
  if (k < a.K) {
    ex_cand(nw, a.U64[3 * k], a.U64[3 * k + 1], a.U64[3 * k + 2], qx, qy, qz);
  } else {
    qx = a.witness64[3 * int64_t(jn)];
    qy = a.witness64[3 * int64_t(jn) + 1];
    qz = a.witness64[3 * int64_t(jn) + 2];
  }
  if (a.box_cull && !ex_inbox(qx, qy, qz)) {
    if (lane == 0) a.dtomb[0][slot] = a.dtomb[1][slot] = 1u;
    return;
  }
  const float qxf = float(qx), qyf = float(qy), qzf = float(qz);
  const float Aq = absmax3(qxf, qyf, qzf);
  // FP32 filter of "q is in the ball of sphere o shrunk by tol": decided in
  // FP32 when |d - r| is provably away from tol (E bounds the rounding of q
  // and p to FP32, of the distance and of r), else by the exact predicate
  auto covered_by = [&](const float4& Pf, int o) {
    if (o == jn) return false;
    const float dx = qxf - Pf.x, dy = qyf - Pf.y, dz = qzf - Pf.z;
    const float df = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    const float r = fabsf(Pf.w);
    const float E = kRel * (df + r + Aq + absmax3(Pf.x, Pf.y, Pf.z)) + 1e-30f;
    if (df - r - E >= ntol_up) return false;
    if (df - r + E < ntol_dn) return true;
    return ex_cov(qx, qy, qz, a.sph64[o], tol);
  };
  bool covered = false;
  // the spheres of the dynamic list that reach the new sphere (its list
  // from k_ins_dyn_near, or all of them when the list overflowed)
  const int nnear = a.near_cnt[which];
  if (nnear <= kNear) {
    const int* L = a.near_list + int64_t(which) * kNear;
    for (int q = lane; q < nnear && !covered; q += 32)
      if (covered_by(a.dyn_f4[L[q]], a.dyn_ids[L[q]])) covered = true;
  } else {
    const int ndyn = a.misc->ndyn;
    for (int q = lane; q < ndyn && !covered; q += 32)
      if (covered_by(a.dyn_f4[q], a.dyn_ids[q])) covered = true;
  }
  warp_walk_until(
      a.st, stk, kUStack, lane, &a.misc->err, [&]() { return !__any_sync(kAll, covered); },
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
  if (lane == 0) {
    const uint32_t g = uint32_t(jn) * uint32_t(KS) + uint32_t(k);
    const float4 item = make_float4(qxf, qyf, qzf, __uint_as_float(g));
    for (int c = 0; c < 2; ++c) {
      const bool mine = c == 0 ? !(nw.w < 0.0) : !(nw.w > 0.0);
      if (mine && !covered) a.dsurv[c][slot] = item;
      a.dtomb[c][slot] = (mine && !covered) ? 0u : 1u;
    }
    if (!covered) atomicAdd(a.counts + jn, 1);
  }
}

// LOST_WITNESS: a sphere whose last survivor went this round marks the largest
// step that removed one of its survivors (the step after which, in step
// order, it had none).
__global__ void k_ins_lost(InsertArgs a) {
  const unsigned n = a.misc->nlost;
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const int step = a.maxrem[a.lost_list[q]];
    // every writer of a step's word in this launch stores the same value
    if (step >= 0 && a.fl_out) a.fl_out[step] = uint16_t(a.fl_out[step] | GFS_FLAG_LOST_WITNESS);
  }
}

cudaError_t launch_ins_update(const InsertArgs& a, int nnew, int ndyn_start, cudaStream_t st) {
  if (nnew <= 0) return cudaSuccess;
  k_ins_kill_static<<<nnew, 64, 0, st>>>(a);
  // survivors of the spheres inserted before this round since the rebuild
  if (ndyn_start > 0) k_ins_kill_dynamic<<<(ndyn_start + 7) / 8, 256, 0, st>>>(a);
  k_ins_dyn_near<<<nnew, 256, 0, st>>>(a);
  k_ins_cull_new<<<nnew * ((a.KS + 3) / 4), 128, 0, st>>>(a);
  k_ins_lost<<<64, 256, 0, st>>>(a);
  g_insert_launches += ndyn_start > 0 ? 5 : 4;
  return cudaGetLastError();
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

// Consecutive numbering of the inserted spheres: step t's sphere (provisional
// index n0 + t) becomes n0 + newid[t], newid the exclusive prefix count of
// inserted steps.  Spheres and witnesses are copied to the new numbering and
// the argmins of the outputs renumbered.
__global__ void k_ins_renumber(InsertArgs a, const int* __restrict__ newid, D4* __restrict__ sph_out,
                               double* __restrict__ wit_out) {
  const int64_t total = int64_t(a.n0) + a.T;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    if (i < a.n0) {
      sph_out[i] = a.sph64[i];
      wit_out[3 * i] = a.witness64[3 * i];
      wit_out[3 * i + 1] = a.witness64[3 * i + 1];
      wit_out[3 * i + 2] = a.witness64[3 * i + 2];
      continue;
    }
    const int64_t t = i - a.n0;
    if (a.inserted[t]) {
      const int64_t o = a.n0 + newid[t];
      sph_out[o] = a.sph64[i];
      wit_out[3 * o] = a.witness64[3 * i];
      wit_out[3 * o + 1] = a.witness64[3 * i + 1];
      wit_out[3 * o + 2] = a.witness64[3 * i + 2];
    }
    if (a.arg_out) {
      const int code = a.codes[t];
      const int64_t g = a.arg_out[t];
      if (code == GFS_CODE_SURVIVOR) {
        const int64_t sph = g / a.KS;
        if (sph >= a.n0) a.arg_out[t] = (a.n0 + newid[sph - a.n0]) * int64_t(a.KS) + g % a.KS;
      } else if ((code == GFS_CODE_OPPOSITE || code == GFS_CODE_LOWER || code == GFS_CODE_SAMPLE) && g >= a.n0) {
        a.arg_out[t] = a.n0 + newid[g - a.n0];
      }
    }
  }
}

__global__ void k_ins_remap_survivors(float4* __restrict__ items, unsigned n, const int* __restrict__ newid, int n0,
                                      int KS) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const uint32_t g = __float_as_uint(items[t].w);
  const uint32_t sph = g / uint32_t(KS);
  if (sph >= uint32_t(n0))
    items[t].w = __uint_as_float(uint32_t(n0 + newid[sph - n0]) * uint32_t(KS) + g % uint32_t(KS));
}

__global__ void k_gather_d4(const D4* __restrict__ src, const int* __restrict__ ids, int64_t n, D4* __restrict__ dst) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    dst[i] = src[ids[i]];
}

__global__ void k_remap_sid(int* __restrict__ sid, const int* __restrict__ ids, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    sid[i] = ids[sid[i]];
}

namespace {
unsigned grid_for(int64_t n, int bs) {
  const int64_t g = (n + bs - 1) / bs;
  return unsigned(g < 1 ? 1 : (g > 65535 ? 65535 : g));
}
}  // namespace

cudaError_t launch_ins_counts(const float4* s0, unsigned n0, const float4* s1, unsigned n1, const D4* sph64, int KS,
                              int* counts, cudaStream_t st) {
  if (n0 + n1 == 0) return cudaSuccess;
  k_ins_counts<<<(n0 + n1 + 255) / 256, 256, 0, st>>>(s0, n0, s1, n1, sph64, KS, counts);
  ++g_insert_launches;
  return cudaGetLastError();
}

cudaError_t launch_ins_compact(const float4* ssurv, const uint32_t* tomb, unsigned ns, const float4* dsurv,
                               const uint32_t* dtomb, unsigned nd, float4* out, unsigned* count, cudaStream_t st) {
  if (ns + nd == 0) return cudaSuccess;
  k_ins_compact<<<(ns + nd + 255) / 256, 256, 0, st>>>(ssurv, tomb, ns, dsurv, dtomb, nd, out, count);
  ++g_insert_launches;
  return cudaGetLastError();
}

cudaError_t launch_ins_renumber(const InsertArgs& a, const int* newid, D4* sph_out, double* wit_out,
                                cudaStream_t st) {
  k_ins_renumber<<<grid_for(int64_t(a.n0) + a.T, 256), 256, 0, st>>>(a, newid, sph_out, wit_out);
  ++g_insert_launches;
  return cudaGetLastError();
}

cudaError_t launch_ins_remap_survivors(float4* items, unsigned n, const int* newid, int n0, int KS, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_ins_remap_survivors<<<(n + 255) / 256, 256, 0, st>>>(items, n, newid, n0, KS);
  ++g_insert_launches;
  return cudaGetLastError();
}

cudaError_t exclusive_scan_i32(void* temp, size_t& bytes, const int* in, int* out, int64_t n,
                              cudaStream_t st) {
  return cub::DeviceScan::ExclusiveSum(temp, bytes, in, out, int(n), st);
}

cudaError_t launch_gather_d4(const D4* src, const int* ids, int64_t n, D4* dst, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_gather_d4<<<grid_for(n, 256), 256, 0, st>>>(src, ids, n, dst);
  ++g_insert_launches;
  return cudaGetLastError();
}

cudaError_t launch_remap_sid(int* sid, const int* ids, int64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_remap_sid<<<grid_for(n, 256), 256, 0, st>>>(sid, ids, n);
  ++g_insert_launches;
  return cudaGetLastError();
}

}  // namespace gfs
