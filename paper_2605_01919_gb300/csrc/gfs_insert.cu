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
//   k_ins_query  -- one warp evaluates the value at y_t exactly (FP64, the
//                   oracle's expressions and tie rules), with a warp-parallel
//                   walk of the hierarchies (32 nodes per round);
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
constexpr int kQStack = 4096;

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

// lexicographic (value, index) minimum across the warp
__device__ __forceinline__ void warp_min_vi(double& v, int& idx) {
  for (int o = 16; o > 0; o >>= 1) {
    const double v2 = __shfl_xor_sync(kAll, v, o);
    const int i2 = __shfl_xor_sync(kAll, idx, o);
    if (v2 < v || (v2 == v && i2 < idx)) {
      v = v2;
      idx = i2;
    }
  }
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
__device__ __forceinline__ double warp_min_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(kAll, v, o));
  return v;
}

// Warp-parallel walk: pops up to 32 nodes per round (one per lane), lets the
// caller expand each, and pushes the children the caller marks.
template <class Refresh, class NeedChild, class Leaf>
__device__ void warp_walk(const Tree& T, uint32_t* stk, int lane, unsigned* err, Refresh refresh, NeedChild need_child,
                          Leaf leaf) {
  if (T.nlevels == 0) return;
  const int top = T.nlevels - 1;
  int sp = int(T.count[top]);
  if (lane < sp) stk[lane] = pack_node(top, lane);
  __syncwarp();
  while (sp > 0) {
    const int take = min(sp, 32);
    const uint32_t nd = lane < take ? stk[sp - 1 - lane] : 0xffffffffu;
    sp -= take;
    __syncwarp();
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
    int pre = cnt;
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(kAll, pre, o);
      if (lane >= o) pre += v;
    }
    const int total = __shfl_sync(kAll, pre, 31);
    pre -= cnt;
    if (sp + total > kQStack) {
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

// Greedy descent to the leaf whose box is nearest to (x, y, z) (uniform
// across the warp); used to seed the pruning thresholds of a walk.
__device__ int64_t nearest_leaf(const Tree& T, double x, double y, double z) {
  int lev = T.nlevels - 1;
  int64_t best = 0;
  double bd = INFINITY;
  for (int64_t j = 0; j < T.count[lev]; ++j) {
    const double d = box_d2_64(x, y, z, T.lo[T.offset[lev] + j], T.hi[T.offset[lev] + j]);
    if (d < bd) {
      bd = d;
      best = j;
    }
  }
  while (lev > 0) {
    const int64_t cb = best * kFan, ce = min(cb + kFan, T.count[lev - 1]);
    const int64_t off = T.offset[lev - 1];
    bd = INFINITY;
    for (int64_t c = cb; c < ce; ++c) {
      const double d = box_d2_64(x, y, z, T.lo[off + c], T.hi[off + c]);
      if (d < bd) {
        bd = d;
        best = c;
      }
    }
    --lev;
  }
  return best;
}

}  // namespace

__global__ void __launch_bounds__(32) k_ins_query(InsertArgs a, int64_t t) {
  __shared__ uint32_t stk[kQStack];
  const int lane = threadIdx.x;
  const double x = a.y[3 * t], y = a.y[3 * t + 1], z = a.y[3 * t + 2];
  const double tol = a.tol;
  const int n_total = *a.n_total;
  // ---- spheres: sample, containment, nearest tangent per class, far bound
  bool cov[2] = {false, false};
  double bestA[2] = {INFINITY, INFINITY};
  int idxA[2] = {INT_MAX, INT_MAX};
  double bestF = INFINITY;
  int sample = INT_MAX;
  double thA[2] = {INFINITY, INFINITY}, thF = INFINITY;
  bool covw[2] = {false, false};
  auto sphere_item = [&](int o) {
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
  };
  // seed the thresholds with the spheres of the nearest leaf
  if (a.st.nlevels > 0) {
    const int64_t nl = nearest_leaf(a.st, x, y, z);
    const int64_t j = nl * kLeaf + lane;
    if (lane < kLeaf && j < a.st.nitems) sphere_item(a.sid[j]);
  }
  warp_walk(
      a.st, stk, lane, a.err,
      [&]() {
        thA[0] = warp_min_d(bestA[0]);
        thA[1] = warp_min_d(bestA[1]);
        thF = warp_min_d(bestF);
        covw[0] = __any_sync(kAll, cov[0]);
        covw[1] = __any_sync(kAll, cov[1]);
      },
      [&](int64_t node) {
        const float4 L = a.st.lo[node], H = a.st.hi[node];
        if (x >= double(L.x) && x <= double(H.x) && y >= double(L.y) && y <= double(H.y) && z >= double(L.z) &&
            z <= double(H.z))
          return true;
        const float4 Bs[2] = {a.st.bp[node], a.st.bn[node]};
        for (int c = 0; c < 2; ++c) {
          if (!(Bs[c].w > -INFINITY)) continue;
          double th = thA[c];
          if (!covw[c]) th = fmax(th, -tol);
          const double tt = (th + double(Bs[c].w)) * (1.0 + 1e-12) + 1e-12;
          if (tt > 0.0 && ball_d2_64(x, y, z, Bs[c]) <= tt * tt) return true;
        }
        const float4 B = a.st.bf[node];
        const double tt = (thF + double(B.w)) * (1.0 + 1e-12) + 1e-12;
        return tt > 0.0 && ball_d2_64(x, y, z, B) <= tt * tt;
      },
      [&](int64_t leaf) {
        const int64_t b = leaf * kLeaf, e = min(b + kLeaf, a.st.nitems);
        for (int64_t j = b; j < e; ++j) sphere_item(a.sid[j]);
      });
  for (int o = a.n_static + lane; o < n_total; o += 32) sphere_item(o);
  cov[0] = __any_sync(kAll, cov[0]);
  cov[1] = __any_sync(kAll, cov[1]);
  warp_min_vi(bestA[0], idxA[0]);
  warp_min_vi(bestA[1], idxA[1]);
  bestF = warp_min_d(bestF);
  for (int o = 16; o > 0; o >>= 1) sample = min(sample, __shfl_xor_sync(kAll, sample, o));
  int code = -1;
  double value = 0.0;
  int64_t arg = -1;
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
  if (code >= 0) {
    if (lane == 0) {
      if (a.s_out) a.s_out[t] = value;
      if (a.arg_out) a.arg_out[t] = arg;
      if (a.fl_out) a.fl_out[t] = uint16_t(code);
      a.rec->insert = 0;
    }
    return;
  }
  const int cs = cov[0] ? 0 : 1, co = 1 - cs;
  // ---- nearest live survivor of x's class ----------------------------------
  double bd = INFINITY;
  uint32_t gbest = 0xffffffffu;
  double thd = INFINITY;
  const double slack = 2.0 * 1.7320508075688772 * double(a.bc->eq) + 1e-12;
  auto surv_item = [&](const float4& P) {
    const uint32_t g = __float_as_uint(P.w);
    double qx, qy, qz;
    surv64(a, g, qx, qy, qz);
    const double d2 = ex_d2(x, y, z, qx, qy, qz);
    if (d2 < bd || (d2 == bd && g < gbest)) {
      bd = d2;
      gbest = g;
    }
  };
  {
    const Tree& T = a.vt[cs];
    const float4* items = a.surv[cs];
    const uint32_t* tomb = a.tomb[cs];
    // seed with the live survivors of the nearest leaf
    if (T.nlevels > 0) {
      const int64_t nl = nearest_leaf(T, x, y, z);
      const int64_t j = nl * kLeaf + lane;
      if (lane < kLeaf && j < T.nitems && !tombed(tomb, j)) surv_item(items[j]);
    }
    warp_walk(
        T, stk, lane, a.err, [&]() { thd = warp_min_d(bd); },
        [&](int64_t node) {
          const double tt = sqrt(thd) * (1.0 + 1e-12) + slack;
          return box_d2_64(x, y, z, T.lo[node], T.hi[node]) <= tt * tt;
        },
        [&](int64_t leaf) {
          const int64_t b = leaf * kLeaf, e = min(b + kLeaf, T.nitems);
          for (int64_t j = b; j < e; ++j)
            if (!tombed(tomb, j)) surv_item(items[j]);
        });
    const unsigned nd = a.dcount_start[cs];
    for (unsigned j = lane; j < nd; j += 32)
      if (!a.dtomb[cs][j]) surv_item(a.dsurv[cs][j]);
  }
  warp_min_vu(bd, gbest);
  const bool have_s = gbest != 0xffffffffu, have_u = idxA[co] != INT_MAX;
  const double ds = have_s ? __dsqrt_rn(bd) : INFINITY;
  const double ub = have_u ? bestA[co] : INFINITY;
  const double lb = -bestA[cs];
  double m;
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
  value = cs == 0 ? m : -m;
  if (lane == 0) {
    if (a.s_out) a.s_out[t] = value;
    if (a.arg_out) a.arg_out[t] = arg;
    if (a.fl_out) a.fl_out[t] = uint16_t(flags);
    // witness: the point that set the value
    double wx, wy, wz;
    if (code == GFS_CODE_SURVIVOR) {
      surv64(a, gbest, wx, wy, wz);
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
}

// Cull the new sphere's candidates and witness; tombstone covered survivors.
// Blocks [0, nc) hold one warp per candidate (k = 0..K, k = K the witness):
// a warp-parallel exact walk of the sphere hierarchy that stops at the first
// covering ball.  The last block walks both survivor hierarchies with the new
// ball (warps 0, 1) and scans the lists added since the rebuild (warps 2, 3).
// The block that finishes last sets LOST_WITNESS and opens the next step.
constexpr int kUStack = 2048;

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
          bool covered = false;
          for (int o = a.n_static + lane; o < jn && !covered; o += 32)
            if (ex_cov(qx, qy, qz, a.sph64[o], tol)) covered = true;
          warp_walk_until(
              a.st, stk, kUStack, lane, a.err, [&]() { return !__any_sync(kAll, covered); },
              [&](int64_t node) {
                const float4 Bs[2] = {a.st.bp[node], a.st.bn[node]};
                for (int cl = 0; cl < 2; ++cl) {
                  const double rr = (double(Bs[cl].w) - tol) * (1.0 + 1e-12) + 1e-12;
                  if (rr > 0.0 && ball_d2_64(qx, qy, qz, Bs[cl]) < rr * rr) return true;
                }
                return false;
              },
              [&](int64_t leaf) {
                const int64_t b = leaf * kLeaf, e = min(b + kLeaf, a.st.nitems);
                for (int64_t j = b; j < e && !covered; ++j)
                  if (ex_cov(qx, qy, qz, a.sph64[a.sid[j]], tol)) covered = true;
              });
          covered = __any_sync(kAll, covered);
          if (!covered && lane == 0) {
            const uint32_t g = uint32_t(jn) * uint32_t(KS) + uint32_t(k);
            const float4 item = make_float4(float(qx), float(qy), float(qz), __uint_as_float(g));
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
      const double reach = rn + 2.0 * 1.7320508075688772 * double(a.bc->eq) + 1e-9;
      auto kill = [&](int cls, const float4& P, bool dyn, int64_t j) {
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
      if (wib < 2) {
        const int cls = wib;
        const Tree& T = a.vt[cls];
        warp_walk_until(
            T, stk, kUStack, lane, a.err, [&]() { return true; },
            [&](int64_t node) {
              const double rr = reach * (1.0 + 1e-12);
              return box_d2_64(nw.x, nw.y, nw.z, T.lo[node], T.hi[node]) < rr * rr;
            },
            [&](int64_t leaf) {
              const int64_t b = leaf * kLeaf, e = min(b + kLeaf, T.nitems);
              for (int64_t j = b; j < e; ++j) kill(cls, a.surv[cls][j], false, j);
            });
      } else {
        const int cls = wib - 2;
        const unsigned nd = a.dcount_start[cls];
        for (unsigned j = lane; j < nd; j += 32) kill(cls, a.dsurv[cls][j], true, j);
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
  k_ins_query<<<1, 32, 0, st>>>(a, t);
  k_ins_update<<<(a.KS + 3) / 4 + 1, 128, 0, st>>>(a, t);
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
