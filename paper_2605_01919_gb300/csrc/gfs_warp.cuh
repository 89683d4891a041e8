// Warp-cooperative hierarchy walk shared by the GPU kernels (device code
// only: it uses warp intrinsics).
#pragma once

#include "gfs_internal.cuh"

namespace gfs {

// A warp's walk over a hierarchy with one stack stk of cap (+ kFan)
// entries: each round refresh() runs on every lane (false ends the walk),
// then the lanes take up to 32 nodes off the stack (at most (cap - sp) /
// kFan, at least one, so the stack stays below cap + kFan); a lane calls
// leaf(index) for a leaf and need_child(node) for each child of an inner
// node, and the children it needs are pushed in lane order.  The lanes must
// enter together; *err gets bit 0 if the stack guard ever trips (it cannot,
// by the bound above).
template <class Refresh, class NeedChild, class Leaf>
__device__ void warp_walk_until(const Tree& T, uint32_t* stk, int cap, int lane, unsigned* err, Refresh refresh,
                                NeedChild need_child, Leaf leaf) {
  const unsigned kWarpAll = 0xffffffffu;
  if (T.nlevels == 0) return;
  const int top = T.nlevels - 1;
  int sp = int(T.count[top]);
  if (lane < sp) stk[lane] = pack_node(top, lane);
  __syncwarp();
  while (sp > 0) {
    if (!refresh()) return;
    const int take = min(min(sp, 32), max(1, (cap - sp) / kFan));
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
      const int v = __shfl_up_sync(kWarpAll, pre, o);
      if (lane >= o) pre += v;
    }
    const int total = __shfl_sync(kWarpAll, pre, 31);
    pre -= cnt;
    if (sp + total > cap + kFan) {  // cannot happen (see above); kept as a guard
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

}  // namespace gfs
