// Refinement order (Sec. 4.2): covered area ratio of grid cells, device
// routines.  A cell is sampled at sub^3 regularly spaced points (the centres
// of a sub x sub x sub split of the cell) and each point is tested for
// containment in the balls of the current samples, shrunk by tol -- the
// coverage predicate of the cull, decided in FP64.
#pragma once

#include "gfs_tangent.cuh"

namespace gfs {
namespace order {

// coordinate origin + h * (i + (a + 1/2) / sub), rounded per operation in
// this order
__device__ __forceinline__ double cell_coord(double origin, double h, int i, int a, int sub) {
  return __dadd_rn(origin, __dmul_rn(h, __dadd_rn(double(i), __ddiv_rn(__dadd_rn(double(a), 0.5), double(sub)))));
}

// Covered points among the cell's sub-points first, first + stride, ...
// (sub-point t = (a * sub + b) * sub + c for offsets a, b, c along x, y, z).
__device__ inline unsigned cell_cover_count(const QueryArgs& q, const int* cell, double ox, double oy, double oz,
                                            double h, int sub, int first, int stride) {
  unsigned cnt = 0;
  const int total = sub * sub * sub;
  for (int t = first; t < total; t += stride) {
    const int a = t / (sub * sub), b = (t / sub) % sub, c = t % sub;
    const double x = cell_coord(ox, h, cell[0], a, sub);
    const double y = cell_coord(oy, h, cell[1], b, sub);
    const double z = cell_coord(oz, h, cell[2], c, sub);
    if (tangent::covered_by_other(q, x, y, z, -1) >= 0) ++cnt;
  }
  return cnt;
}

}  // namespace order
}  // namespace gfs
