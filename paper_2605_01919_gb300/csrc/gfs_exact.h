// Launcher of the exact uncovered test per sphere (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gfs_kernels.h"

namespace gfs {

// out[i] (device, n bytes, input order): 1 uncovered, 0 covered, 2 undecided;
// witness (device, 3n doubles, or null): the uncovered point, NaN otherwise
cudaError_t launch_sphere_uncovered(const QueryArgs& a, uint8_t* out, double* witness, cudaStream_t st);

namespace exact {
// Outputs of the intersections kernel (device pointers)
struct UDOut {
  unsigned long long* cnt;  // [0] circles, [1] points found (may exceed the capacities)
  int64_t cap_c, cap_p;
  int64_t* circ;            // (i, j) per circle
  int64_t* quad;            // (i, j, m, side) per point
  double* pts;              // (x, y, z) per point
  unsigned* status;         // bit 0: a circle's certificate outgrew its capacity (taken as uncovered)
};
// The precomputed uncovered points and circles an exact minimum radius
// draws from (device pointers)
struct UDLists {
  const int64_t* quad;  // (i, j, m, side) per uncovered point
  const double* pts;    // (x, y, z) per uncovered point
  int64_t np;
  const int64_t* circ;  // (i, j) per uncovered circle
  int64_t nc;
};
}  // namespace exact

// pairs i < j of spheres with uncov != 0 that cut in a circle, as
// (i << 32) | j, appended through *count (written below cap)
cudaError_t launch_ud_pairs(const QueryArgs& a, const uint8_t* uncov, unsigned long long* pairs, int64_t cap,
                            unsigned long long* count, cudaStream_t st);
// the circles of the pairs with an uncovered point, and their uncovered
// points (unsorted, appended through o.cnt)
cudaError_t launch_intersections(const QueryArgs& a, const unsigned long long* pairs, int64_t np,
                                 const exact::UDOut& o, cudaStream_t st);
cudaError_t launch_ud_circle_keys(const int64_t* circ, int64_t nc, unsigned long long* key, cudaStream_t st);
// primary = 0: keys (m << 1) | side of quad[order[k]] (order may be null);
// primary = 1: keys (i << 32) | j; val[k] = the quad index
cudaError_t launch_ud_point_keys(const int64_t* quad, const int* order, int64_t np, int primary,
                                 unsigned long long* key, int* val, cudaStream_t st);
cudaError_t launch_ud_gather(const unsigned long long* ckey, int64_t nc, int64_t* circ_out, const int* order,
                             const int64_t* quad, const double* pts, int64_t np, int64_t* quad_out, double* pts_out,
                             cudaStream_t st);

// rmin_out[q]: the exact minimum valid radius at x[q] for sign sigma[q]
cudaError_t launch_exact_rmin(const QueryArgs& a, int box_cull, const exact::UDLists& L, const double* x,
                              const int8_t* sigma, int64_t m, double* out, cudaStream_t st);

unsigned long long exact_launch_count();

}  // namespace gfs
