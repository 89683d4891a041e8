// Exact uncovered test per sphere (Prop. 1 (ii)) and the uncovered
// intersection circles and points (Sec. 4.1): one thread per sphere.
#include <cuda_runtime.h>

#include "gfs_exact.cuh"
#include "gfs_exact.h"

namespace gfs {

namespace {

// One warp per sphere, spheres in hierarchy (Morton) order, the lanes
// sharing one certificate in shared memory: the six probe points are tested
// by lanes 0-5; then each round the lanes take the next 32 entries (n, u) of
// the members' triangular enumeration (the order of the one-thread routine),
// build their test points and test them against the members and, when no
// member holds one, against every ball; a point that no ball holds ends the
// search (the lowest lane's point is the witness), and the balls that held
// the others join the certificate in lane order (lane 0 appends).  The
// certificate is complete when every entry of its members has been tested.
constexpr int kWarpsU = 4;

__device__ __forceinline__ void decode_entry(int64_t p, int& n, int& u) {
  int64_t nn = int64_t((sqrt(8.0 * double(p) + 1.0) - 1.0) * 0.5);
  while (nn * (nn + 1) / 2 > p) --nn;
  while ((nn + 1) * (nn + 2) / 2 <= p) ++nn;
  n = int(nn);
  u = int(p - nn * (nn + 1) / 2);
}

__global__ void __launch_bounds__(32 * kWarpsU) k_sphere_uncovered(QueryArgs a, uint8_t* __restrict__ out,
                                                                  double* __restrict__ witness) {
  __shared__ int s_set[kWarpsU][exact::kMaxSet];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t jj = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  if (jj >= a.n) return;  // the same for the whole warp
  const int i = a.sid[jj];
  int* S = s_set[w];
  uint32_t stack[kStack];
  const D4 P = a.sph64[i];
  const double pi[3] = {P.x, P.y, P.z};
  const double ri = fabs(P.w);
  int res = 0;
  double wit[3] = {pi[0], pi[1], pi[2]};
  if (ri == 0.0) {
    int r = 0;
    if (lane == 0) r = tangent::covered_except_on(stack, a, P.x, P.y, P.z, i, -1, -1) >= 0 ? 0 : 1;
    res = __shfl_sync(0xffffffffu, r, 0);
  } else {
    int ns = 0;
    bool full = false;
    // lane 0 appends ball b (held a point of the sphere) when it is in N_i
    // and not yet a member; every lane learns the new count
    auto join_lanes = [&](int cand) {
      unsigned todo = __ballot_sync(0xffffffffu, cand >= 0);
      while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const int b = __shfl_sync(0xffffffffu, cand, src);
        if (lane == 0) {
          bool member = false;
          for (int u = 0; u < ns && !member; ++u) member = S[u] == b;
          if (!member && exact::meets(a, P, ri, b)) {
            if (ns == exact::kMaxSet) full = true;
            else S[ns++] = b;
          }
        }
        ns = __shfl_sync(0xffffffffu, ns, 0);
      }
      full = __shfl_sync(0xffffffffu, full ? 1 : 0, 0) != 0;
      __syncwarp();
    };
    int cand = -1;
    if (lane < 6) {
      double t[3] = {pi[0], pi[1], pi[2]};
      t[lane >> 1] = __dadd_rn(pi[lane >> 1], (lane & 1) ? -ri : ri);
      cand = tangent::covered_except_on(stack, a, t[0], t[1], t[2], i, -1, -1);
    }
    join_lanes(cand);
    if (ns == 0) {
      int k = -1;
      if (lane == 0) {
        k = exact::first_member(a, i, stack);
        if (k >= 0) S[0] = k;
      }
      k = __shfl_sync(0xffffffffu, k, 0);
      __syncwarp();
      if (k < 0) {  // N_i is empty: every point is uncovered
        res = 1;
        wit[0] = __dadd_rn(pi[0], ri);
      } else {
        ns = 1;
      }
    }
    if (ns > 0) {
      double ref[3];
      exact::circle_ref(pi, ri, ref);
      int last = -1;
      int64_t done = 0;
      while (!full) {
        const int64_t total = int64_t(ns) * (ns + 1) / 2;
        if (done >= total) break;
        const int64_t p = done + lane;
        int c[2] = {-1, -1};  // the balls that held this lane's two points
        bool found = false;
        double pts[6];
        int h_found = 0;
        if (p < total) {
          int n, u, k, m;
          decode_entry(p, n, u);
          if (exact::entry_points(a, pi, ri, ref, S, n, u, pts, k, m)) {
            for (int h = 0; h < 2 && !found; ++h) {
              const double* t = pts + 3 * h;
              if (exact::held_by_member(a, t, S, ns, k, m, last)) continue;
              const int b = tangent::covered_except_on(stack, a, t[0], t[1], t[2], i, k, m);
              if (b < 0) {
                found = true;
                h_found = h;
              } else {
                c[h] = b;
              }
            }
          }
        }
        const unsigned fb = __ballot_sync(0xffffffffu, found);
        if (fb) {
          const int src = __ffs(fb) - 1;
          for (int q = 0; q < 3; ++q) {
            const double v = found ? pts[3 * h_found + q] : 0.0;
            wit[q] = __shfl_sync(0xffffffffu, v, src);
          }
          res = 1;
          break;
        }
        done += total - done < 32 ? total - done : 32;
        join_lanes(c[0]);
        join_lanes(c[1]);
      }
      if (full && res == 0) res = 2;
    }
  }
  if (lane == 0) {
    out[i] = uint8_t(res);
    if (witness)
      for (int q = 0; q < 3; ++q)
        witness[3 * int64_t(i) + q] = res == 1 ? wit[q] : __longlong_as_double(0x7ff8000000000000ll);
  }
}

// One thread per uncovered sphere, spheres in hierarchy (Morton) order: the
// spheres after it that cut it, appended to the pair list as (i << 32) | j
// (counted only when the count exceeds the capacity).
__global__ void __launch_bounds__(128) k_ud_pairs(QueryArgs a, const uint8_t* __restrict__ uncov,
                                                  unsigned long long* __restrict__ pairs, int64_t cap,
                                                  unsigned long long* __restrict__ count) {
  const int64_t u = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (u >= a.n) return;
  const int i = a.sid[u];
  if (uncov[i] == 0) return;
  uint32_t stack[kStack];
  exact::sphere_pairs(a, i, uncov, stack, [&](int j) {
    const unsigned long long k = atomicAdd(count, 1ull);
    if (k < (unsigned long long)cap)
      pairs[k] = (static_cast<unsigned long long>(i) << 32) | static_cast<unsigned long long>(j);
  });
}

// One thread per pair: the circle's certificate and, on an uncovered circle,
// its uncovered points.
__global__ void __launch_bounds__(128) k_intersections(QueryArgs a, const unsigned long long* __restrict__ pairs,
                                                       int64_t np, exact::UDOut o) {
  const int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (k >= np) return;
  const int i = int(pairs[k] >> 32), j = int(pairs[k] & 0xffffffffull);
  int M[exact::kMaxSet];
  uint32_t stacks[2 * kStack];
  exact::circle_intersections(a, i, j, M, stacks, o);
}

// Sort keys: circles (i << 32) | j; points first by (m << 1) | side, then
// (stable) by (i << 32) | j.
__global__ void k_ud_circle_keys(const int64_t* __restrict__ circ, int64_t nc, unsigned long long* __restrict__ key) {
  const int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (k >= nc) return;
  key[k] = (static_cast<unsigned long long>(circ[2 * k]) << 32) | static_cast<unsigned long long>(circ[2 * k + 1]);
}

__global__ void k_ud_point_keys(const int64_t* __restrict__ quad, const int* __restrict__ order, int64_t np,
                                int primary, unsigned long long* __restrict__ key, int* __restrict__ val) {
  const int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (k >= np) return;
  const int64_t s = order ? order[k] : k;
  const int64_t* q = quad + 4 * s;
  key[k] = primary ? (static_cast<unsigned long long>(q[0]) << 32) | static_cast<unsigned long long>(q[1])
                   : (static_cast<unsigned long long>(q[2]) << 1) | static_cast<unsigned long long>(q[3]);
  val[k] = int(s);
}

__global__ void k_ud_gather(const unsigned long long* __restrict__ ckey, int64_t nc, int64_t* __restrict__ circ_out,
                            const int* __restrict__ order, const int64_t* __restrict__ quad,
                            const double* __restrict__ pts, int64_t np, int64_t* __restrict__ quad_out,
                            double* __restrict__ pts_out) {
  const int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (k < nc) {
    circ_out[2 * k] = int64_t(ckey[k] >> 32);
    circ_out[2 * k + 1] = int64_t(ckey[k] & 0xffffffffull);
  }
  if (k < np) {
    const int64_t s = order[k];
    for (int c = 0; c < 4; ++c) quad_out[4 * k + c] = quad[4 * s + c];
    for (int c = 0; c < 3; ++c) pts_out[3 * k + c] = pts[3 * s + c];
  }
}

// One warp per query point: the lanes split each candidate set (U, D, T in
// that order) and take the warp's minimum after each, so that later sets are
// tested against the best point so far.
__global__ void __launch_bounds__(128) k_exact_rmin(QueryArgs a, int box_cull, exact::UDLists L,
                                                   const double* __restrict__ x, const int8_t* __restrict__ sigma,
                                                   int64_t m, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t q = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  if (q >= m) return;  // the same for the whole warp
  uint32_t stack[kStack];
  const double xq[3] = {x[3 * q], x[3 * q + 1], x[3 * q + 2]};
  const int sg = sigma[q];
  double best = INFINITY;
  for (int phase = 0; phase < 3; ++phase) {
    best = exact::rmin_phase(a, box_cull, L, xq, sg, phase, lane, 32, best, stack);
    for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
  }
  if (lane == 0) out[q] = best;
}

unsigned long long g_exact_launches = 0;

}  // namespace

cudaError_t launch_exact_rmin(const QueryArgs& a, int box_cull, const exact::UDLists& L, const double* x,
                              const int8_t* sigma, int64_t m, double* out, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  k_exact_rmin<<<(unsigned int)((m + 3) / 4), 128, 0, st>>>(a, box_cull, L, x, sigma, m, out);
  ++g_exact_launches;
  return cudaGetLastError();
}

cudaError_t launch_ud_pairs(const QueryArgs& a, const uint8_t* uncov, unsigned long long* pairs, int64_t cap,
                            unsigned long long* count, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  k_ud_pairs<<<(unsigned int)((a.n + 127) / 128), 128, 0, st>>>(a, uncov, pairs, cap, count);
  ++g_exact_launches;
  return cudaGetLastError();
}

cudaError_t launch_intersections(const QueryArgs& a, const unsigned long long* pairs, int64_t np,
                                 const exact::UDOut& o, cudaStream_t st) {
  if (np <= 0) return cudaSuccess;
  k_intersections<<<(unsigned int)((np + 127) / 128), 128, 0, st>>>(a, pairs, np, o);
  ++g_exact_launches;
  return cudaGetLastError();
}

cudaError_t launch_ud_circle_keys(const int64_t* circ, int64_t nc, unsigned long long* key, cudaStream_t st) {
  if (nc <= 0) return cudaSuccess;
  k_ud_circle_keys<<<(unsigned int)((nc + 255) / 256), 256, 0, st>>>(circ, nc, key);
  ++g_exact_launches;
  return cudaGetLastError();
}

cudaError_t launch_ud_point_keys(const int64_t* quad, const int* order, int64_t np, int primary,
                                 unsigned long long* key, int* val, cudaStream_t st) {
  if (np <= 0) return cudaSuccess;
  k_ud_point_keys<<<(unsigned int)((np + 255) / 256), 256, 0, st>>>(quad, order, np, primary, key, val);
  ++g_exact_launches;
  return cudaGetLastError();
}

cudaError_t launch_ud_gather(const unsigned long long* ckey, int64_t nc, int64_t* circ_out, const int* order,
                             const int64_t* quad, const double* pts, int64_t np, int64_t* quad_out, double* pts_out,
                             cudaStream_t st) {
  const int64_t n = nc > np ? nc : np;
  if (n <= 0) return cudaSuccess;
  k_ud_gather<<<(unsigned int)((n + 255) / 256), 256, 0, st>>>(ckey, nc, circ_out, order, quad, pts, np, quad_out,
                                                                 pts_out);
  ++g_exact_launches;
  return cudaGetLastError();
}

cudaError_t launch_sphere_uncovered(const QueryArgs& a, uint8_t* out, double* witness, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  k_sphere_uncovered<<<(unsigned int)((a.n + kWarpsU - 1) / kWarpsU), 32 * kWarpsU, 0, st>>>(a, out, witness);
  ++g_exact_launches;
  return cudaGetLastError();
}

unsigned long long exact_launch_count() { return g_exact_launches; }

}  // namespace gfs
