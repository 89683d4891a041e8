// Scored value of the query (Sec. 3.3): the kernel and its launchers; the
// per-point routine is in gfs_scored.cuh.
#include <cuda_runtime.h>

#include "gfs.h"
#include "gfs_scored.cuh"
#include "gfs_scored.h"

namespace gfs {

namespace {

unsigned long long g_scored_launches = 0;

__global__ void __launch_bounds__(128) k_query_scored(QueryArgs a, int box_cull, const uint32_t* __restrict__ csr_ids,
                                                      const int64_t* __restrict__ csr_off, unsigned* status) {
  const int64_t slot = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (slot >= a.m) return;
  scored::scored_one(a, box_cull, csr_ids, csr_off, a.perm ? int64_t(a.perm[slot]) : slot, status);
}

// csr_off[i] = first position of sphere i's ids in the sorted id list
__global__ void k_csr_offsets(const uint32_t* __restrict__ ids, int64_t nid, int64_t n, int KS,
                              int64_t* __restrict__ off) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i > n) return;
  const uint64_t key = uint64_t(i) * uint64_t(KS);
  int64_t lo = 0, hi = nid;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (uint64_t(ids[mid]) < key) lo = mid + 1;
    else hi = mid;
  }
  off[i] = lo;
}

}  // namespace

cudaError_t launch_query_scored(const QueryArgs& a, int box_cull, const uint32_t* csr_ids, const int64_t* csr_off,
                                unsigned* status, cudaStream_t st) {
  if (a.m == 0) return cudaSuccess;
  k_query_scored<<<unsigned((a.m + 127) / 128), 128, 0, st>>>(a, box_cull, csr_ids, csr_off, status);
  ++g_scored_launches;
  return cudaGetLastError();
}

cudaError_t launch_csr_offsets(const uint32_t* ids, int64_t nid, int64_t n, int KS, int64_t* off, cudaStream_t st) {
  k_csr_offsets<<<unsigned((n + 1 + 255) / 256), 256, 0, st>>>(ids, nid, n, KS, off);
  ++g_scored_launches;
  return cudaGetLastError();
}

unsigned long long scored_launch_count() { return g_scored_launches; }

}  // namespace gfs
