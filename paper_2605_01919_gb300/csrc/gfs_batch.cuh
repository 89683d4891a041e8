// Batched P build and query over many independent shapes.
//
// All shapes' samples live in one array, sorted by (shape, Morton code), so
// each shape owns a contiguous range; every shape gets its own implicit
// hierarchy inside shared node arrays (a forest).  The hot kernels are
// persistent: a fixed grid of warps pulls work items -- (shape, 32 spheres,
// direction k) for the cull, (shape, 32 query points) for the query -- from a
// global counter, so shapes of very different sizes share the GPU evenly.
// Each shape is seen through a per-shape argument block ("view") whose
// pointers are offset to the shape's range and whose indices are local, so
// the per-warp code is the single-shape packet code.
// Included at the end of gfs_kernels.cu (one translation unit, so the
// per-warp packet code is shared without relocatable device code).

namespace gfs {

namespace {

constexpr unsigned kAllB = 0xffffffffu;

// segment of v in a prefix array (prefix[0] = 0, prefix[ns] = total)
__device__ __forceinline__ int find_seg(const int64_t* __restrict__ prefix, int ns, int64_t v) {
  int lo = 0, hi = ns;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= v) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint32_t morton_of(float x, float y, float z) { return morton3(x, y, z); }

}  // namespace

// inputs of all shapes into one FP64 array, Morton keys with the shape in the
// high bits, per-shape data bounds
__global__ void k_batch_copy(const ShapeDesc* __restrict__ d, const int64_t* __restrict__ off, int ns, int64_t N,
                             D4* __restrict__ sph64, unsigned long long* __restrict__ keys, int* __restrict__ vals,
                             unsigned int* __restrict__ bits) {
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < N; t += int64_t(gridDim.x) * blockDim.x) {
    const int s = find_seg(off, ns, t);
    const int64_t i = t - off[s];
    const D4 v{d[s].p[3 * i], d[s].p[3 * i + 1], d[s].p[3 * i + 2], d[s].s[i]};
    sph64[t] = v;
    keys[t] = (static_cast<unsigned long long>(s) << 32) | morton_of(float(v.x), float(v.y), float(v.z));
    vals[t] = int(t);
    atomicMax(bits + 2 * s, __float_as_uint(__double2float_ru(fmax(fabs(v.x), fmax(fabs(v.y), fabs(v.z))))));
    atomicMax(bits + 2 * s + 1, __float_as_uint(__double2float_ru(fabs(v.w))));
  }
}

__global__ void k_batch_consts(const unsigned int* __restrict__ bits, int ns, BuildConsts* __restrict__ bc) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < ns) bc[s] = make_consts(bits[2 * s], bits[2 * s + 1]);
}

__global__ void k_batch_gather(const D4* __restrict__ sph64, const int* __restrict__ order,
                               const int64_t* __restrict__ off, int ns, int64_t N, const BuildConsts* __restrict__ bc,
                               float tol32, double tol, float4* __restrict__ sph, float4* __restrict__ thr,
                               int* __restrict__ sid) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= N) return;
  const int o = order[t];
  const int s = find_seg(off, ns, o);
  const D4 d = sph64[o];
  float w = float(d.w);
  if (w == 0.f && d.w != 0.0) w = copysignf(1.4e-45f, float(d.w > 0 ? 1 : -1));
  sph[t] = make_float4(float(d.x), float(d.y), float(d.z), w);
  sid[t] = int(o - off[s]);
  const float A = bc[s].A;
  float lc, hc, lq, hq;
  cov_thresholds(d.w, fabsf(w), tol32, tol, bc[s].eq, A, lc, hc);
  cov_thresholds(d.w, fabsf(w), tol32, tol, 5.9604644775390625e-8f * A, A, lq, hq);
  thr[t] = make_float4(lc, hc, lq, hq);
}

// one level of every shape's hierarchy; prefix[s] = first node of shape s
// at this level in the launch's index space
__global__ void k_batch_tree_level(const Tree* __restrict__ trees, const int64_t* __restrict__ prefix, int ns,
                                   int level, const float4* __restrict__ items_base,
                                   const int64_t* __restrict__ item_off, const BuildConsts* __restrict__ bc,
                                   int is_sphere) {
  const int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (g >= prefix[ns]) return;
  const int s = find_seg(prefix, ns, g);
  const Tree& T = trees[s];
  const int64_t j = g - prefix[s];
  if (level == 0) {
    const float4* items = items_base + item_off[s];
    if (is_sphere) sphere_leaf_node(items, T.nitems, bc[s].A, T.lo, T.hi, T.na, T.nb, T.nf, j);
    else point_leaf_node(items, T.nitems, T.lo, T.hi, j);
  } else {
    if (is_sphere)
      sphere_level_node(T.lo, T.hi, T.na, T.nb, T.nf, bc[s].A, T.offset[level - 1], T.count[level - 1],
                        T.offset[level], j);
    else
      point_level_node(T.lo, T.hi, T.offset[level - 1], T.count[level - 1], T.offset[level], j);
  }
}

// survivors per (shape, class)
__global__ void k_batch_hist(const uint16_t* __restrict__ shape, unsigned n, unsigned* __restrict__ counts) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) atomicAdd(counts + shape[t], 1u);
}

__global__ void k_batch_surv_keys(const float4* __restrict__ items, const uint16_t* __restrict__ shape, unsigned n,
                                  unsigned long long* __restrict__ keys, int* __restrict__ vals) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float4 v = items[t];
  keys[t] = (static_cast<unsigned long long>(shape[t]) << 32) | morton_of(v.x, v.y, v.z);
  vals[t] = int(t);
}

__global__ void k_batch_gather_points(const float4* __restrict__ src, const int* __restrict__ order, unsigned n,
                                      float4* __restrict__ dst) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) dst[t] = src[order[t]];
}

// query points of all shapes: Morton keys with the shape in the high bits;
// the sort payload is the point's index within its shape
__global__ void k_batch_qkeys(const ShapeDesc* __restrict__ d, const int64_t* __restrict__ off, int ns, int64_t M,
                              unsigned long long* __restrict__ keys, int* __restrict__ vals) {
  const int64_t u = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (u >= M) return;
  const int s = find_seg(off, ns, u);
  const int64_t i = u - off[s];
  float x, y, z;
  if (d[s].x_is_fp32) {
    const float* X = static_cast<const float*>(d[s].x);
    x = X[3 * i]; y = X[3 * i + 1]; z = X[3 * i + 2];
  } else {
    const double* X = static_cast<const double*>(d[s].x);
    x = float(X[3 * i]); y = float(X[3 * i + 1]); z = float(X[3 * i + 2]);
  }
  keys[u] = (static_cast<unsigned long long>(s) << 32) | morton_of(x, y, z);
  vals[u] = int(i);
}

// Cull over a group of shapes as one flat launch: block b is item b of
// (shape, direction k, BS Morton-consecutive spheres) -- BS the group's tile,
// picked by the autotuner --, so the candidates left open by the neighbour
// pre-test are packed into full warps as in the single-shape cull, and the
// hardware schedules the uneven blocks.
template <int BS>
__global__ void __launch_bounds__(BS) k_batch_cull_blocks(const CullArgs* __restrict__ views,
                                                          const int64_t* __restrict__ bprefix, int ns) {
  __shared__ uint32_t s_stack[BS / 32][kPStack];
  __shared__ int s_idx[BS], s_wcnt[BS / 32];
  WarpStack W{s_stack[threadIdx.x >> 5], 0};
  const int64_t w = blockIdx.x;
  const int s = find_seg(bprefix, ns, w);
  const CullArgs& a = views[s];
  const int64_t local = w - bprefix[s];
  const int64_t nbs = (a.n + BS - 1) / BS;
  const int k = int(local / nbs);
  const int64_t bl = local - int64_t(k) * nbs;
  cull_packet<true>(a, bl * BS + threadIdx.x, k, W, threadIdx.x & 31, s_idx, s_wcnt);
}

// Persistent query over all shapes: work item = (shape, 32 consecutive
// points of the shape's Morton order).
// kPhase 1: the sphere pass (state per point to the view's state array);
// kPhase 2: the rest of the query (as the single-shape query's two kernels)
template <int kPhase>
__global__ void __launch_bounds__(128) k_batch_query(const QueryArgs* __restrict__ views,
                                                     const int64_t* __restrict__ wprefix, int ns, int64_t limit,
                                                     unsigned long long* __restrict__ ctr) {
  __shared__ uint32_t s_stack[4][kPStack];
  const int lane = threadIdx.x & 31;
  WarpStack W{s_stack[threadIdx.x >> 5], 0};
  for (;;) {
    unsigned long long w = 0;
    if (lane == 0) w = atomicAdd(ctr, 1ull);
    w = __shfl_sync(kAllB, w, 0);
    if (int64_t(w) >= limit) break;
    const int s = find_seg(wprefix, ns, int64_t(w));
    const int64_t wl = int64_t(w) - wprefix[s];
    query_packet<true, kPhase>(views[s], wl * 32 + lane, W, lane);
  }
}

// ---------------------------------------------------------------------------
// Survivor forests laid out on the device (no host round trip, so a rebuild
// can be captured in a CUDA graph): the survivor counts of a class are read
// where the cull left them, capped at the list capacity.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned surv_count(const Counters* cnt, int cls, unsigned cap) {
  return min(cnt->nsurv[cls], cap);
}

__global__ void k_batch_hist_dev(const uint16_t* __restrict__ shape, const Counters* __restrict__ cnt, int cls,
                                 unsigned cap, unsigned* __restrict__ counts) {
  const unsigned n = surv_count(cnt, cls, cap);
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
    atomicAdd(counts + shape[t], 1u);
}

// keys of the capacity's slots: live survivors by (shape, Morton code),
// slots past the count last (so the sorted prefix is the live survivors)
__global__ void k_batch_surv_keys_dev(const float4* __restrict__ items, const uint16_t* __restrict__ shape,
                                      const Counters* __restrict__ cnt, int cls, unsigned cap,
                                      unsigned long long* __restrict__ keys, int* __restrict__ vals) {
  const unsigned n = surv_count(cnt, cls, cap);
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < cap; t += gridDim.x * blockDim.x) {
    if (t < n) {
      const float4 v = items[t];
      keys[t] = (static_cast<unsigned long long>(shape[t]) << 32) | morton_of(v.x, v.y, v.z);
    } else {
      keys[t] = ~0ull;
    }
    vals[t] = int(t);
  }
}

__global__ void k_batch_gather_points_dev(const float4* __restrict__ src, const int* __restrict__ order,
                                          const Counters* __restrict__ cnt, int cls, unsigned cap,
                                          float4* __restrict__ dst) {
  const unsigned n = surv_count(cnt, cls, cap);
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) dst[t] = src[order[t]];
}

// The forest of one class from the per-shape counts (one block; thread 0
// walks the shapes in order): each shape's tree layout (the host's
// tree_layout, levels of ceil(n / 8^l) nodes until a level has at most 8),
// its node range in the shared node arrays, the per-level node prefixes the
// level kernel reads, the shape's survivor offset, and the query views'
// survivor pointer and tree.  status bit (1 << cls): the capacity
// overflowed (counts were capped; results are not valid).
__global__ void k_batch_surv_layout(const unsigned* __restrict__ counts, int ns, const Counters* __restrict__ cnt,
                                    int cls, unsigned cap, int64_t node_cap, float4* lo, float4* hi,
                                    const float4* sorted, Tree* __restrict__ trees, int64_t* __restrict__ prefix,
                                    int nlev, int64_t* __restrict__ soff, QueryArgs* __restrict__ views,
                                    unsigned* __restrict__ status) {
  if (threadIdx.x != 0) return;
  if (cnt->nsurv[cls] > cap) atomicOr(status, 1u << cls);
  int64_t base = 0, so = 0;
  for (int l = 0; l < nlev; ++l) prefix[int64_t(l) * (ns + 1)] = 0;
  for (int s = 0; s < ns; ++s) {
    Tree T;
    T.nitems = counts[s];
    T.nlevels = 0;
    for (int l = 0; l < kMaxLevels; ++l) T.count[l] = T.offset[l] = 0;
    if (T.nitems > 0) {
      int64_t c = (T.nitems + kLeaf - 1) / kLeaf, off = 0;
      int L = 0;
      for (;;) {
        T.count[L] = c;
        T.offset[L] = off;
        off += c;
        ++L;
        if (c <= kFan || L == kMaxLevels) break;
        c = (c + kFan - 1) / kFan;
      }
      T.nlevels = L;
    }
    const int64_t nodes = T.nlevels ? T.offset[T.nlevels - 1] + T.count[T.nlevels - 1] : 0;
    if (base + nodes > node_cap) {  // cannot happen with the node capacity the build sized
      atomicOr(status, 4u);
      T.nlevels = 0;
      T.nitems = 0;
    }
    T.lo = lo + base;
    T.hi = hi + base;
    T.na = T.nb = T.nf = nullptr;
    trees[s] = T;
    for (int l = 0; l < nlev; ++l) {
      int64_t* P = prefix + int64_t(l) * (ns + 1);
      P[s + 1] = P[s] + (l < T.nlevels ? T.count[l] : 0);
    }
    soff[s] = so;
    views[s].surv[cls] = sorted + so;
    views[s].vt[cls] = T;
    base += T.nlevels ? nodes : 0;
    so += T.nitems;
  }
  soff[ns] = so;
}

// ---------------------------------------------------------------------------
static inline unsigned int nb(int64_t n, int b) { return (unsigned int)((n + b - 1) / b); }

cudaError_t launch_batch_surv_forest(const uint16_t* shape, const float4* raw, const Counters* cnt, int cls,
                                     unsigned cap, int ns, unsigned* hist, unsigned long long* kin,
                                     unsigned long long* kout, int* vin, int* vout, void* sort_temp,
                                     size_t sort_bytes, int end_bit, float4* sorted, int64_t node_cap, float4* lo,
                                     float4* hi, Tree* trees, int64_t* prefix, int nlev, int64_t* soff,
                                     QueryArgs* views, unsigned* status, cudaStream_t st) {
  const unsigned g = cap ? (nb(cap, 256) > 8192 ? 8192 : nb(cap, 256)) : 1;
  cudaMemsetAsync(hist, 0, size_t(ns) * 4, st);
  k_batch_hist_dev<<<g, 256, 0, st>>>(shape, cnt, cls, cap, hist);
  k_batch_surv_layout<<<1, 32, 0, st>>>(hist, ns, cnt, cls, cap, node_cap, lo, hi, sorted, trees, prefix, nlev, soff,
                                        views, status);
  if (cap > 0) {
    k_batch_surv_keys_dev<<<g, 256, 0, st>>>(raw, shape, cnt, cls, cap, kin, vin);
    size_t bytes = sort_bytes;
    cudaError_t e = cub::DeviceRadixSort::SortPairs(sort_temp, bytes, kin, kout, vin, vout, int64_t(cap), 0,
                                                    end_bit, st);
    if (e != cudaSuccess) return e;
    k_batch_gather_points_dev<<<g, 256, 0, st>>>(raw, vout, cnt, cls, cap, sorted);
  }
  // levels: an upper bound of each level's node count over all shapes sizes
  // the grid (the kernel reads the exact total from the prefix)
  int64_t bound = int64_t(cap) / kLeaf + ns + 1;
  for (int l = 0; l < nlev; ++l) {
    k_batch_tree_level<<<nb(bound, 128), 128, 0, st>>>(trees, prefix + int64_t(l) * (ns + 1), ns, l, sorted,
                                                       soff, nullptr, 0);
    bound = bound / kFan + ns + 1;
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_copy(const ShapeDesc* d, const int64_t* off, int ns, int64_t N, D4* sph64,
                              unsigned long long* keys, int* vals, unsigned int* bits, BuildConsts* bc,
                              cudaStream_t st) {
  unsigned g = nb(N, 256);
  if (g > 8192) g = 8192;
  k_batch_copy<<<g, 256, 0, st>>>(d, off, ns, N, sph64, keys, vals, bits);
  k_batch_consts<<<nb(ns, 128), 128, 0, st>>>(bits, ns, bc);
  return cudaGetLastError();
}

cudaError_t sort_pairs64(void* temp, size_t& bytes, const unsigned long long* kin, unsigned long long* kout,
                         const int* vin, int* vout, int64_t n, int end_bit, cudaStream_t st) {
  return cub::DeviceRadixSort::SortPairs(temp, bytes, kin, kout, vin, vout, n, 0, end_bit, st);
}

cudaError_t launch_batch_gather(const D4* sph64, const int* order, const int64_t* off, int ns, int64_t N,
                                const BuildConsts* bc, float tol32, double tol, float4* sph, float4* thr, int* sid,
                                cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  k_batch_gather<<<nb(N, 256), 256, 0, st>>>(sph64, order, off, ns, N, bc, tol32, tol, sph, thr, sid);
  return cudaGetLastError();
}

cudaError_t launch_batch_tree_level(const Tree* trees, const int64_t* prefix, int64_t total, int ns, int level,
                                    const float4* items_base, const int64_t* item_off, const BuildConsts* bc,
                                    int is_sphere, cudaStream_t st) {
  if (total == 0) return cudaSuccess;
  k_batch_tree_level<<<nb(total, 128), 128, 0, st>>>(trees, prefix, ns, level, items_base, item_off, bc, is_sphere);
  return cudaGetLastError();
}

cudaError_t launch_batch_hist(const uint16_t* shape, unsigned n, unsigned* counts, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_batch_hist<<<nb(n, 256), 256, 0, st>>>(shape, n, counts);
  return cudaGetLastError();
}

cudaError_t launch_batch_surv_keys(const float4* items, const uint16_t* shape, unsigned n, unsigned long long* keys,
                                   int* vals, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_batch_surv_keys<<<nb(n, 256), 256, 0, st>>>(items, shape, n, keys, vals);
  return cudaGetLastError();
}

cudaError_t launch_batch_gather_points(const float4* src, const int* order, unsigned n, float4* dst,
                                       cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_batch_gather_points<<<nb(n, 256), 256, 0, st>>>(src, order, n, dst);
  return cudaGetLastError();
}

cudaError_t launch_batch_qkeys(const ShapeDesc* d, const int64_t* off, int ns, int64_t M, unsigned long long* keys,
                               int* vals, cudaStream_t st) {
  if (M == 0) return cudaSuccess;
  k_batch_qkeys<<<nb(M, 256), 256, 0, st>>>(d, off, ns, M, keys, vals);
  return cudaGetLastError();
}

cudaError_t launch_batch_cull_blocks(const CullArgs* views, const int64_t* bprefix, int ns, int64_t nblocks, int tile,
                                     cudaStream_t st) {
  if (nblocks <= 0) return cudaSuccess;
  if (nblocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  if (tile == 64) k_batch_cull_blocks<64><<<unsigned(nblocks), 64, 0, st>>>(views, bprefix, ns);
  else if (tile == 256) k_batch_cull_blocks<256><<<unsigned(nblocks), 256, 0, st>>>(views, bprefix, ns);
  else if (tile == 128) k_batch_cull_blocks<128><<<unsigned(nblocks), 128, 0, st>>>(views, bprefix, ns);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_batch_query(const QueryArgs* views, const int64_t* wprefix, int ns, int64_t limit,
                               unsigned long long* ctr, int grid, int phase, cudaStream_t st) {
  if (phase == 1) k_batch_query<1><<<grid, 128, 0, st>>>(views, wprefix, ns, limit, ctr);
  else k_batch_query<2><<<grid, 128, 0, st>>>(views, wprefix, ns, limit, ctr);
  return cudaGetLastError();
}

}  // namespace gfs
