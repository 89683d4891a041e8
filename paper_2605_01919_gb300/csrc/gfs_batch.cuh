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

// Cull over all shapes as one flat launch: block b is item b of (shape,
// direction k, 128 Morton-consecutive spheres), so the candidates left open
// by the neighbour pre-test are packed into full warps as in the single-shape
// cull, and the hardware schedules the uneven blocks.
__global__ void __launch_bounds__(128) k_batch_cull_blocks(const CullArgs* __restrict__ views,
                                                           const int64_t* __restrict__ bprefix, int ns) {
  __shared__ uint32_t s_stack[4][kPStack];
  __shared__ int s_idx[128], s_wcnt[4];
  WarpStack W{s_stack[threadIdx.x >> 5], 0};
  const int64_t w = blockIdx.x;
  const int s = find_seg(bprefix, ns, w);
  const CullArgs& a = views[s];
  const int64_t local = w - bprefix[s];
  const int64_t nb128 = (a.n + 127) / 128;
  const int k = int(local / nb128);
  const int64_t bl = local - int64_t(k) * nb128;
  cull_packet<true>(a, bl * 128 + threadIdx.x, k, W, threadIdx.x & 31, s_idx, s_wcnt);
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
static inline unsigned int nb(int64_t n, int b) { return (unsigned int)((n + b - 1) / b); }

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

cudaError_t launch_batch_cull_blocks(const CullArgs* views, const int64_t* bprefix, int ns, int64_t nblocks,
                                     cudaStream_t st) {
  if (nblocks <= 0) return cudaSuccess;
  if (nblocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  k_batch_cull_blocks<<<unsigned(nblocks), 128, 0, st>>>(views, bprefix, ns);
  return cudaGetLastError();
}

cudaError_t launch_batch_query(const QueryArgs* views, const int64_t* wprefix, int ns, int64_t limit,
                               unsigned long long* ctr, int grid, int phase, cudaStream_t st) {
  if (phase == 1) k_batch_query<1><<<grid, 128, 0, st>>>(views, wprefix, ns, limit, ctr);
  else k_batch_query<2><<<grid, 128, 0, st>>>(views, wprefix, ns, limit, ctr);
  return cudaGetLastError();
}

}  // namespace gfs
