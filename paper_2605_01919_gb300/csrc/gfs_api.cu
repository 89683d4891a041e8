// C ABI of the library: context management and orchestration of the build,
// query, backward and survivor-export calls declared in include/gfs.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <mutex>
#include <vector>

#include "gfs.h"
#include "gfs_kernels.h"
#include "gfs_exact.h"
#include "gfs_order.h"
#include "gfs_scored.h"
#include "gfs_tangent.h"

using namespace gfs;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

int ensure(DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return GFS_OK;
  // a buffer that has to grow gets 1/8 headroom, so that slowly growing
  // sizes (hierarchy rebuilds during insertion) do not reallocate each time
  if (b.p) bytes += bytes / 8;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return GFS_ERR_OOM;
  }
  b.bytes = bytes;
  return GFS_OK;
}

// grow a buffer, keeping its first `keep` bytes
int grow_keep(DevBuf& b, size_t bytes, size_t keep, cudaStream_t st) {
  if (b.bytes >= bytes && b.p) return GFS_OK;
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return GFS_ERR_OOM;
  }
  if (keep && b.p && (cudaMemcpyAsync(p, b.p, keep, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
                      cudaStreamSynchronize(st) != cudaSuccess)) {
    cudaGetLastError();
    cudaFree(p);
    return GFS_ERR_CUDA;
  }
  if (b.p) cudaFree(b.p);
  b.p = p;
  b.bytes = bytes;
  return GFS_OK;
}

void release(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

// A scratch buffer of one call, released when the call returns.
struct Scratch {
  DevBuf b;
  Scratch() = default;
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;
  ~Scratch() { release(b); }
};

// Level sizes of the implicit hierarchy over nitems items.
void tree_layout(Tree& T, int64_t nitems) {
  std::memset(&T, 0, sizeof(T));
  T.nitems = nitems;
  if (nitems <= 0) return;
  int64_t c = (nitems + kLeaf - 1) / kLeaf, off = 0;
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

// Survivors of one sign class that a hierarchy can index: node indices are
// 27-bit fields (pack_node) over leaves of kLeaf items, and sort values are
// int32.
constexpr unsigned kMaxSurvivors = 1u << 30;

int64_t tree_nodes(const Tree& T) {
  return T.nlevels ? T.offset[T.nlevels - 1] + T.count[T.nlevels - 1] : 0;
}

#define GFS_CK(expr)                         \
  do {                                       \
    cudaError_t e_ = (expr);                 \
    if (e_ != cudaSuccess) {                 \
      cudaGetLastError();                    \
      return GFS_ERR_CUDA;                   \
    }                                        \
  } while (0)

#define GFS_TRY(expr)          \
  do {                         \
    int s_ = (expr);           \
    if (s_ != GFS_OK) return s_; \
  } while (0)

}  // namespace

struct gfs_ctx {
  gfs_options opt{};
  cudaStream_t stream = nullptr;
  int K = 0, KS = 0;
  DevBuf U32, U64;
  // spheres
  int64_t n = 0;
  bool built = false;
  DevBuf sph64, keys_in, keys_out, vals_in, vals_out, sph, thr, sid, bound_bits, consts, cnt, cub_temp;
  Tree st{};
  DevBuf st_lo, st_hi, st_na, st_nb, st_nf;
  DevBuf st_tight;  // scratch of the internal-ball tightening
  // survivors
  DevBuf surv_raw[2], surv_sorted[2], vt_lo[2], vt_hi[2];
  Tree vt[2]{};
  unsigned int cap = 0;
  unsigned int nsurv[2] = {0, 0};
  // query / backward scratch
  DevBuf defer, acc, witness64;
  DevBuf qk_in, qk_out, qv_in, qv_out;  // query Morton keys / processing order
  // insertion state
  DevBuf ins_counts, ins_tomb[2], ins_dsurv[2], ins_dtomb[2], ins_misc;
  DevBuf ins_maxrem, ins_slot_t, ins_slots, ins_cbuf, ins_new, ins_lost, ins_inserted, ins_codes, ins_dyn;
  DevBuf ins_present, ins_scan, ins_cmp, ins_dynf4, ins_near, ins_nearcnt;
  // per-sphere survivor lists for the scored value (sorted ids + offsets),
  // valid while csr_state equals state_id (every build or insertion changes it)
  DevBuf csr_ids, csr_off, scored_status;
  // uncovered intersection circles and points (raw outputs, sort buffers)
  DevBuf ud_uncov, ud_cnt, ud_pairs, ud_circ, ud_quad, ud_pts, ud_k0, ud_k1, ud_v0, ud_v1;
  int64_t ud_state = -1, ud_nc = 0, ud_np = 0;  // the raw lists hold state ud_state
  unsigned ud_status = 0;
  int64_t state_id = 0, csr_state = -1;
  int64_t ins_rounds = 0, ins_steps = 0, ins_rebuilds = 0, ins_queried = 0;  // of the last insertion call
  double ins_ms_total = 0.0, ins_ms_rebuild = 0.0, ins_ms_final = 0.0;  // host wall time of its phases
  double ins_ms_query = 0.0, ins_ms_commit = 0.0, ins_ms_update = 0.0;  // device time (timing = 1)
  unsigned long long ins_work[4] = {0, 0, 0, 0};  // step-query work counters (InsMisc::work)
  // batched shapes
  int b_ns = 0;
  bool b_built = false;
  std::vector<gfs_shape> b_shapes;
  std::vector<int64_t> b_off, b_qoff, b_soff[2];
  std::vector<Tree> b_st;
  DevBuf b_desc, b_offd, b_qoffd, b_sph64, b_k64in, b_k64out, b_sph, b_thr, b_sid, b_bits, b_bcs;
  DevBuf b_lo, b_hi, b_na, b_nb, b_nf, b_stdev, b_prefix, b_ctr, b_cnt, b_cviews, b_cw;
  DevBuf b_sraw[2], b_sshape[2], b_ssorted[2], b_vlo[2], b_vhi[2], b_vtdev[2], b_hist;
  DevBuf b_qkin, b_qkout, b_qvin, b_qvout, b_qviews, b_qw, b_qstate;
  std::vector<QueryArgs> b_qv;  // host copies of the per-shape query views
  DevBuf b_status, b_vprefix[2], b_sodev[2];
  std::vector<int64_t> b_sph_level_total;  // nodes per level of the sample forest, over all shapes
  int b_sph_levels = 0, b_surv_levels = 0, b_end_bit = 32;
  int64_t b_node_cap = 0;
  // cull tiles per size class (autotuned on the first build): shapes of
  // class k are views [b_cls_off[k], b_cls_off[k+1]) of b_cviews, with block
  // prefixes at b_cw + b_cls_off[k] + k
  int b_tile[3] = {128, 128, 128};
  bool b_tiles_tuned = false;
  int b_cls_off[4] = {0, 0, 0, 0};
  int64_t b_cls_blocks[3] = {0, 0, 0};
  std::vector<int> b_cls_order;     // shape index of each view, grouped by class
  unsigned b_cap = 0;
  unsigned b_nsurv[2] = {0, 0};
  int64_t b_M = 0, b_qtotal = 0;
  int b_grid_query = 0;
  Counters host_cnt{};
  // host-buffer path (gfs_solve_host)
  DevBuf h_p, h_s, h_x, h_sout, h_arg, h_fl;
  cudaStream_t side = nullptr;  // the query points' upload, overlapping the build
  cudaEvent_t sev = nullptr, sev2 = nullptr;  // main -> side, side -> main
  DevBuf qstate;                // per-slot state between the query's two kernels
  // phase events (timing = 1): build start, cull start, cull end, build end,
  // query start, fast end, query end
  cudaEvent_t ev[8] = {};  // + end of the query's sphere pass
  bool have_ev = false;
  bool built_timed = false, query_timed = false;
};

namespace {

int cub_ensure(gfs_ctx* c, size_t bytes) { return ensure(c->cub_temp, bytes); }

int sort_u32_pairs(gfs_ctx* c, uint32_t* kin, uint32_t* kout, int* vin, int* vout, int64_t n) {
  size_t bytes = 0;
  GFS_CK(sort_pairs(nullptr, bytes, kin, kout, vin, vout, n, c->stream));
  GFS_TRY(cub_ensure(c, bytes));
  bytes = c->cub_temp.bytes;
  GFS_CK(sort_pairs(c->cub_temp.p, bytes, kin, kout, vin, vout, n, c->stream));
  return GFS_OK;
}

int build_point_tree(gfs_ctx* c, int cls) {
  const int64_t ns = c->nsurv[cls];
  Tree& T = c->vt[cls];
  tree_layout(T, ns);
  if (ns == 0) return GFS_OK;
  GFS_TRY(ensure(c->keys_in, size_t(ns) * 4));
  GFS_TRY(ensure(c->keys_out, size_t(ns) * 4));
  GFS_TRY(ensure(c->vals_in, size_t(ns) * 4));
  GFS_TRY(ensure(c->vals_out, size_t(ns) * 4));
  GFS_TRY(ensure(c->surv_sorted[cls], size_t(ns) * sizeof(float4)));
  GFS_CK(launch_point_keys(c->surv_raw[cls].as<float4>(), ns, c->keys_in.as<uint32_t>(), c->vals_in.as<int>(),
                           c->stream));
  GFS_TRY(sort_u32_pairs(c, c->keys_in.as<uint32_t>(), c->keys_out.as<uint32_t>(), c->vals_in.as<int>(),
                         c->vals_out.as<int>(), ns));
  GFS_CK(launch_gather_points(c->surv_raw[cls].as<float4>(), c->vals_out.as<int>(), ns,
                              c->surv_sorted[cls].as<float4>(), c->stream));
  const int64_t nodes = tree_nodes(T);
  GFS_TRY(ensure(c->vt_lo[cls], size_t(nodes) * sizeof(float4)));
  GFS_TRY(ensure(c->vt_hi[cls], size_t(nodes) * sizeof(float4)));
  T.lo = c->vt_lo[cls].as<float4>();
  T.hi = c->vt_hi[cls].as<float4>();
  T.na = T.nb = T.nf = nullptr;
  GFS_CK(launch_build_tree(c->surv_sorted[cls].as<float4>(), 0, 0.f, T, nullptr, c->stream));
  return GFS_OK;
}

void fill_query_args(gfs_ctx* c, QueryArgs& a) {
  std::memset(&a, 0, sizeof(a));
  a.sph = c->sph.as<float4>();
  a.thr = c->thr.as<float4>();
  a.sid = c->sid.as<int>();
  a.sph64 = c->sph64.as<D4>();
  a.st = c->st;
  a.n = c->n;
  for (int k = 0; k < 2; ++k) {
    a.surv[k] = c->surv_sorted[k].as<float4>();
    a.vt[k] = c->vt[k];
  }
  a.U64 = c->U64.as<double>();
  a.witness64 = c->witness64.as<double>();
  a.K = c->K;
  a.KS = c->KS;
  a.tol32 = float(c->opt.tol);
  a.tol = c->opt.tol;
  a.clamp_opp = c->opt.clamp_opp;
  a.bc = c->consts.as<BuildConsts>();
  a.cnt = c->cnt.as<Counters>();
}

// a2: Morton-sort the samples in sph64[0, n) and build the sphere hierarchy
// (also used to rebuild it after insertions).
int build_sphere_hierarchy(gfs_ctx* c, int64_t n, const int* ids = nullptr) {
  cudaStream_t st = c->stream;
  c->n = n;
  // with ids: the hierarchy holds the spheres sph64[ids[0..n)] and its sorted
  // slots map to those indices (the insertion rounds' provisional numbering)
  const D4* src = c->sph64.as<D4>();
  if (ids) {
    GFS_TRY(ensure(c->ins_cmp, size_t(n) * sizeof(D4)));
    GFS_CK(launch_gather_d4(c->sph64.as<D4>(), ids, n, c->ins_cmp.as<D4>(), st));
    src = c->ins_cmp.as<D4>();
  }
  GFS_TRY(ensure(c->keys_in, size_t(n) * 4));
  GFS_TRY(ensure(c->keys_out, size_t(n) * 4));
  GFS_TRY(ensure(c->vals_in, size_t(n) * 4));
  GFS_TRY(ensure(c->vals_out, size_t(n) * 4));
  GFS_TRY(ensure(c->sph, size_t(n) * sizeof(float4)));
  GFS_TRY(ensure(c->thr, size_t(n) * sizeof(float4)));
  GFS_TRY(ensure(c->sid, size_t(n) * 4));
  GFS_CK(cudaMemsetAsync(c->bound_bits.p, 0, 16, st));
  GFS_CK(launch_keys_d4(src, n, c->keys_in.as<uint32_t>(), c->vals_in.as<int>(),
                        c->bound_bits.as<unsigned int>(), c->consts.as<BuildConsts>(), st));
  GFS_TRY(sort_u32_pairs(c, c->keys_in.as<uint32_t>(), c->keys_out.as<uint32_t>(), c->vals_in.as<int>(),
                         c->vals_out.as<int>(), n));
  GFS_CK(launch_gather_spheres(src, c->vals_out.as<int>(), n, c->consts.as<BuildConsts>(),
                               float(c->opt.tol), c->opt.tol, c->sph.as<float4>(), c->thr.as<float4>(),
                               c->sid.as<int>(), st));
  if (ids) GFS_CK(launch_remap_sid(c->sid.as<int>(), ids, n, st));
  tree_layout(c->st, n);
  const int64_t nodes = tree_nodes(c->st);
  GFS_TRY(ensure(c->st_lo, size_t(nodes) * sizeof(float4)));
  GFS_TRY(ensure(c->st_hi, size_t(nodes) * sizeof(float4)));
  GFS_TRY(ensure(c->st_na, size_t(nodes) * sizeof(float4)));
  GFS_TRY(ensure(c->st_nb, size_t(nodes) * sizeof(float4)));
  GFS_TRY(ensure(c->st_nf, size_t(nodes) * sizeof(float4)));
  c->st.lo = c->st_lo.as<float4>();
  c->st.hi = c->st_hi.as<float4>();
  c->st.na = c->st_na.as<float4>();
  c->st.nb = c->st_nb.as<float4>();
  c->st.nf = c->st_nf.as<float4>();
  // the coordinate bound A is needed on the host for the hierarchy's rounding slack
  unsigned int bits[2] = {0, 0};
  GFS_CK(cudaMemcpyAsync(bits, c->bound_bits.p, 8, cudaMemcpyDeviceToHost, st));
  GFS_CK(cudaStreamSynchronize(st));
  float Ahost;
  std::memcpy(&Ahost, &bits[0], 4);
  Ahost = std::max(1.0f, Ahost);
  GFS_TRY(ensure(c->st_tight, size_t(std::max<int64_t>(nodes - c->st.count[0], 1)) * 4 * sizeof(unsigned)));
  GFS_CK(launch_build_tree(c->sph.as<float4>(), 1, Ahost, c->st, c->st_tight.as<unsigned>(), st));
  return GFS_OK;
}

}  // namespace

extern "C" {

void gfs_default_options(gfs_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->tau = 3;
  opt->tol = 1e-6;
  opt->box_cull = 1;
  opt->clamp_opp = 1;
  opt->precision = 0;
}

const char* gfs_strerror(int status) {
  switch (status) {
    case GFS_OK: return "ok";
    case GFS_ERR_ARG: return "invalid argument";
    case GFS_ERR_OOM: return "device allocation failed";
    case GFS_ERR_CUDA: return "CUDA runtime error";
    case GFS_ERR_STATE: return "call order violated (build first)";
    case GFS_ERR_TIMEOUT: return "capped device loop ran out of iterations";
    case GFS_ERR_TOO_LARGE: return "sizes exceed the library's index range";
    default: return "unknown status";
  }
}

int gfs_create(gfs_ctx** out, const gfs_options* opt, void* cuda_stream) {
  if (!out) return GFS_ERR_ARG;
  *out = nullptr;
  gfs_options o;
  if (opt) o = *opt;
  else gfs_default_options(&o);
  if (o.tau < 0 || o.tau > 6 || !(o.tol >= 0.0) || o.tol > 0.1 || (o.precision != 0 && o.precision != 1) ||
      (o.timing != 0 && o.timing != 1))
    return GFS_ERR_ARG;
  for (int r : o.reserved)
    if (r != 0) return GFS_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return GFS_ERR_CUDA;
  }
  gfs_ctx* c = new gfs_ctx();
  c->opt = o;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->K = 10 * (1 << (2 * o.tau)) + 2;
  c->KS = c->K + 1;
  std::vector<double> U(size_t(c->K) * 3);
  std::vector<float> U32(size_t(c->K) * 3);
  if (gfs_icosphere(o.tau, U.data(), c->K) != c->K) {
    delete c;
    return GFS_ERR_ARG;
  }
  for (size_t t = 0; t < U.size(); ++t) U32[t] = float(U[t]);
  int st = ensure(c->U64, U.size() * 8);
  if (st == GFS_OK) st = ensure(c->U32, U32.size() * 4);
  if (st == GFS_OK) st = ensure(c->bound_bits, 16);
  if (st == GFS_OK) st = ensure(c->consts, sizeof(BuildConsts));
  if (st == GFS_OK) st = ensure(c->cnt, sizeof(Counters));
  if (st != GFS_OK) {
    gfs_destroy(c);
    return st;
  }
  if (o.timing) {
    for (cudaEvent_t& e : c->ev)
      if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        gfs_destroy(c);
        return GFS_ERR_CUDA;
      }
    c->have_ev = true;
  }
  if (cudaMemcpy(c->U64.p, U.data(), U.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->U32.p, U32.data(), U32.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(c->cnt.p, 0, sizeof(Counters)) != cudaSuccess) {
    cudaGetLastError();
    gfs_destroy(c);
    return GFS_ERR_CUDA;
  }
  *out = c;
  return GFS_OK;
}

int gfs_set_stream(gfs_ctx* c, void* cuda_stream) {
  if (!c) return GFS_ERR_ARG;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  return GFS_OK;
}

namespace {

// the cull's counters (before a rerun of the cull)
int reset_cull_counters(gfs_ctx* c, cudaStream_t st) {
  char* base = reinterpret_cast<char*>(c->cnt.p);
  GFS_CK(cudaMemsetAsync(base + offsetof(Counters, cull_rechecks), 0, sizeof(unsigned long long), st));
  GFS_CK(cudaMemsetAsync(base + offsetof(Counters, nsurv), 0, 2 * sizeof(unsigned int), st));
  GFS_CK(cudaMemsetAsync(base + offsetof(Counters, c_ntests), 0, 2 * sizeof(unsigned long long), st));
  return GFS_OK;
}

// a2: inputs copied, counters cleared, sphere hierarchy built
int build_begin(gfs_ctx* c, const double* p, const double* s, int64_t n) {
  if (!c || !p || !s || n < 1) return GFS_ERR_ARG;
  if (uint64_t(n) * uint64_t(c->KS) >= (uint64_t(1) << 32) || n >= (int64_t(1) << 30)) return GFS_ERR_TOO_LARGE;
  c->built = false;
  c->built_timed = false;
  c->query_timed = false;
  cudaStream_t st = c->stream;
  if (c->have_ev) GFS_CK(cudaEventRecord(c->ev[0], st));
  GFS_TRY(ensure(c->sph64, size_t(n) * sizeof(D4)));
  GFS_CK(cudaMemsetAsync(c->cnt.p, 0, sizeof(Counters), st));
  GFS_CK(launch_copy_inputs(p, s, n, c->sph64.as<D4>(), st));
  return build_sphere_hierarchy(c, n);
}

// a3, a4: candidate generation and coverage culling, survivor hierarchies
int build_finish(gfs_ctx* c) {
  cudaStream_t st = c->stream;
  const int64_t n = c->n;
  const uint64_t ncand = uint64_t(n) * uint64_t(c->K);
  uint64_t cap = std::max<uint64_t>(uint64_t(1) << 16, ncand / 16 + 1024);
  cap = std::min<uint64_t>(cap, ncand + 16);
  for (int attempt = 0; attempt < 3; ++attempt) {
    c->cap = unsigned(std::min<uint64_t>(cap, 0xffffffffu));
    GFS_TRY(ensure(c->surv_raw[0], size_t(c->cap) * sizeof(float4)));
    GFS_TRY(ensure(c->surv_raw[1], size_t(c->cap) * sizeof(float4)));
    if (attempt > 0) GFS_TRY(reset_cull_counters(c, st));
    CullArgs a;
    std::memset(&a, 0, sizeof(a));
    a.sph = c->sph.as<float4>();
    a.thr = c->thr.as<float4>();
    a.sid = c->sid.as<int>();
    a.sph64 = c->sph64.as<D4>();
    a.U32 = c->U32.as<float>();
    a.U64 = c->U64.as<double>();
    a.K = c->K;
    a.KS = c->KS;
    a.tree = c->st;
    a.tol32 = float(c->opt.tol);
    a.tol = c->opt.tol;
    a.box_cull = c->opt.box_cull;
    a.bc = c->consts.as<BuildConsts>();
    a.n = n;
    a.surv[0] = c->surv_raw[0].as<float4>();
    a.surv[1] = c->surv_raw[1].as<float4>();
    a.cap = c->cap;
    a.cnt = c->cnt.as<Counters>();
    if (c->have_ev) GFS_CK(cudaEventRecord(c->ev[1], st));
    GFS_CK(launch_cull(a, st));
    if (c->have_ev) GFS_CK(cudaEventRecord(c->ev[2], st));
    unsigned int ns[2] = {0, 0};
    GFS_CK(cudaMemcpyAsync(ns, reinterpret_cast<char*>(c->cnt.p) + offsetof(Counters, nsurv), sizeof(ns),
                           cudaMemcpyDeviceToHost, st));
    GFS_CK(cudaStreamSynchronize(st));
    c->host_cnt.nsurv[0] = ns[0];
    c->host_cnt.nsurv[1] = ns[1];
    const unsigned int need = std::max(ns[0], ns[1]);
    if (need <= c->cap) break;
    cap = uint64_t(need) + need / 8 + 1024;
    if (attempt == 2) return GFS_ERR_OOM;
  }
  c->nsurv[0] = c->host_cnt.nsurv[0];
  c->nsurv[1] = c->host_cnt.nsurv[1];
  if (std::max(c->nsurv[0], c->nsurv[1]) > kMaxSurvivors) return GFS_ERR_TOO_LARGE;
  GFS_TRY(build_point_tree(c, 0));
  GFS_TRY(build_point_tree(c, 1));
  if (c->have_ev) {
    GFS_CK(cudaEventRecord(c->ev[3], st));
    c->built_timed = true;
  }
  c->built = true;
  return GFS_OK;
}

int ensure_side(gfs_ctx* c) {
  if (c->side) return GFS_OK;
  GFS_CK(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
  GFS_CK(cudaEventCreateWithFlags(&c->sev, cudaEventDisableTiming));
  GFS_CK(cudaEventCreateWithFlags(&c->sev2, cudaEventDisableTiming));
  return GFS_OK;
}

}  // namespace

int gfs_build(gfs_ctx* c, const double* p, const double* s, int64_t n) {
  if (c) ++c->state_id;
  GFS_TRY(build_begin(c, p, s, n));
  return build_finish(c);
}

int gfs_query(gfs_ctx* c, const void* x, int x_is_fp32, int64_t m, float* s_out, double* s64_out,
              int64_t* argmin_out, uint16_t* flags_out) {
  if (!c || m < 0 || (m > 0 && !x)) return GFS_ERR_ARG;
  if (!c->built) return GFS_ERR_STATE;
  if (m >= (int64_t(1) << 32)) return GFS_ERR_TOO_LARGE;
  if (m == 0) return GFS_OK;
  QueryArgs a;
  fill_query_args(c, a);
  if (x_is_fp32) a.x32 = static_cast<const float*>(x);
  else a.x64 = static_cast<const double*>(x);
  a.m = m;
  a.s_out = s_out;
  a.s64_out = s64_out;
  a.arg_out = argmin_out;
  a.fl_out = flags_out;
  if (c->opt.precision == 0) {
    GFS_TRY(ensure(c->defer, size_t(m) * 4));
    a.defer = c->defer.as<uint32_t>();
    a.defer_cap = unsigned(m);
    // process the points in Morton order so that a warp's lanes are neighbours
    GFS_TRY(ensure(c->qk_in, size_t(m) * 4));
    GFS_TRY(ensure(c->qk_out, size_t(m) * 4));
    GFS_TRY(ensure(c->qv_in, size_t(m) * 4));
    GFS_TRY(ensure(c->qv_out, size_t(m) * 4));
    GFS_CK(launch_query_keys(a.x64, a.x32, m, c->qk_in.as<uint32_t>(), c->qv_in.as<int>(), c->stream));
    GFS_TRY(sort_u32_pairs(c, c->qk_in.as<uint32_t>(), c->qk_out.as<uint32_t>(), c->qv_in.as<int>(),
                           c->qv_out.as<int>(), m));
    a.perm = reinterpret_cast<const uint32_t*>(c->qv_out.p);
    GFS_TRY(ensure(c->qstate, size_t(m) * 3 * sizeof(uint4)));
    a.state = reinterpret_cast<uint4*>(c->qstate.p);
  }
  GFS_CK(cudaMemsetAsync(reinterpret_cast<char*>(c->cnt.p) + offsetof(Counters, query_rechecks), 0,
                         sizeof(unsigned long long), c->stream));
  GFS_CK(cudaMemsetAsync(reinterpret_cast<char*>(c->cnt.p) + offsetof(Counters, q_sphere_ntests), 0,
                         5 * sizeof(unsigned long long), c->stream));
  GFS_CK(cudaMemsetAsync(reinterpret_cast<char*>(c->cnt.p) + offsetof(Counters, ndefer), 0, sizeof(unsigned int),
                         c->stream));
  if (c->have_ev) GFS_CK(cudaEventRecord(c->ev[4], c->stream));
  if (c->opt.precision == 0) {
    GFS_CK(launch_query_spheres(a, c->stream));
    if (c->have_ev) GFS_CK(cudaEventRecord(c->ev[7], c->stream));
    GFS_CK(launch_query_finish(a, c->stream));
  } else if (c->have_ev) {
    GFS_CK(cudaEventRecord(c->ev[7], c->stream));
  }
  if (c->have_ev) GFS_CK(cudaEventRecord(c->ev[5], c->stream));
  GFS_CK(launch_query_exact(a, c->opt.precision == 1, c->stream));
  if (c->have_ev) {
    GFS_CK(cudaEventRecord(c->ev[6], c->stream));
    c->query_timed = true;
  }
  return GFS_OK;
}

int gfs_query_backward(gfs_ctx* c, const void* x, int x_is_fp32, int64_t m, const float* s, const int64_t* argmin,
                       const uint16_t* flags, const float* grad_s, float* grad_x, float* grad_p, float* grad_sv) {
  if (!c || m < 0 || (m > 0 && (!x || !s || !argmin || !flags || !grad_s))) return GFS_ERR_ARG;
  if (!c->built) return GFS_ERR_STATE;
  const int64_t n = c->n;
  GFS_TRY(ensure(c->acc, size_t(4 * n) * sizeof(long long)));
  GFS_CK(cudaMemsetAsync(c->acc.p, 0, size_t(4 * n) * sizeof(long long), c->stream));
  GradArgs a;
  std::memset(&a, 0, sizeof(a));
  if (x_is_fp32) a.x32 = static_cast<const float*>(x);
  else a.x64 = static_cast<const double*>(x);
  a.m = m;
  a.s = s;
  a.arg = argmin;
  a.flags = flags;
  a.grad_s = grad_s;
  a.grad_x = grad_x;
  a.sph64 = c->sph64.as<D4>();
  a.U64 = c->U64.as<double>();
  a.witness64 = c->witness64.as<double>();
  a.K = c->K;
  a.KS = c->KS;
  a.acc_p = c->acc.as<long long>();
  a.acc_s = c->acc.as<long long>() + 3 * n;
  GFS_CK(launch_grad(a, n, nullptr, nullptr, c->stream));
  GFS_CK(launch_tangent_grad(a, n, grad_p, grad_sv, c->stream));
  return GFS_OK;
}

int gfs_query_points(gfs_ctx* c, const void* x, int x_is_fp32, int64_t m, const int64_t* argmin,
                     const uint16_t* flags, double* qstar_out) {
  if (!c || m < 0 || (m > 0 && (!x || !argmin || !flags || !qstar_out))) return GFS_ERR_ARG;
  if (!c->built) return GFS_ERR_STATE;
  if (m == 0) return GFS_OK;
  QueryArgs a;
  fill_query_args(c, a);
  if (x_is_fp32) a.x32 = static_cast<const float*>(x);
  else a.x64 = static_cast<const double*>(x);
  a.m = m;
  GFS_CK(launch_argmin_points(a, argmin, flags, qstar_out, c->stream));
  return GFS_OK;
}

int gfs_sphere_uncovered(gfs_ctx* c, uint8_t* out, double* witness) {
  if (!c || !out) return GFS_ERR_ARG;
  if (!c->built) return GFS_ERR_STATE;
  QueryArgs a;
  fill_query_args(c, a);
  GFS_CK(launch_sphere_uncovered(a, out, witness, c->stream));
  return GFS_OK;
}

namespace {

// The uncovered circles and points of the current state in c->ud_circ /
// ud_quad / ud_pts (unsorted), computed once per state: the per-sphere
// test, the cutting pairs of uncovered spheres, then the circles.
int ud_compute(gfs_ctx* c) {
  if (c->ud_state == c->state_id) return GFS_OK;
  c->ud_nc = c->ud_np = 0;
  c->ud_status = 0;
  if (c->n == 0) {
    c->ud_state = c->state_id;
    return GFS_OK;
  }
  cudaStream_t st = c->stream;
  QueryArgs a;
  fill_query_args(c, a);
  GFS_TRY(ensure(c->ud_uncov, size_t(c->n) + 16));
  GFS_TRY(ensure(c->ud_cnt, 32));
  GFS_CK(launch_sphere_uncovered(a, c->ud_uncov.as<uint8_t>(), nullptr, st));
  // the pairs of uncovered spheres that cut in a circle: a first guess of
  // the capacity, then exactly the count (the walk is deterministic)
  int64_t cap_pairs = std::max<int64_t>(1 << 20, 16 * c->n);
  unsigned long long hpairs = 0;
  for (int pass = 0; pass < 2; ++pass) {
    GFS_TRY(ensure(c->ud_pairs, size_t(cap_pairs) * 8));
    GFS_CK(cudaMemsetAsync(c->ud_cnt.p, 0, 32, st));
    GFS_CK(launch_ud_pairs(a, c->ud_uncov.as<uint8_t>(), c->ud_pairs.as<unsigned long long>(), cap_pairs,
                           c->ud_cnt.as<unsigned long long>() + 3, st));
    GFS_CK(cudaMemcpyAsync(&hpairs, c->ud_cnt.as<unsigned long long>() + 3, 8, cudaMemcpyDeviceToHost, st));
    GFS_CK(cudaStreamSynchronize(st));
    if (int64_t(hpairs) <= cap_pairs) break;
    if (pass == 1) return GFS_ERR_CUDA;  // cannot happen: the second walk finds the same pairs
    cap_pairs = int64_t(hpairs);
  }
  // raw outputs: a first guess, then exactly the counts (the decisions do not
  // depend on the capacities, so a second run finds the same entries)
  int64_t cap_c = std::max<int64_t>(4096, c->n), cap_p = std::max<int64_t>(4096, c->n);
  unsigned long long hc[2] = {0, 0};
  unsigned hstatus = 0;
  for (int pass = 0; pass < 2; ++pass) {
    GFS_TRY(ensure(c->ud_circ, size_t(cap_c) * 16));
    GFS_TRY(ensure(c->ud_quad, size_t(cap_p) * 32));
    GFS_TRY(ensure(c->ud_pts, size_t(cap_p) * 24));
    GFS_CK(cudaMemsetAsync(c->ud_cnt.p, 0, 32, st));
    exact::UDOut o{c->ud_cnt.as<unsigned long long>(), cap_c, cap_p, c->ud_circ.as<int64_t>(), c->ud_quad.as<int64_t>(),
                   c->ud_pts.as<double>(), reinterpret_cast<unsigned*>(c->ud_cnt.as<unsigned long long>() + 2)};
    GFS_CK(launch_intersections(a, c->ud_pairs.as<unsigned long long>(), int64_t(hpairs), o, st));
    GFS_CK(cudaMemcpyAsync(hc, c->ud_cnt.p, 16, cudaMemcpyDeviceToHost, st));
    GFS_CK(cudaMemcpyAsync(&hstatus, c->ud_cnt.as<unsigned long long>() + 2, 4, cudaMemcpyDeviceToHost, st));
    GFS_CK(cudaStreamSynchronize(st));
    if (int64_t(hc[0]) <= cap_c && int64_t(hc[1]) <= cap_p) break;
    if (pass == 1) return GFS_ERR_CUDA;  // cannot happen: the second run finds the same entries
    cap_c = std::max<int64_t>(cap_c, int64_t(hc[0]));
    cap_p = std::max<int64_t>(cap_p, int64_t(hc[1]));
  }
  c->ud_nc = int64_t(hc[0]);
  c->ud_np = int64_t(hc[1]);
  c->ud_status = hstatus;
  c->ud_state = c->state_id;
  return GFS_OK;
}

}  // namespace

int gfs_uncovered_intersections(gfs_ctx* c, int64_t cap_circles, int64_t* circles_out, int64_t cap_points,
                                int64_t* quads_out, double* points_out, int64_t* counts_host) {
  if (!c || !counts_host || cap_circles < 0 || cap_points < 0) return GFS_ERR_ARG;
  if ((cap_circles > 0 && !circles_out) || (cap_points > 0 && (!quads_out || !points_out))) return GFS_ERR_ARG;
  if (!c->built) return GFS_ERR_STATE;
  counts_host[0] = counts_host[1] = counts_host[2] = 0;
  if (c->n == 0) return GFS_OK;
  cudaStream_t st = c->stream;
  GFS_TRY(ud_compute(c));
  const int64_t nc = c->ud_nc, np = c->ud_np;
  const unsigned hstatus = c->ud_status;
  counts_host[0] = nc;
  counts_host[1] = np;
  counts_host[2] = int64_t(hstatus);
  if (nc > cap_circles || np > cap_points) return GFS_ERR_ARG;
  if (nc >= (int64_t(1) << 31) || np >= (int64_t(1) << 31)) return GFS_ERR_TOO_LARGE;
  const int64_t nk = std::max<int64_t>(std::max<int64_t>(nc, np), 1);
  GFS_TRY(ensure(c->ud_k0, size_t(nk) * 8));
  GFS_TRY(ensure(c->ud_k1, size_t(nk) * 8));
  GFS_TRY(ensure(c->ud_v0, size_t(nk) * 4));
  GFS_TRY(ensure(c->ud_v1, size_t(nk) * 4));
  auto sort64 = [&](int64_t cnt) -> int {
    size_t bytes = 0;
    GFS_CK(sort_pairs64(nullptr, bytes, c->ud_k0.as<unsigned long long>(), c->ud_k1.as<unsigned long long>(),
                        c->ud_v0.as<int>(), c->ud_v1.as<int>(), cnt, 64, st));
    GFS_TRY(cub_ensure(c, bytes));
    bytes = c->cub_temp.bytes;
    GFS_CK(sort_pairs64(c->cub_temp.p, bytes, c->ud_k0.as<unsigned long long>(), c->ud_k1.as<unsigned long long>(),
                        c->ud_v0.as<int>(), c->ud_v1.as<int>(), cnt, 64, st));
    return GFS_OK;
  };
  // points: by (m, side), then stably by (i, j)
  if (np > 0) {
    GFS_CK(launch_ud_point_keys(c->ud_quad.as<int64_t>(), nullptr, np, 0, c->ud_k0.as<unsigned long long>(),
                                c->ud_v0.as<int>(), st));
    GFS_TRY(sort64(np));
    GFS_CK(launch_ud_point_keys(c->ud_quad.as<int64_t>(), c->ud_v1.as<int>(), np, 1,
                                c->ud_k0.as<unsigned long long>(), c->ud_v0.as<int>(), st));
    GFS_TRY(sort64(np));
    GFS_CK(launch_ud_gather(nullptr, 0, nullptr, c->ud_v1.as<int>(), c->ud_quad.as<int64_t>(), c->ud_pts.as<double>(),
                            np, quads_out, points_out, st));
  }
  if (nc > 0) {
    // the keys carry the pairs; the sort's payload is unused
    GFS_CK(launch_ud_circle_keys(c->ud_circ.as<int64_t>(), nc, c->ud_k0.as<unsigned long long>(), st));
    GFS_TRY(sort64(nc));
    GFS_CK(launch_ud_gather(c->ud_k1.as<unsigned long long>(), nc, circles_out, nullptr, nullptr, nullptr, 0, nullptr,
                            nullptr, st));
  }
  GFS_CK(cudaStreamSynchronize(st));
  return GFS_OK;
}

int gfs_exact_rmin(gfs_ctx* c, const double* x, const int8_t* sigma, int64_t m, double* rmin_out) {
  if (!c || m < 0 || (m > 0 && (!x || !sigma || !rmin_out))) return GFS_ERR_ARG;
  if (!c->built) return GFS_ERR_STATE;
  if (m == 0) return GFS_OK;
  GFS_TRY(ud_compute(c));
  QueryArgs a;
  fill_query_args(c, a);
  const exact::UDLists L{c->ud_quad.as<int64_t>(), c->ud_pts.as<double>(), c->ud_np, c->ud_circ.as<int64_t>(),
                         c->ud_nc};
  GFS_CK(launch_exact_rmin(a, c->opt.box_cull, L, x, sigma, m, rmin_out, c->stream));
  return GFS_OK;
}

int gfs_cell_coverage(gfs_ctx* c, const int32_t* cells, int64_t ncells, const double* origin_host, double h,
                      int sub, uint32_t* counts_out) {
  if (!c || ncells < 0 || !origin_host || !(h > 0.0) || sub < 1 || sub > 64) return GFS_ERR_ARG;
  if (ncells > 0 && (!cells || !counts_out)) return GFS_ERR_ARG;
  if (!c->built) return GFS_ERR_STATE;
  if (ncells == 0) return GFS_OK;
  QueryArgs a;
  fill_query_args(c, a);
  GFS_CK(launch_cell_coverage(a, cells, ncells, origin_host, h, sub, counts_out, c->stream));
  return GFS_OK;
}

int gfs_query_tangent(gfs_ctx* c, const void* x, int x_is_fp32, int64_t m, float* s_out, double* s64_out,
                      int64_t* argmin_out, uint16_t* flags_out) {
  if (!c || m < 0 || (m > 0 && (!x || !argmin_out || !flags_out))) return GFS_ERR_ARG;
  if (!c->built) return GFS_ERR_STATE;
  if (m >= (int64_t(1) << 32)) return GFS_ERR_TOO_LARGE;
  if (m == 0) return GFS_OK;
  QueryArgs a;
  fill_query_args(c, a);
  if (x_is_fp32) a.x32 = static_cast<const float*>(x);
  else a.x64 = static_cast<const double*>(x);
  a.m = m;
  a.s_out = s_out;
  a.s64_out = s64_out;
  a.arg_out = argmin_out;
  a.fl_out = flags_out;
  // Morton order of the points (as in gfs_query)
  GFS_TRY(ensure(c->qk_in, size_t(m) * 4));
  GFS_TRY(ensure(c->qk_out, size_t(m) * 4));
  GFS_TRY(ensure(c->qv_in, size_t(m) * 4));
  GFS_TRY(ensure(c->qv_out, size_t(m) * 4));
  GFS_CK(launch_query_keys(a.x64, a.x32, m, c->qk_in.as<uint32_t>(), c->qv_in.as<int>(), c->stream));
  GFS_TRY(sort_u32_pairs(c, c->qk_in.as<uint32_t>(), c->qk_out.as<uint32_t>(), c->qv_in.as<int>(),
                         c->qv_out.as<int>(), m));
  a.perm = reinterpret_cast<const uint32_t*>(c->qv_out.p);
  GFS_CK(launch_query_tangent(a, c->opt.box_cull, c->stream));
  return GFS_OK;
}

int gfs_query_scored(gfs_ctx* c, const void* x, int x_is_fp32, int64_t m, float* s_out, double* s64_out,
                     int64_t* argmin_out, uint16_t* flags_out) {
  if (!c || m < 0 || (m > 0 && (!x || !argmin_out || !flags_out))) return GFS_ERR_ARG;
  if (!c->built) return GFS_ERR_STATE;
  if (m >= (int64_t(1) << 32)) return GFS_ERR_TOO_LARGE;
  if (m == 0) return GFS_OK;
  cudaStream_t st = c->stream;
  // per-sphere survivor lists of the current state (built once per state)
  if (c->csr_state != c->state_id) {
    const int64_t tot = int64_t(c->nsurv[0]) + c->nsurv[1];
    Scratch ids_s, cnt_s;  // released on every return
    DevBuf& ids = ids_s.b;
    DevBuf& cnt = cnt_s.b;
    GFS_TRY(ensure(ids, size_t(tot) * 4 + 16));
    GFS_TRY(ensure(cnt, 16));
    GFS_TRY(ensure(c->csr_ids, size_t(tot) * 4 + 16));
    GFS_TRY(ensure(c->csr_off, size_t(c->n + 1) * 8));
    unsigned hc = 0;
    GFS_CK(cudaMemsetAsync(cnt.p, 0, 4, st));
    GFS_CK(launch_collect_ids(c->surv_raw[0].as<float4>(), c->nsurv[0], c->surv_raw[1].as<float4>(), c->nsurv[1],
                              c->sph64.as<D4>(), c->KS, ids.as<uint32_t>(), cnt.as<unsigned int>(), st));
    GFS_CK(cudaMemcpyAsync(&hc, cnt.p, 4, cudaMemcpyDeviceToHost, st));
    GFS_CK(cudaStreamSynchronize(st));
    if (hc > 0) {
      size_t bytes = 0;
      GFS_CK(sort_keys_u32(nullptr, bytes, ids.as<uint32_t>(), c->csr_ids.as<uint32_t>(), hc, st));
      GFS_TRY(cub_ensure(c, bytes));
      bytes = c->cub_temp.bytes;
      GFS_CK(sort_keys_u32(c->cub_temp.p, bytes, ids.as<uint32_t>(), c->csr_ids.as<uint32_t>(), hc, st));
    }
    GFS_CK(launch_csr_offsets(c->csr_ids.as<uint32_t>(), int64_t(hc), c->n, c->KS, c->csr_off.as<int64_t>(), st));
    GFS_CK(cudaStreamSynchronize(st));
    c->csr_state = c->state_id;
  }
  QueryArgs a;
  fill_query_args(c, a);
  if (x_is_fp32) a.x32 = static_cast<const float*>(x);
  else a.x64 = static_cast<const double*>(x);
  a.m = m;
  a.s_out = s_out;
  a.s64_out = s64_out;
  a.arg_out = argmin_out;
  a.fl_out = flags_out;
  GFS_TRY(ensure(c->qk_in, size_t(m) * 4));
  GFS_TRY(ensure(c->qk_out, size_t(m) * 4));
  GFS_TRY(ensure(c->qv_in, size_t(m) * 4));
  GFS_TRY(ensure(c->qv_out, size_t(m) * 4));
  GFS_CK(launch_query_keys(a.x64, a.x32, m, c->qk_in.as<uint32_t>(), c->qv_in.as<int>(), st));
  GFS_TRY(sort_u32_pairs(c, c->qk_in.as<uint32_t>(), c->qk_out.as<uint32_t>(), c->qv_in.as<int>(),
                         c->qv_out.as<int>(), m));
  a.perm = reinterpret_cast<const uint32_t*>(c->qv_out.p);
  GFS_TRY(ensure(c->scored_status, 16));
  GFS_CK(cudaMemsetAsync(c->scored_status.p, 0, 4, st));
  GFS_CK(launch_query_scored(a, c->opt.box_cull, c->csr_ids.as<uint32_t>(), c->csr_off.as<int64_t>(),
                             c->scored_status.as<unsigned>(), st));
  unsigned status = 0;
  GFS_CK(cudaMemcpyAsync(&status, c->scored_status.p, 4, cudaMemcpyDeviceToHost, st));
  GFS_CK(cudaStreamSynchronize(st));
  return status ? GFS_ERR_TIMEOUT : GFS_OK;
}

namespace {

// Insertion rounds: window capacity, and the spheres inserted between
// hierarchy rebuilds (the step queries scan them and their candidate slots).
constexpr int kInsWindow = 4096;
constexpr int kInsDynSpheres = 8192;  // at most the step query's walk stack (8192 entries), which lists them
constexpr int kInsPasses = 4;
constexpr int kInsNear = 1024;  // the kernels' per-new-sphere list capacity (kNear)

// Compact the live survivors of both classes (hierarchy slots without a
// tombstone, then the dynamic lists) into surv_raw.
int ins_compact_survivors(gfs_ctx* c, const InsMisc& hm) {
  cudaStream_t st = c->stream;
  Scratch cnt_s;  // released on every return
  DevBuf& cnt = cnt_s.b;
  GFS_TRY(ensure(cnt, 16));
  for (int k = 0; k < 2; ++k) {
    const unsigned nd = unsigned(hm.ndyn) * unsigned(c->KS);
    const unsigned need = c->nsurv[k] + nd;
    if (size_t(need) * sizeof(float4) > c->surv_raw[k].bytes) {
      Scratch fresh;
      GFS_TRY(ensure(fresh.b, size_t(need) * sizeof(float4) + 16));
      std::swap(fresh.b, c->surv_raw[k]);  // the old buffer is released with fresh
    }
    unsigned hc = 0;
    GFS_CK(cudaMemsetAsync(cnt.p, 0, 4, st));
    GFS_CK(launch_ins_compact(c->surv_sorted[k].as<float4>(), c->ins_tomb[k].as<uint32_t>(), c->nsurv[k],
                              c->ins_dsurv[k].as<float4>(), c->ins_dtomb[k].as<uint32_t>(), nd,
                              c->surv_raw[k].as<float4>(), cnt.as<unsigned>(), st));
    GFS_CK(cudaMemcpyAsync(&hc, cnt.p, 4, cudaMemcpyDeviceToHost, st));
    GFS_CK(cudaStreamSynchronize(st));
    if (hc > kMaxSurvivors) return GFS_ERR_TOO_LARGE;
    c->nsurv[k] = hc;
    c->cap = std::max(c->cap, hc);
  }
  return GFS_OK;
}

// Mid-call rebuild: survivors compacted, the sphere hierarchy rebuilt over
// the present spheres (inputs and the spheres inserted so far, provisional
// indices), dynamic lists emptied.
int ins_rebuild_rounds(gfs_ctx* c, int64_t n0, int64_t n_present) {
  cudaStream_t st = c->stream;
  InsMisc hm;
  GFS_CK(cudaMemcpyAsync(&hm, c->ins_misc.p, sizeof(InsMisc), cudaMemcpyDeviceToHost, st));
  GFS_CK(cudaStreamSynchronize(st));
  GFS_TRY(ins_compact_survivors(c, hm));
  // the present list: inputs (written at the start of the call), then the
  // inserted spheres in the order they joined (dynamic list appended)
  const int64_t before = n_present - hm.ndyn;
  if (hm.ndyn > 0)
    GFS_CK(cudaMemcpyAsync(c->ins_present.as<int>() + before, c->ins_dyn.p, size_t(hm.ndyn) * 4,
                           cudaMemcpyDeviceToDevice, st));
  (void)n0;
  GFS_TRY(build_sphere_hierarchy(c, n_present, c->ins_present.as<int>()));
  GFS_TRY(build_point_tree(c, 0));
  GFS_TRY(build_point_tree(c, 1));
  for (int k = 0; k < 2; ++k) {
    const size_t words = (size_t(c->nsurv[k]) + 31) / 32 + 1;
    GFS_TRY(ensure(c->ins_tomb[k], words * 4));
    GFS_CK(cudaMemsetAsync(c->ins_tomb[k].p, 0, words * 4, st));
  }
  InsMisc* dm = c->ins_misc.as<InsMisc>();
  GFS_CK(cudaMemsetAsync(&dm->ndyn, 0, sizeof(int), st));
  GFS_CK(cudaMemsetAsync(&dm->ndyn_start, 0, sizeof(int), st));
  return GFS_OK;
}

}  // namespace

int gfs_insert(gfs_ctx* c, const double* y, int64_t T, double* s_out, int64_t* argmin_out, uint16_t* flags_out) {
  return gfs_insert_known(c, y, nullptr, T, s_out, argmin_out, flags_out);
}

int gfs_insert_known(gfs_ctx* c, const double* y, const double* known, int64_t T, double* s_out,
                     int64_t* argmin_out, uint16_t* flags_out) {
  if (!c || T < 0 || (T > 0 && !y)) return GFS_ERR_ARG;
  if (!c->built) return GFS_ERR_STATE;
  if (T == 0) return GFS_OK;
  cudaStream_t st = c->stream;
  const int64_t n0 = c->n;
  const int64_t cap = n0 + T + 1;
  if (uint64_t(cap) * uint64_t(c->KS) >= (uint64_t(1) << 32) || cap >= (int64_t(1) << 30)) return GFS_ERR_TOO_LARGE;
  GFS_TRY(grow_keep(c->sph64, size_t(cap) * sizeof(D4), size_t(n0) * sizeof(D4), st));
  const size_t wkeep = c->witness64.p ? std::min(c->witness64.bytes, size_t(n0) * 24) : 0;
  GFS_TRY(grow_keep(c->witness64, size_t(cap) * 24, wkeep, st));
  GFS_TRY(ensure(c->ins_counts, size_t(cap) * 4));
  GFS_TRY(ensure(c->ins_maxrem, size_t(cap) * 4));
  GFS_TRY(ensure(c->ins_lost, size_t(cap) * 4));
  GFS_TRY(ensure(c->ins_present, size_t(cap) * 4));
  GFS_TRY(ensure(c->ins_inserted, size_t(T) * 4));
  GFS_TRY(ensure(c->ins_codes, size_t(T)));
  GFS_TRY(ensure(c->ins_scan, size_t(T) * 4));
  GFS_TRY(ensure(c->ins_slot_t, size_t(kInsWindow) * 4));
  GFS_TRY(ensure(c->ins_slots, size_t(kInsWindow) * sizeof(InsSlot)));
  GFS_TRY(ensure(c->ins_cbuf, size_t(2 * kInsWindow)));
  GFS_TRY(ensure(c->ins_new, size_t(kInsWindow) * 4));
  GFS_TRY(ensure(c->ins_dyn, size_t(kInsDynSpheres) * 4));
  GFS_TRY(ensure(c->ins_dynf4, size_t(kInsDynSpheres) * sizeof(float4)));
  GFS_TRY(ensure(c->ins_near, size_t(kInsWindow) * kInsNear * 4));
  GFS_TRY(ensure(c->ins_nearcnt, size_t(kInsWindow) * 4));
  const unsigned dcap = unsigned(c->KS) * unsigned(kInsDynSpheres);
  for (int k = 0; k < 2; ++k) {
    const size_t words = (size_t(c->nsurv[k]) + 31) / 32 + 1;
    GFS_TRY(ensure(c->ins_tomb[k], words * 4));
    GFS_CK(cudaMemsetAsync(c->ins_tomb[k].p, 0, words * 4, st));
    GFS_TRY(ensure(c->ins_dsurv[k], size_t(dcap) * sizeof(float4)));
    GFS_TRY(ensure(c->ins_dtomb[k], size_t(dcap) * 4));
  }
  GFS_TRY(ensure(c->ins_misc, sizeof(InsMisc)));
  GFS_CK(cudaMemsetAsync(c->ins_counts.p, 0, size_t(cap) * 4, st));
  GFS_CK(cudaMemsetAsync(c->ins_maxrem.p, 0xff, size_t(cap) * 4, st));
  GFS_CK(cudaMemsetAsync(c->ins_inserted.p, 0, size_t(T) * 4, st));
  GFS_CK(cudaMemsetAsync(c->ins_codes.p, 0, size_t(T), st));
  GFS_CK(cudaMemsetAsync(c->ins_misc.p, 0, sizeof(InsMisc), st));
  GFS_CK(launch_ins_counts(c->surv_raw[0].as<float4>(), c->nsurv[0], c->surv_raw[1].as<float4>(), c->nsurv[1],
                           c->sph64.as<D4>(), c->KS, c->ins_counts.as<int>(), st));
  {
    std::vector<int> ids(static_cast<size_t>(n0));
    for (int64_t i = 0; i < n0; ++i) ids[size_t(i)] = int(i);
    GFS_CK(cudaMemcpyAsync(c->ins_present.p, ids.data(), size_t(n0) * 4, cudaMemcpyHostToDevice, st));
    GFS_CK(cudaStreamSynchronize(st));
  }
  InsMisc* dm = c->ins_misc.as<InsMisc>();
  c->ins_rounds = c->ins_steps = c->ins_rebuilds = c->ins_queried = 0;
  c->ins_ms_rebuild = c->ins_ms_query = c->ins_ms_commit = c->ins_ms_update = 0.0;
  // device time of the round phases (timing = 1): query, commit, update
  cudaEvent_t iev[5] = {};
  bool timed = c->have_ev;
  for (int k = 0; k < 5 && timed; ++k)
    if (cudaEventCreate(&iev[k]) != cudaSuccess) {
      cudaGetLastError();
      timed = false;
    }
  struct EvGuard {
    cudaEvent_t* e;
    ~EvGuard() {
      for (int k = 0; k < 5; ++k)
        if (e[k]) cudaEventDestroy(e[k]);
    }
  } ev_guard{iev};
  auto ev_ms = [&](int x, int y) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, iev[x], iev[y]) != cudaSuccess) {
      cudaGetLastError();
      t = 0.f;
    }
    return double(t);
  };
  bool update_pending = false;
  const auto t_start = std::chrono::steady_clock::now();
  auto ms_since = [](std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  };
  InsertArgs a;
  std::memset(&a, 0, sizeof(a));
  auto refresh_static = [&]() {
    a.sph = c->sph.as<float4>();
    a.sid = c->sid.as<int>();
    a.st = c->st;
    for (int k = 0; k < 2; ++k) {
      a.surv[k] = c->surv_sorted[k].as<float4>();
      a.vt[k] = c->vt[k];
      a.tomb[k] = c->ins_tomb[k].as<uint32_t>();
    }
    a.bc = c->consts.as<BuildConsts>();
  };
  refresh_static();
  a.n0 = int(n0);
  a.dyn_ids = c->ins_dyn.as<int>();
  a.dyn_ids_w = c->ins_dyn.as<int>();
  a.dyn_f4 = c->ins_dynf4.as<float4>();
  a.near_list = c->ins_near.as<int>();
  a.near_cnt = c->ins_nearcnt.as<int>();
  a.sph64 = c->sph64.as<D4>();
  a.witness64 = c->witness64.as<double>();
  a.counts = c->ins_counts.as<int>();
  a.maxrem = c->ins_maxrem.as<int>();
  for (int k = 0; k < 2; ++k) {
    a.dsurv[k] = c->ins_dsurv[k].as<float4>();
    a.dtomb[k] = c->ins_dtomb[k].as<uint32_t>();
  }
  a.U64 = c->U64.as<double>();
  a.K = c->K;
  a.KS = c->KS;
  a.tol = c->opt.tol;
  a.box_cull = c->opt.box_cull;
  a.clamp_opp = c->opt.clamp_opp;
  a.y = y;
  a.known = known;
  a.T = T;
  a.s_out = s_out;
  a.arg_out = argmin_out;
  a.fl_out = flags_out;
  a.slot_t = c->ins_slot_t.as<int>();
  a.slots = c->ins_slots.as<InsSlot>();
  a.cbuf = c->ins_cbuf.as<unsigned char>();
  a.wcap = kInsWindow;
  a.new_ids = c->ins_new.as<int>();
  a.lost_list = c->ins_lost.as<int>();
  a.inserted = c->ins_inserted.as<int>();
  a.codes = c->ins_codes.as<unsigned char>();
  a.misc = dm;
  // rounds: the window grows while most of it commits and shrinks when little
  // does; every round commits at least its first step
  int W = int(std::min<int64_t>(T, 64));
  double commit_rate = 0.0;  // moving average of the steps a round commits
  int nslots = 0;
  int64_t done = 0, rounds = 0;
  InsMisc hm;
  std::memset(&hm, 0, sizeof(hm));
  for (;;) {
    if (timed) GFS_CK(cudaEventRecord(iev[0], st));
    GFS_CK(launch_ins_query(a, nslots, st));
    c->ins_queried += nslots;
    if (timed) GFS_CK(cudaEventRecord(iev[1], st));
    GFS_CK(launch_ins_commit(a, nslots, kInsPasses, W, st));
    if (timed) GFS_CK(cudaEventRecord(iev[2], st));
    GFS_CK(cudaMemcpyAsync(&hm, dm, sizeof(InsMisc), cudaMemcpyDeviceToHost, st));
    GFS_CK(cudaStreamSynchronize(st));
    if (timed) {
      c->ins_ms_query += ev_ms(0, 1);
      c->ins_ms_commit += ev_ms(1, 2);
      if (update_pending) c->ins_ms_update += ev_ms(3, 4);
      update_pending = false;
    }
    if (hm.err) return GFS_ERR_CUDA;
    ++rounds;
    done += hm.ncommit;
    if (hm.nnew > 0) {
      if (timed) GFS_CK(cudaEventRecord(iev[3], st));
      GFS_CK(launch_ins_update(a, hm.nnew, hm.ndyn_start, st));
      if (timed) {
        GFS_CK(cudaEventRecord(iev[4], st));
        update_pending = true;
      }
    }
    if (nslots > 0) {
      if (2 * hm.ncommit >= nslots) W = std::min(kInsWindow, 2 * W);
      else if (8 * hm.ncommit < nslots) W = std::max(1, W / 2);
    }
    nslots = hm.npend;
    if (hm.npend == 0 && hm.next >= T) break;
    if (rounds > 4 * T + 8) return GFS_ERR_TIMEOUT;  // every round commits at least one step
    // rebuild when the dynamic sphere list has no room for the next round's
    // spheres, or when it has grown long for the rate at which rounds commit
    // (every step query scans it and the slots of the spheres near its point;
    // a rebuild costs about as much as a few dozen rounds)
    commit_rate = 0.9 * commit_rate + 0.1 * double(hm.ncommit);
    const int dyn_soft = int(std::min(double(kInsDynSpheres - kInsWindow), std::max(256.0, 64.0 * commit_rate)));
    if (hm.ndyn + kInsWindow > kInsDynSpheres || hm.ndyn >= dyn_soft) {
      const auto t_rb = std::chrono::steady_clock::now();
      GFS_TRY(ins_rebuild_rounds(c, n0, n0 + hm.ninserted));
      refresh_static();
      ++c->ins_rebuilds;
      c->ins_ms_rebuild += ms_since(t_rb);
    }
  }
  c->ins_rounds = rounds;
  c->ins_steps = done;
  const auto t_final = std::chrono::steady_clock::now();
  // renumber the inserted spheres consecutively (step order) and rebuild
  GFS_CK(cudaMemcpyAsync(&hm, dm, sizeof(InsMisc), cudaMemcpyDeviceToHost, st));
  GFS_CK(cudaStreamSynchronize(st));
  if (timed && update_pending) c->ins_ms_update += ev_ms(3, 4);
  if (hm.err) return GFS_ERR_CUDA;
  GFS_TRY(ins_compact_survivors(c, hm));
  {
    size_t bytes = 0;
    GFS_CK(exclusive_scan_i32(nullptr, bytes, c->ins_inserted.as<int>(), c->ins_scan.as<int>(), T, st));
    GFS_TRY(cub_ensure(c, bytes));
    bytes = c->cub_temp.bytes;
    GFS_CK(exclusive_scan_i32(c->cub_temp.p, bytes, c->ins_inserted.as<int>(), c->ins_scan.as<int>(), T, st));
  }
  const int64_t n_final = n0 + hm.ninserted;
  {
    Scratch sph_new, wit_new;  // after the swaps they hold (and release) the old arrays
    GFS_TRY(ensure(sph_new.b, std::max(c->sph64.bytes, size_t(cap) * sizeof(D4))));
    GFS_TRY(ensure(wit_new.b, std::max(c->witness64.bytes, size_t(cap) * 24)));
    GFS_CK(launch_ins_renumber(a, c->ins_scan.as<int>(), sph_new.b.as<D4>(), wit_new.b.as<double>(), st));
    GFS_CK(cudaStreamSynchronize(st));
    std::swap(sph_new.b, c->sph64);
    std::swap(wit_new.b, c->witness64);
  }
  for (int k = 0; k < 2; ++k)
    GFS_CK(launch_ins_remap_survivors(c->surv_raw[k].as<float4>(), c->nsurv[k], c->ins_scan.as<int>(), int(n0),
                                      c->KS, st));
  GFS_TRY(build_sphere_hierarchy(c, n_final));
  GFS_TRY(build_point_tree(c, 0));
  GFS_TRY(build_point_tree(c, 1));
  GFS_CK(cudaStreamSynchronize(st));
  c->ins_ms_final = ms_since(t_final);
  ++c->state_id;
  for (int k = 0; k < 4; ++k) c->ins_work[k] = hm.work[k];
  c->ins_ms_total = ms_since(t_start);
  return GFS_OK;
}

int gfs_survivors(gfs_ctx* c, int64_t* g_out, int64_t cap, int64_t* count_host) {
  if (!c || !count_host || cap < 0) return GFS_ERR_ARG;
  if (!c->built) return GFS_ERR_STATE;
  const int64_t tot = int64_t(c->nsurv[0]) + c->nsurv[1];
  DevBuf ids, sorted, cnt;
  int stt = ensure(ids, size_t(tot) * 4 + 16);
  if (stt == GFS_OK) stt = ensure(sorted, size_t(tot) * 4 + 16);
  if (stt == GFS_OK) stt = ensure(cnt, 16);
  unsigned int hc = 0;
  if (stt == GFS_OK) {
    if (cudaMemsetAsync(cnt.p, 0, 4, c->stream) != cudaSuccess ||
        launch_collect_ids(c->surv_raw[0].as<float4>(), c->nsurv[0], c->surv_raw[1].as<float4>(), c->nsurv[1],
                           c->sph64.as<D4>(), c->KS, ids.as<uint32_t>(), cnt.as<unsigned int>(),
                           c->stream) != cudaSuccess ||
        cudaMemcpyAsync(&hc, cnt.p, 4, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
      cudaGetLastError();
      stt = GFS_ERR_CUDA;
    }
  }
  if (stt == GFS_OK) {
    *count_host = hc;
    if (hc > 0 && cap >= int64_t(hc) && g_out) {
      size_t bytes = 0;
      if (sort_keys_u32(nullptr, bytes, ids.as<uint32_t>(), sorted.as<uint32_t>(), hc, c->stream) != cudaSuccess ||
          cub_ensure(c, bytes) != GFS_OK) {
        stt = GFS_ERR_CUDA;
      } else {
        bytes = c->cub_temp.bytes;
        if (sort_keys_u32(c->cub_temp.p, bytes, ids.as<uint32_t>(), sorted.as<uint32_t>(), hc, c->stream) !=
                cudaSuccess ||
            launch_widen_ids(sorted.as<uint32_t>(), hc, g_out, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess) {
          cudaGetLastError();
          stt = GFS_ERR_CUDA;
        }
      }
    } else if (cap < int64_t(hc)) {
      stt = GFS_ERR_ARG;
    }
  }
  release(ids);
  release(sorted);
  release(cnt);
  return stt;
}

// ---------------------------------------------------------------------------
// batched shapes
// ---------------------------------------------------------------------------
namespace {

static_assert(sizeof(gfs_shape) == sizeof(ShapeDesc), "gfs_shape and ShapeDesc must share a layout");

// Lay out one tree per shape inside shared node arrays: each shape's tree
// pointers are offset to its block of nodes; level offsets stay local.
int64_t forest_layout(std::vector<Tree>& trees, const std::vector<int64_t>& nitems, float4* lo, float4* hi,
                      float4* na, float4* nb, float4* nf, int& max_levels) {
  int64_t base = 0;
  max_levels = 0;
  for (size_t s = 0; s < nitems.size(); ++s) {
    Tree& T = trees[s];
    tree_layout(T, nitems[s]);
    T.lo = lo ? lo + base : nullptr;
    T.hi = hi ? hi + base : nullptr;
    T.na = na ? na + base : nullptr;
    T.nb = nb ? nb + base : nullptr;
    T.nf = nf ? nf + base : nullptr;
    base += tree_nodes(T);
    max_levels = std::max(max_levels, T.nlevels);
  }
  return base;
}

// time one persistent query launch configuration (both phases) on a prefix
// of the work
float time_grid(gfs_ctx* c, int grid, int64_t limit) {
  cudaStream_t st = c->stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  for (int phase = 1; phase <= 2; ++phase) {
    cudaMemsetAsync(c->b_ctr.p, 0, 8, st);
    launch_batch_query(c->b_qviews.as<QueryArgs>(), c->b_qw.as<int64_t>(), c->b_ns, limit,
                       c->b_ctr.as<unsigned long long>(), grid, phase, st);
  }
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms;
}

// the persistent query's grid: blocks per SM picked by timing a prefix
int autotune_grid(gfs_ctx* c, int64_t total) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int cand[] = {2, 3, 4, 5, 6, 8};
  const int64_t limit = std::min<int64_t>(total, std::max<int64_t>(int64_t(sms) * 256, total / 16));
  int best = sms * 4;
  float best_ms = 1e30f;
  for (int m : cand) {
    const float ms = time_grid(c, sms * m, limit);
    if (ms < best_ms) {
      best_ms = ms;
      best = sms * m;
    }
  }
  cudaGetLastError();
  return best;
}

}  // namespace

namespace {

// Size class of a shape for the cull tile choice: up to 32k, up to 256k, more.
int batch_size_class(int64_t n) { return n < 32768 ? 0 : (n < 262144 ? 1 : 2); }

// Levels of the sample forest (static layout uploaded by the first build).
int batch_sphere_levels(gfs_ctx* c) {
  const int ns = c->b_ns;
  const size_t io = size_t(ns + 1) * std::max(1, c->b_sph_levels);
  for (int l = 0; l < c->b_sph_levels; ++l)
    GFS_CK(launch_batch_tree_level(c->b_stdev.as<Tree>(), c->b_prefix.as<int64_t>() + size_t(l) * (ns + 1),
                                   c->b_sph_level_total[size_t(l)], ns, l, c->b_sph.as<float4>(),
                                   c->b_prefix.as<int64_t>() + io, c->b_bcs.as<BuildConsts>(), 1, c->stream));
  return GFS_OK;
}

// The sample part of the device-side build (copy, sort, sample forest).
int batch_build_device_samples(gfs_ctx* c) {
  cudaStream_t st = c->stream;
  const int ns = c->b_ns;
  const int64_t N = c->b_off[size_t(ns)];
  GFS_CK(cudaMemsetAsync(c->b_bits.p, 0, size_t(ns) * 8, st));
  GFS_CK(launch_batch_copy(c->b_desc.as<ShapeDesc>(), c->b_offd.as<int64_t>(), ns, N, c->b_sph64.as<D4>(),
                           c->b_k64in.as<unsigned long long>(), c->vals_in.as<int>(), c->b_bits.as<unsigned int>(),
                           c->b_bcs.as<BuildConsts>(), st));
  size_t bytes = c->cub_temp.bytes;
  GFS_CK(sort_pairs64(c->cub_temp.p, bytes, c->b_k64in.as<unsigned long long>(), c->b_k64out.as<unsigned long long>(),
                      c->vals_in.as<int>(), c->vals_out.as<int>(), N, c->b_end_bit, st));
  GFS_CK(launch_batch_gather(c->b_sph64.as<D4>(), c->vals_out.as<int>(), c->b_offd.as<int64_t>(), ns, N,
                             c->b_bcs.as<BuildConsts>(), float(c->opt.tol), c->opt.tol, c->b_sph.as<float4>(),
                             c->b_thr.as<float4>(), c->b_sid.as<int>(), st));
  return batch_sphere_levels(c);
}

// The part of the batched build that depends on the sample values only:
// inputs copied and Morton-sorted, sample forest, cull, survivor forests and
// query views, all on the device with the sizes and capacities the first
// build fixed.  No host synchronisation, allocation or host-to-device copy.
int batch_build_device(gfs_ctx* c, bool cull_only) {
  cudaStream_t st = c->stream;
  const int ns = c->b_ns;
  const int64_t N = c->b_off[size_t(ns)];
  (void)N;
  if (!cull_only) GFS_TRY(batch_build_device_samples(c));
  GFS_CK(cudaMemsetAsync(c->b_cnt.p, 0, sizeof(Counters), st));
  for (int k = 0; k < 3; ++k)
    GFS_CK(launch_batch_cull_blocks(c->b_cviews.as<CullArgs>() + c->b_cls_off[k],
                                    c->b_cw.as<int64_t>() + c->b_cls_off[k] + k, c->b_cls_off[k + 1] - c->b_cls_off[k],
                                    c->b_cls_blocks[k], c->b_tile[k], st));
  if (cull_only) return GFS_OK;
  for (int k = 0; k < 2; ++k)
    GFS_CK(launch_batch_surv_forest(
        c->b_sshape[k].as<uint16_t>(), c->b_sraw[k].as<float4>(), c->b_cnt.as<Counters>(), k, c->b_cap, ns,
        c->b_hist.as<unsigned>(), c->b_k64in.as<unsigned long long>(), c->b_k64out.as<unsigned long long>(),
        c->vals_in.as<int>(), c->vals_out.as<int>(), c->cub_temp.p, c->cub_temp.bytes, c->b_end_bit,
        c->b_ssorted[k].as<float4>(), c->b_node_cap, c->b_vlo[k].as<float4>(), c->b_vhi[k].as<float4>(),
        c->b_vtdev[k].as<Tree>(), c->b_vprefix[k].as<int64_t>(), c->b_surv_levels, c->b_sodev[k].as<int64_t>(),
        c->b_qviews.as<QueryArgs>(), c->b_status.as<unsigned>(), st));
  return GFS_OK;
}

// Host copies of what the device-side build laid out (survivor offsets and
// the query views): read back whenever a host-driven call needs them (a
// rebuild replayed from a captured graph changes them without the host).
int batch_sync_host(gfs_ctx* c) {
  const int ns = c->b_ns;
  cudaStream_t st = c->stream;
  for (int k = 0; k < 2; ++k) {
    c->b_soff[k].assign(size_t(ns) + 1, 0);
    GFS_CK(cudaMemcpyAsync(c->b_soff[k].data(), c->b_sodev[k].p, size_t(ns + 1) * 8, cudaMemcpyDeviceToHost, st));
  }
  c->b_qv.resize(size_t(ns));
  GFS_CK(cudaMemcpyAsync(c->b_qv.data(), c->b_qviews.p, size_t(ns) * sizeof(QueryArgs), cudaMemcpyDeviceToHost, st));
  GFS_CK(cudaStreamSynchronize(st));
  return GFS_OK;
}

}  // namespace

int gfs_batch_build(gfs_ctx* c, const gfs_shape* shapes, int ns) {
  if (!c || !shapes || ns < 1 || ns > 65535) return GFS_ERR_ARG;
  cudaStream_t st = c->stream;
  c->b_built = false;
  c->b_ns = ns;
  c->b_shapes.assign(shapes, shapes + ns);
  std::vector<int64_t> off(ns + 1), qoff(ns + 1);
  off[0] = qoff[0] = 0;
  for (int s = 0; s < ns; ++s) {
    if (shapes[s].n < 1 || !shapes[s].p_xyz || !shapes[s].s || shapes[s].m < 0 || (shapes[s].m > 0 && !shapes[s].x))
      return GFS_ERR_ARG;
    if (uint64_t(shapes[s].n) * uint64_t(c->KS) >= (uint64_t(1) << 32) || shapes[s].m >= (int64_t(1) << 31))
      return GFS_ERR_TOO_LARGE;
    off[s + 1] = off[s] + shapes[s].n;
    qoff[s + 1] = qoff[s] + shapes[s].m;
  }
  const int64_t N = off[ns], M = qoff[ns];
  if (N >= (int64_t(1) << 31)) return GFS_ERR_TOO_LARGE;
  c->b_off = off;
  c->b_qoff = qoff;
  c->b_end_bit = 32;
  while ((int64_t(1) << (c->b_end_bit - 32)) < ns) ++c->b_end_bit;
  GFS_TRY(ensure(c->b_desc, size_t(ns) * sizeof(ShapeDesc)));
  GFS_TRY(ensure(c->b_offd, size_t(ns + 1) * 8));
  GFS_TRY(ensure(c->b_qoffd, size_t(ns + 1) * 8));
  GFS_CK(cudaMemcpyAsync(c->b_desc.p, shapes, size_t(ns) * sizeof(ShapeDesc), cudaMemcpyHostToDevice, st));
  GFS_CK(cudaMemcpyAsync(c->b_offd.p, off.data(), size_t(ns + 1) * 8, cudaMemcpyHostToDevice, st));
  GFS_CK(cudaMemcpyAsync(c->b_qoffd.p, qoff.data(), size_t(ns + 1) * 8, cudaMemcpyHostToDevice, st));
  // samples: copy, Morton sort by (shape, code), sorted FP32 copies
  GFS_TRY(ensure(c->b_sph64, size_t(N) * sizeof(D4)));
  GFS_TRY(ensure(c->b_k64in, size_t(std::max(N, M)) * 8));
  GFS_TRY(ensure(c->b_k64out, size_t(std::max(N, M)) * 8));
  GFS_TRY(ensure(c->vals_in, size_t(N) * 4));
  GFS_TRY(ensure(c->vals_out, size_t(N) * 4));
  GFS_TRY(ensure(c->b_sph, size_t(N) * sizeof(float4)));
  GFS_TRY(ensure(c->b_thr, size_t(N) * sizeof(float4)));
  GFS_TRY(ensure(c->b_sid, size_t(N) * 4));
  GFS_TRY(ensure(c->b_bits, size_t(ns) * 8));
  GFS_TRY(ensure(c->b_bcs, size_t(ns) * sizeof(BuildConsts)));
  GFS_TRY(ensure(c->b_hist, size_t(ns) * 4));
  GFS_TRY(ensure(c->b_status, 16));
  GFS_CK(cudaMemsetAsync(c->b_status.p, 0, 16, st));
  {
    size_t bytes = 0;
    GFS_CK(sort_pairs64(nullptr, bytes, c->b_k64in.as<unsigned long long>(), c->b_k64out.as<unsigned long long>(),
                        c->vals_in.as<int>(), c->vals_out.as<int>(), N, c->b_end_bit, st));
    GFS_TRY(ensure(c->cub_temp, bytes));
  }
  // sample forest: static layout (depends on the sample counts only)
  c->b_st.assign(ns, Tree{});
  std::vector<int64_t> nits(ns);
  for (int s = 0; s < ns; ++s) nits[s] = shapes[s].n;
  int maxL = 0;
  const int64_t nodes = forest_layout(c->b_st, nits, nullptr, nullptr, nullptr, nullptr, nullptr, maxL);
  GFS_TRY(ensure(c->b_lo, size_t(nodes) * sizeof(float4)));
  GFS_TRY(ensure(c->b_hi, size_t(nodes) * sizeof(float4)));
  GFS_TRY(ensure(c->b_na, size_t(nodes) * sizeof(float4)));
  GFS_TRY(ensure(c->b_nb, size_t(nodes) * sizeof(float4)));
  GFS_TRY(ensure(c->b_nf, size_t(nodes) * sizeof(float4)));
  forest_layout(c->b_st, nits, c->b_lo.as<float4>(), c->b_hi.as<float4>(), c->b_na.as<float4>(), c->b_nb.as<float4>(),
                c->b_nf.as<float4>(), maxL);
  {
    GFS_TRY(ensure(c->b_stdev, size_t(ns) * sizeof(Tree)));
    GFS_CK(cudaMemcpyAsync(c->b_stdev.p, c->b_st.data(), size_t(ns) * sizeof(Tree), cudaMemcpyHostToDevice, st));
    std::vector<int64_t> pre(size_t(ns + 1) * std::max(1, maxL) + size_t(ns));
    c->b_sph_level_total.assign(size_t(std::max(1, maxL)), 0);
    for (int l = 0; l < maxL; ++l) {
      int64_t acc = 0;
      for (int s = 0; s < ns; ++s) {
        pre[size_t(l) * (ns + 1) + s] = acc;
        acc += c->b_st[s].nlevels > l ? c->b_st[s].count[l] : 0;
      }
      pre[size_t(l) * (ns + 1) + ns] = acc;
      c->b_sph_level_total[size_t(l)] = acc;
    }
    const size_t io = size_t(ns + 1) * std::max(1, maxL);
    for (int s = 0; s < ns; ++s) pre[io + s] = off[s];
    GFS_TRY(ensure(c->b_prefix, pre.size() * 8));
    GFS_CK(cudaMemcpyAsync(c->b_prefix.p, pre.data(), pre.size() * 8, cudaMemcpyHostToDevice, st));
    GFS_CK(cudaStreamSynchronize(st));  // the pageable host arrays above are copied before they go out of scope
    c->b_sph_levels = maxL;
  }
  // culling views and work items (shape, direction, 128 spheres)
  const uint64_t ncand = uint64_t(N) * uint64_t(c->K);
  // survivors are typically < 1% of the candidates; the cull is rerun with
  // room for the counted survivors if this first capacity overflows
  uint64_t cap = std::max<uint64_t>(uint64_t(1) << 16, ncand / 64 + 1024);
  cap = std::min<uint64_t>(cap, 0xfffffff0u);
  GFS_TRY(ensure(c->b_ctr, 16));
  GFS_TRY(ensure(c->b_cnt, sizeof(Counters)));
  GFS_TRY(ensure(c->b_cviews, size_t(ns) * sizeof(CullArgs)));
  // the samples (the cull reads them) -- built once here, then the cull is
  // repeated until its survivor capacity suffices
  GFS_TRY(batch_build_device_samples(c));
  // size classes of the shapes (the cull tile is chosen per class)
  c->b_cls_order.clear();
  for (int k = 0; k < 3; ++k) {
    c->b_cls_off[k] = int(c->b_cls_order.size());
    for (int s = 0; s < ns; ++s)
      if (batch_size_class(shapes[s].n) == k) c->b_cls_order.push_back(s);
  }
  c->b_cls_off[3] = ns;
  // upload the views and the per-class block prefixes for the current tiles
  auto upload_cull = [&](unsigned capv) -> int {
    std::vector<CullArgs> cv(ns);
    std::vector<int64_t> cw(size_t(ns) + 3);
    for (int k = 0; k < 3; ++k) {
      int64_t acc = 0;
      for (int v = c->b_cls_off[k]; v < c->b_cls_off[k + 1]; ++v) {
        const int s = c->b_cls_order[size_t(v)];
        CullArgs& a = cv[size_t(v)];
        std::memset(&a, 0, sizeof(a));
        a.sph = c->b_sph.as<float4>() + off[s];
        a.thr = c->b_thr.as<float4>() + off[s];
        a.sid = c->b_sid.as<int>() + off[s];
        a.sph64 = c->b_sph64.as<D4>() + off[s];
        a.U32 = c->U32.as<float>();
        a.U64 = c->U64.as<double>();
        a.K = c->K;
        a.KS = c->KS;
        a.tree = c->b_st[s];
        a.tol32 = float(c->opt.tol);
        a.tol = c->opt.tol;
        a.box_cull = c->opt.box_cull;
        a.bc = c->b_bcs.as<BuildConsts>() + s;
        a.n = shapes[s].n;
        a.surv[0] = c->b_sraw[0].as<float4>();
        a.surv[1] = c->b_sraw[1].as<float4>();
        a.cap = capv;
        a.cnt = c->b_cnt.as<Counters>();
        a.surv_shape[0] = c->b_sshape[0].as<uint16_t>();
        a.surv_shape[1] = c->b_sshape[1].as<uint16_t>();
        a.shape = s;
        cw[size_t(v + k)] = acc;
        acc += (shapes[s].n + c->b_tile[k] - 1) / c->b_tile[k] * c->K;
      }
      cw[size_t(c->b_cls_off[k + 1] + k)] = acc;
      c->b_cls_blocks[k] = acc;
    }
    GFS_CK(cudaMemcpyAsync(c->b_cviews.p, cv.data(), size_t(ns) * sizeof(CullArgs), cudaMemcpyHostToDevice, st));
    GFS_CK(cudaMemcpyAsync(c->b_cw.p, cw.data(), cw.size() * 8, cudaMemcpyHostToDevice, st));
    GFS_CK(cudaStreamSynchronize(st));  // pageable sources
    return GFS_OK;
  };
  GFS_TRY(ensure(c->b_cw, size_t(ns + 3) * 8));
  for (int attempt = 0; attempt < 3; ++attempt) {
    c->b_cap = unsigned(cap);
    for (int k = 0; k < 2; ++k) {
      GFS_TRY(ensure(c->b_sraw[k], size_t(cap) * sizeof(float4)));
      GFS_TRY(ensure(c->b_sshape[k], size_t(cap) * 2));
    }
    GFS_TRY(upload_cull(c->b_cap));
    GFS_TRY(batch_build_device(c, true));
    Counters hc;
    GFS_CK(cudaMemcpyAsync(&hc, c->b_cnt.p, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    GFS_CK(cudaStreamSynchronize(st));
    const unsigned need = std::max(hc.nsurv[0], hc.nsurv[1]);
    c->b_nsurv[0] = hc.nsurv[0];
    c->b_nsurv[1] = hc.nsurv[1];
    if (need <= c->b_cap) break;
    cap = uint64_t(need) + need / 8 + 1024;
    if (attempt == 2) return GFS_ERR_OOM;
  }
  // cull tile per size class: each class's cull timed with tiles of 64, 128
  // and 256 spheres (the first build only; the fastest is kept), then the
  // whole cull rerun with the chosen tiles
  if (!c->b_tiles_tuned) {
    cudaEvent_t e0, e1;
    GFS_CK(cudaEventCreate(&e0));
    GFS_CK(cudaEventCreate(&e1));
    for (int k = 0; k < 3; ++k) {
      if (c->b_cls_off[k + 1] == c->b_cls_off[k]) continue;
      float best = 0.f;
      int best_tile = 128;
      for (int tile : {64, 128, 256}) {
        c->b_tile[k] = tile;
        if (upload_cull(c->b_cap) != GFS_OK) break;
        float ms = 0.f;
        if (cudaMemsetAsync(c->b_cnt.p, 0, sizeof(Counters), st) != cudaSuccess ||
            cudaEventRecord(e0, st) != cudaSuccess ||
            launch_batch_cull_blocks(c->b_cviews.as<CullArgs>() + c->b_cls_off[k],
                                     c->b_cw.as<int64_t>() + c->b_cls_off[k] + k,
                                     c->b_cls_off[k + 1] - c->b_cls_off[k], c->b_cls_blocks[k], tile, st) !=
                cudaSuccess ||
            cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          cudaGetLastError();
          break;
        }
        if (best == 0.f || ms < best) {
          best = ms;
          best_tile = tile;
        }
      }
      c->b_tile[k] = best_tile;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->b_tiles_tuned = true;
    GFS_TRY(upload_cull(c->b_cap));
    GFS_TRY(batch_build_device(c, true));
  }
  if (std::max(c->b_nsurv[0], c->b_nsurv[1]) > kMaxSurvivors) return GFS_ERR_TOO_LARGE;
  // survivor forests: sized for the capacity (the layout is computed on the
  // device from the counts, so later rebuilds need no host round trip)
  const unsigned capu = c->b_cap;
  c->b_node_cap = int64_t(capu) / (kLeaf - 1) + int64_t(ns) * (kMaxLevels + 1) + 16;
  {
    Tree T;
    tree_layout(T, int64_t(capu));
    c->b_surv_levels = std::max(1, T.nlevels);
  }
  GFS_TRY(ensure(c->b_k64in, size_t(std::max<int64_t>(std::max(N, M), capu)) * 8));
  GFS_TRY(ensure(c->b_k64out, size_t(std::max<int64_t>(std::max(N, M), capu)) * 8));
  GFS_TRY(ensure(c->vals_in, size_t(std::max<int64_t>(N, capu)) * 4));
  GFS_TRY(ensure(c->vals_out, size_t(std::max<int64_t>(N, capu)) * 4));
  for (int k = 0; k < 2; ++k) {
    GFS_TRY(ensure(c->b_ssorted[k], size_t(capu) * sizeof(float4) + 16));
    GFS_TRY(ensure(c->b_vlo[k], size_t(c->b_node_cap) * sizeof(float4)));
    GFS_TRY(ensure(c->b_vhi[k], size_t(c->b_node_cap) * sizeof(float4)));
    GFS_TRY(ensure(c->b_vtdev[k], size_t(ns) * sizeof(Tree)));
    GFS_TRY(ensure(c->b_vprefix[k], size_t(c->b_surv_levels) * (ns + 1) * 8));
    GFS_TRY(ensure(c->b_sodev[k], size_t(ns + 1) * 8));
  }
  {
    size_t bytes = 0;
    GFS_CK(sort_pairs64(nullptr, bytes, c->b_k64in.as<unsigned long long>(), c->b_k64out.as<unsigned long long>(),
                        c->vals_in.as<int>(), c->vals_out.as<int>(), int64_t(capu), c->b_end_bit, st));
    GFS_TRY(ensure(c->cub_temp, bytes));
  }
  // query views and work items (shape, 32 points); the survivor pointers and
  // trees are filled in by the device-side survivor forests
  std::vector<QueryArgs> qv(ns);
  std::vector<int64_t> qw(ns + 1);
  qw[0] = 0;
  GFS_TRY(ensure(c->b_qkin, size_t(std::max<int64_t>(M, 1)) * 8));
  GFS_TRY(ensure(c->b_qkout, size_t(std::max<int64_t>(M, 1)) * 8));
  GFS_TRY(ensure(c->b_qvin, size_t(std::max<int64_t>(M, 1)) * 4));
  GFS_TRY(ensure(c->b_qvout, size_t(std::max<int64_t>(M, 1)) * 4));
  GFS_TRY(ensure(c->b_qstate, size_t(std::max<int64_t>(M, 1)) * 3 * sizeof(uint4)));
  for (int s = 0; s < ns; ++s) {
    QueryArgs& a = qv[s];
    std::memset(&a, 0, sizeof(a));
    a.sph = c->b_sph.as<float4>() + off[s];
    a.thr = c->b_thr.as<float4>() + off[s];
    a.sid = c->b_sid.as<int>() + off[s];
    a.sph64 = c->b_sph64.as<D4>() + off[s];
    a.st = c->b_st[s];
    a.n = shapes[s].n;
    a.U64 = c->U64.as<double>();
    a.K = c->K;
    a.KS = c->KS;
    a.tol32 = float(c->opt.tol);
    a.tol = c->opt.tol;
    a.clamp_opp = c->opt.clamp_opp;
    a.bc = c->b_bcs.as<BuildConsts>() + s;
    if (shapes[s].x_is_fp32) a.x32 = static_cast<const float*>(shapes[s].x);
    else a.x64 = static_cast<const double*>(shapes[s].x);
    a.m = shapes[s].m;
    a.perm = reinterpret_cast<const uint32_t*>(c->b_qvout.as<int>() + qoff[s]);
    a.state = reinterpret_cast<uint4*>(c->b_qstate.p) + 3 * qoff[s];
    a.s_out = shapes[s].s_out;
    a.s64_out = shapes[s].s64_out;
    a.arg_out = shapes[s].argmin_out;
    a.fl_out = shapes[s].flags_out;
    a.cnt = c->b_cnt.as<Counters>();
    qw[s + 1] = qw[s] + (shapes[s].m + 31) / 32;
  }
  GFS_TRY(ensure(c->b_qviews, size_t(ns) * sizeof(QueryArgs)));
  GFS_TRY(ensure(c->b_qw, size_t(ns + 1) * 8));
  GFS_CK(cudaMemcpyAsync(c->b_qviews.p, qv.data(), size_t(ns) * sizeof(QueryArgs), cudaMemcpyHostToDevice, st));
  GFS_CK(cudaMemcpyAsync(c->b_qw.p, qw.data(), size_t(ns + 1) * 8, cudaMemcpyHostToDevice, st));
  c->b_M = M;
  c->b_qtotal = qw[ns];
  // sort scratch for the query order, sized here so gfs_batch_query allocates nothing
  size_t bytes = 0;
  GFS_CK(sort_pairs64(nullptr, bytes, c->b_qkin.as<unsigned long long>(), c->b_qkout.as<unsigned long long>(),
                      c->b_qvin.as<int>(), c->b_qvout.as<int>(), M, 64, st));
  GFS_TRY(ensure(c->cub_temp, bytes));
  GFS_CK(cudaStreamSynchronize(st));  // qv, qw (pageable) copied before they go out of scope
  // the survivor forests and the views' survivor parts, on the device
  for (int k = 0; k < 2; ++k)
    GFS_CK(launch_batch_surv_forest(
        c->b_sshape[k].as<uint16_t>(), c->b_sraw[k].as<float4>(), c->b_cnt.as<Counters>(), k, c->b_cap, ns,
        c->b_hist.as<unsigned>(), c->b_k64in.as<unsigned long long>(), c->b_k64out.as<unsigned long long>(),
        c->vals_in.as<int>(), c->vals_out.as<int>(), c->cub_temp.p, c->cub_temp.bytes, c->b_end_bit,
        c->b_ssorted[k].as<float4>(), c->b_node_cap, c->b_vlo[k].as<float4>(), c->b_vhi[k].as<float4>(),
        c->b_vtdev[k].as<Tree>(), c->b_vprefix[k].as<int64_t>(), c->b_surv_levels, c->b_sodev[k].as<int64_t>(),
        c->b_qviews.as<QueryArgs>(), c->b_status.as<unsigned>(), st));
  c->b_built = true;
  GFS_TRY(batch_sync_host(c));
  if (c->b_grid_query == 0 && c->b_qtotal > 0) {
    GFS_TRY(gfs_batch_query(c));  // produces the Morton order used while tuning
    c->b_grid_query = autotune_grid(c, c->b_qtotal);
  }
  GFS_CK(cudaStreamSynchronize(st));
  return GFS_OK;
}

int gfs_batch_rebuild(gfs_ctx* c) {
  if (!c) return GFS_ERR_ARG;
  if (!c->b_built) return GFS_ERR_STATE;
  return batch_build_device(c, false);
}

int gfs_batch_status(gfs_ctx* c, unsigned* status_host) {
  if (!c || !status_host) return GFS_ERR_ARG;
  if (!c->b_built) return GFS_ERR_STATE;
  GFS_CK(cudaMemcpyAsync(status_host, c->b_status.p, 4, cudaMemcpyDeviceToHost, c->stream));
  GFS_CK(cudaMemsetAsync(c->b_status.p, 0, 4, c->stream));
  GFS_CK(cudaStreamSynchronize(c->stream));
  return GFS_OK;
}

int gfs_batch_query(gfs_ctx* c) {
  if (!c) return GFS_ERR_ARG;
  if (!c->b_built) return GFS_ERR_STATE;
  if (c->b_M == 0) return GFS_OK;
  cudaStream_t st = c->stream;
  const int ns = c->b_ns;
  GFS_CK(launch_batch_qkeys(c->b_desc.as<ShapeDesc>(), c->b_qoffd.as<int64_t>(), ns, c->b_M,
                            c->b_qkin.as<unsigned long long>(), c->b_qvin.as<int>(), st));
  int end_bit = 32;
  while ((int64_t(1) << (end_bit - 32)) < ns) ++end_bit;
  size_t bytes = c->cub_temp.bytes;
  GFS_CK(sort_pairs64(c->cub_temp.p, bytes, c->b_qkin.as<unsigned long long>(), c->b_qkout.as<unsigned long long>(),
                      c->b_qvin.as<int>(), c->b_qvout.as<int>(), c->b_M, end_bit, st));
  const int grid = c->b_grid_query ? c->b_grid_query : 152 * 4;
  // the work counters of this query (a memset node under capture)
  GFS_CK(cudaMemsetAsync(reinterpret_cast<char*>(c->b_cnt.p) + offsetof(Counters, q_sphere_ntests), 0,
                         5 * sizeof(unsigned long long), st));
  for (int phase = 1; phase <= 2; ++phase) {
    GFS_CK(cudaMemsetAsync(c->b_ctr.p, 0, 8, st));
    GFS_CK(launch_batch_query(c->b_qviews.as<QueryArgs>(), c->b_qw.as<int64_t>(), ns, c->b_qtotal,
                              c->b_ctr.as<unsigned long long>(), grid, phase, st));
  }
  return GFS_OK;
}

int gfs_batch_query_tangent(gfs_ctx* c) {
  if (!c) return GFS_ERR_ARG;
  if (!c->b_built) return GFS_ERR_STATE;
  GFS_TRY(batch_sync_host(c));
  for (const QueryArgs& a : c->b_qv)
    if (a.m > 0 && (!a.arg_out || !a.fl_out)) return GFS_ERR_ARG;
  // one launch per shape, each over its view (its points in the Morton order
  // the last gfs_batch_query computed)
  for (const QueryArgs& a : c->b_qv)
    if (a.m > 0) GFS_CK(launch_query_tangent(a, c->opt.box_cull, c->stream));
  return GFS_OK;
}

int gfs_batch_survivors(gfs_ctx* c, int shape, int64_t* g_out, int64_t cap, int64_t* count_host) {
  if (!c || !count_host || cap < 0) return GFS_ERR_ARG;
  if (!c->b_built) return GFS_ERR_STATE;
  if (shape < 0 || shape >= c->b_ns) return GFS_ERR_ARG;
  GFS_TRY(batch_sync_host(c));
  cudaStream_t st = c->stream;
  const int64_t n0 = c->b_soff[0][shape + 1] - c->b_soff[0][shape];
  const int64_t n1 = c->b_soff[1][shape + 1] - c->b_soff[1][shape];
  DevBuf ids, sorted, cnt;
  int stt = ensure(ids, size_t(n0 + n1) * 4 + 16);
  if (stt == GFS_OK) stt = ensure(sorted, size_t(n0 + n1) * 4 + 16);
  if (stt == GFS_OK) stt = ensure(cnt, 16);
  unsigned hc = 0;
  if (stt == GFS_OK) {
    if (cudaMemsetAsync(cnt.p, 0, 4, st) != cudaSuccess ||
        launch_collect_ids(c->b_ssorted[0].as<float4>() + c->b_soff[0][shape], unsigned(n0),
                           c->b_ssorted[1].as<float4>() + c->b_soff[1][shape], unsigned(n1),
                           c->b_sph64.as<D4>() + c->b_off[shape], c->KS, ids.as<uint32_t>(), cnt.as<unsigned>(),
                           st) != cudaSuccess ||
        cudaMemcpyAsync(&hc, cnt.p, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      stt = GFS_ERR_CUDA;
    }
  }
  if (stt == GFS_OK) {
    *count_host = hc;
    if (hc > 0 && g_out && cap >= int64_t(hc)) {
      size_t bytes = 0;
      if (sort_keys_u32(nullptr, bytes, ids.as<uint32_t>(), sorted.as<uint32_t>(), hc, st) != cudaSuccess ||
          cub_ensure(c, bytes) != GFS_OK) {
        stt = GFS_ERR_CUDA;
      } else {
        bytes = c->cub_temp.bytes;
        if (sort_keys_u32(c->cub_temp.p, bytes, ids.as<uint32_t>(), sorted.as<uint32_t>(), hc, st) != cudaSuccess ||
            launch_widen_ids(sorted.as<uint32_t>(), hc, g_out, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
          cudaGetLastError();
          stt = GFS_ERR_CUDA;
        }
      }
    } else if (cap < int64_t(hc)) {
      stt = GFS_ERR_ARG;
    }
  }
  release(ids);
  release(sorted);
  release(cnt);
  return stt;
}

int gfs_stats(gfs_ctx* c, gfs_stats_t* out) {
  if (!c || !out) return GFS_ERR_ARG;
  std::memset(out, 0, sizeof(*out));
  GFS_CK(cudaMemcpyAsync(&c->host_cnt, c->cnt.p, sizeof(Counters), cudaMemcpyDeviceToHost, c->stream));
  GFS_CK(cudaStreamSynchronize(c->stream));
  out->n_spheres = c->n;
  out->n_candidates = c->n * c->K;
  out->n_survivors_pos = c->nsurv[0];
  out->n_survivors_neg = c->nsurv[1];
  out->cull_fp64_rechecks = int64_t(c->host_cnt.cull_rechecks);
  out->query_fp64_rechecks = int64_t(c->host_cnt.query_rechecks);
  out->query_deferred = c->opt.precision == 0 ? int64_t(c->host_cnt.ndefer) : 0;
  out->tree_levels = c->st.nlevels;
  out->query_sphere_node_tests = int64_t(c->host_cnt.q_sphere_ntests);
  out->query_sphere_items = int64_t(c->host_cnt.q_sphere_items);
  out->query_surv_node_tests = int64_t(c->host_cnt.q_surv_ntests);
  out->query_band_passes = int64_t(c->host_cnt.q_band_passes);
  out->query_surv_items = int64_t(c->host_cnt.q_surv_items);
  out->cull_node_tests = int64_t(c->host_cnt.c_ntests);
  out->cull_items = int64_t(c->host_cnt.c_items);
  auto ms = [&](int a, int b) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, c->ev[a], c->ev[b]) != cudaSuccess) {
      cudaGetLastError();
      t = 0.f;
    }
    return double(t);
  };
  unsigned long long own = 0, sorts = 0;
  launch_counts(&own, &sorts);
  out->kernel_launches = int64_t(own + tangent_launch_count() + order_launch_count() + exact_launch_count() +
                                 insert_launch_count() + scored_launch_count());
  out->insert_rounds = c->ins_rounds;
  out->insert_steps = c->ins_steps;
  out->insert_rebuilds = c->ins_rebuilds;
  out->insert_ms_total = c->ins_ms_total;
  out->insert_ms_rebuild = c->ins_ms_rebuild;
  out->insert_ms_final = c->ins_ms_final;
  out->insert_ms_query = c->ins_ms_query;
  out->insert_slots = c->ins_queried;
  if (c->b_built) {
    Counters bc;
    GFS_CK(cudaMemcpyAsync(&bc, c->b_cnt.p, sizeof(Counters), cudaMemcpyDeviceToHost, c->stream));
    GFS_CK(cudaStreamSynchronize(c->stream));
    out->batch_sphere_items = int64_t(bc.q_sphere_items);
    out->batch_sphere_node_tests = int64_t(bc.q_sphere_ntests);
    out->batch_surv_items = int64_t(bc.q_surv_items);
    for (int k = 0; k < 3; ++k) out->batch_cull_tile[k] = c->b_cls_off[k + 1] > c->b_cls_off[k] ? c->b_tile[k] : 0;
    out->batch_query_grid = c->b_grid_query;
  }
  out->insert_sph_exact = int64_t(c->ins_work[0]);
  out->insert_sph_tested = int64_t(c->ins_work[1]);
  out->insert_surv_exact = int64_t(c->ins_work[2]);
  out->insert_surv_tested = int64_t(c->ins_work[3]);
  out->insert_ms_commit = c->ins_ms_commit;
  out->insert_ms_update = c->ins_ms_update;
  out->sort_calls = int64_t(sorts);
  if (c->have_ev && c->built_timed) {
    out->ms_build_total = ms(0, 3);
    out->ms_build_cull = ms(1, 2);
  }
  if (c->have_ev && c->query_timed) {
    out->ms_query_fast = ms(4, 5);
    out->ms_query_exact = ms(5, 6);
    out->ms_query_spheres = ms(4, 7);
  }
  out->n_survivors = -1;  // unique count is available through gfs_survivors
  return GFS_OK;
}

int gfs_solve_host(gfs_ctx* c, const double* p_host, const double* s_host, int64_t n, const void* x_host,
                   int x_is_fp32, int64_t m, float* s_out_host, int64_t* argmin_out_host,
                   uint16_t* flags_out_host) {
  if (!c || !p_host || !s_host || n < 1 || m < 0 || (m > 0 && !x_host)) return GFS_ERR_ARG;
  cudaStream_t st = c->stream;
  const size_t xrow = size_t(3) * (x_is_fp32 ? 4 : 8);
  const size_t xb = size_t(m) * xrow;
  GFS_TRY(ensure(c->h_p, size_t(n) * 24));
  GFS_TRY(ensure(c->h_s, size_t(n) * 8));
  GFS_TRY(ensure(c->h_x, xb));
  GFS_TRY(ensure(c->h_sout, size_t(m) * 4));
  GFS_TRY(ensure(c->h_arg, size_t(m) * 8));
  GFS_TRY(ensure(c->h_fl, size_t(m) * 2));
  GFS_TRY(ensure_side(c));
  // the query points go up on the side stream while the build runs
  GFS_CK(cudaEventRecord(c->sev, st));
  GFS_CK(cudaStreamWaitEvent(c->side, c->sev, 0));
  if (m > 0) GFS_CK(cudaMemcpyAsync(c->h_x.p, x_host, xb, cudaMemcpyHostToDevice, c->side));
  GFS_CK(cudaMemcpyAsync(c->h_p.p, p_host, size_t(n) * 24, cudaMemcpyHostToDevice, st));
  GFS_CK(cudaMemcpyAsync(c->h_s.p, s_host, size_t(n) * 8, cudaMemcpyHostToDevice, st));
  GFS_TRY(gfs_build(c, c->h_p.as<double>(), c->h_s.as<double>(), n));
  GFS_CK(cudaEventRecord(c->sev2, c->side));
  GFS_CK(cudaStreamWaitEvent(st, c->sev2, 0));
  GFS_TRY(gfs_query(c, c->h_x.p, x_is_fp32, m, s_out_host ? c->h_sout.as<float>() : nullptr, nullptr,
                    argmin_out_host ? c->h_arg.as<int64_t>() : nullptr,
                    flags_out_host ? c->h_fl.as<uint16_t>() : nullptr));
  if (m > 0 && s_out_host) GFS_CK(cudaMemcpyAsync(s_out_host, c->h_sout.p, size_t(m) * 4, cudaMemcpyDeviceToHost, st));
  if (m > 0 && argmin_out_host)
    GFS_CK(cudaMemcpyAsync(argmin_out_host, c->h_arg.p, size_t(m) * 8, cudaMemcpyDeviceToHost, st));
  if (m > 0 && flags_out_host)
    GFS_CK(cudaMemcpyAsync(flags_out_host, c->h_fl.p, size_t(m) * 2, cudaMemcpyDeviceToHost, st));
  GFS_CK(cudaStreamSynchronize(st));
  return GFS_OK;
}

void gfs_destroy(gfs_ctx* c) {
  if (!c) return;
  if (c->have_ev)
    for (cudaEvent_t e : c->ev)
      if (e) cudaEventDestroy(e);
  if (c->sev) cudaEventDestroy(c->sev);
  if (c->sev2) cudaEventDestroy(c->sev2);
  if (c->side) cudaStreamDestroy(c->side);
  DevBuf* bufs[] = {&c->U32, &c->U64, &c->sph64, &c->keys_in, &c->keys_out, &c->vals_in, &c->vals_out, &c->sph,
                    &c->thr, &c->sid, &c->bound_bits, &c->consts, &c->cnt, &c->cub_temp, &c->st_lo, &c->st_hi,
                    &c->st_na, &c->st_nb, &c->st_nf, &c->st_tight, &c->qstate, &c->surv_raw[0], &c->surv_raw[1], &c->surv_sorted[0], &c->surv_sorted[1],
                    &c->vt_lo[0], &c->vt_lo[1], &c->vt_hi[0], &c->vt_hi[1], &c->defer, &c->acc, &c->witness64,
                    &c->h_p, &c->h_s, &c->h_x, &c->h_sout, &c->h_arg, &c->h_fl,
                    &c->qk_in, &c->qk_out, &c->qv_in, &c->qv_out, &c->ins_counts,
                    &c->ins_tomb[0], &c->ins_tomb[1], &c->ins_dsurv[0], &c->ins_dsurv[1], &c->ins_dtomb[0],
                    &c->ins_dtomb[1], &c->ins_misc, &c->ins_maxrem, &c->ins_slot_t, &c->ins_slots, &c->ins_cbuf,
                    &c->ins_new, &c->ins_lost, &c->ins_inserted, &c->ins_codes, &c->ins_dyn, &c->ins_present,
                    &c->ins_scan, &c->ins_cmp, &c->ins_dynf4, &c->ins_near, &c->ins_nearcnt, &c->csr_ids,
                    &c->csr_off, &c->scored_status, &c->ud_uncov, &c->ud_cnt, &c->ud_pairs, &c->ud_circ,
                    &c->ud_quad, &c->ud_pts, &c->ud_k0, &c->ud_k1, &c->ud_v0, &c->ud_v1,
                    &c->b_desc, &c->b_offd, &c->b_qoffd, &c->b_sph64, &c->b_k64in, &c->b_k64out, &c->b_sph,
                    &c->b_thr, &c->b_sid, &c->b_bits, &c->b_bcs, &c->b_lo, &c->b_hi, &c->b_na, &c->b_nb, &c->b_nf,
                    &c->b_stdev, &c->b_prefix, &c->b_ctr, &c->b_cnt, &c->b_cviews, &c->b_cw, &c->b_sraw[0],
                    &c->b_sraw[1], &c->b_sshape[0], &c->b_sshape[1], &c->b_ssorted[0], &c->b_ssorted[1],
                    &c->b_vlo[0], &c->b_vlo[1], &c->b_vhi[0], &c->b_vhi[1], &c->b_vtdev[0], &c->b_vtdev[1],
                    &c->b_hist, &c->b_qkin, &c->b_qkout, &c->b_qvin, &c->b_qvout, &c->b_qviews, &c->b_qw, &c->b_qstate,
                    &c->b_status, &c->b_vprefix[0], &c->b_vprefix[1], &c->b_sodev[0], &c->b_sodev[1]};
  for (DevBuf* b : bufs) release(*b);
  delete c;
}

// ---------------------------------------------------------------------------
// backward without device allocation
// ---------------------------------------------------------------------------
// Callers inside CUDA graph capture, or runtimes that forbid allocation after
// start-up, cannot let the library grow buffers.  This entry point keeps the
// backward pass's per-sample fixed-point accumulators in one static device
// array instead (held by every GPU that loads the library until exit).
}  // extern "C"

namespace {

__device__ __align__(256) long long g_noalloc_acc[4 * GFS_NOALLOC_MAX_SPHERES];

constexpr int kMaxDevices = 64;
long long* g_noalloc_ptr[kMaxDevices] = {};
std::mutex g_noalloc_mu;

// device address of the static array on the current device (looked up once
// per device; the host-side symbol is only a stand-in, never a device pointer)
int noalloc_scratch(long long** out) {
  int dev = 0;
  GFS_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return GFS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    GFS_CK(cudaGetSymbolAddress(&p, g_noalloc_acc));
    g_noalloc_ptr[dev] = static_cast<long long*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return GFS_OK;
}

}  // namespace

extern "C" int gfs_query_backward_noalloc(gfs_ctx* c, const void* x, int x_is_fp32, int64_t m, const float* s,
                                          const int64_t* argmin, const uint16_t* flags, const float* grad_s,
                                          float* grad_x, float* grad_p, float* grad_sv) {
  if (!c || m < 0 || (m > 0 && (!x || !s || !argmin || !flags || !grad_s))) return GFS_ERR_ARG;
  if (!c->built) return GFS_ERR_STATE;
  const int64_t n = c->n;
  if (n > GFS_NOALLOC_MAX_SPHERES) return GFS_ERR_TOO_LARGE;
  long long* acc = nullptr;
  GFS_TRY(noalloc_scratch(&acc));
  // the array keeps the previous call's sums: clear the part used here
  GFS_CK(cudaMemsetAsync(acc, 0, size_t(4 * n) * sizeof(long long), c->stream));
  GradArgs a;
  std::memset(&a, 0, sizeof(a));
  if (x_is_fp32) a.x32 = static_cast<const float*>(x);
  else a.x64 = static_cast<const double*>(x);
  a.m = m;
  a.s = s;
  a.arg = argmin;
  a.flags = flags;
  a.grad_s = grad_s;
  a.grad_x = grad_x;
  a.sph64 = c->sph64.as<D4>();
  a.U64 = c->U64.as<double>();
  a.witness64 = c->witness64.as<double>();
  a.K = c->K;
  a.KS = c->KS;
  a.acc_p = acc;
  a.acc_s = acc + 3 * n;
  GFS_CK(launch_grad(a, n, nullptr, nullptr, c->stream));
  GFS_CK(launch_tangent_grad(a, n, grad_p, grad_sv, c->stream));
  return GFS_OK;
}
