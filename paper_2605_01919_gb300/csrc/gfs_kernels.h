// Argument blocks and launch helpers of the device kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gfs.h"
#include "gfs_internal.cuh"

namespace gfs {

// one shape of a batched call (device pointers; outputs nullable)
struct ShapeDesc {
  const double* p;
  const double* s;
  int64_t n;
  const void* x;
  int x_is_fp32;
  int64_t m;
  float* s_out;
  double* s64_out;
  int64_t* argmin_out;
  uint16_t* flags_out;
};

struct CullArgs {
  const float4* sph;     // sorted spheres (x, y, z, s) FP32
  const float4* thr;     // sorted coverage thresholds (lo/hi for candidates, lo/hi for queries)
  const int* sid;        // sorted slot -> input index
  const D4* sph64;       // FP64 spheres in input order
  const float* U32;      // K x 3 directions, FP32
  const double* U64;     // K x 3 directions, FP64
  int K, KS;             // K directions; KS = K + 1 ids per sphere
  Tree tree;             // sphere hierarchy
  float tol32;
  double tol;
  int box_cull;
  const BuildConsts* bc;
  int64_t n;
  float4* surv[2];       // survivors per sign class (x, y, z, id bits)
  unsigned int cap;      // capacity of each survivor list
  Counters* cnt;
  uint16_t* surv_shape[2];  // batched builds: shape index of each survivor (else null)
  int shape;
};

struct QueryArgs {
  const float4* sph;
  const float4* thr;
  const int* sid;
  const D4* sph64;
  Tree st;
  int64_t n;
  const float4* surv[2];
  Tree vt[2];
  const double* U64;
  const double* witness64;  // FP64 witness point per sphere (inserted spheres only)
  int K, KS;
  float tol32;
  double tol;
  int clamp_opp;
  const BuildConsts* bc;
  const double* x64;
  const float* x32;
  int64_t m;
  const uint32_t* perm;     // processing order of the query points (Morton), or null
  float* s_out;
  double* s64_out;
  int64_t* arg_out;
  uint16_t* fl_out;
  uint32_t* defer;
  unsigned int defer_cap;
  Counters* cnt;
  uint4* state;             // 3 x uint4 per processing slot, between the query's two kernels
};

// One pending step of the insertion window: its value against the state at
// the start of the round, and what the commit test needs.
struct InsSlot {
  double value;          // FP64 value
  double wx, wy, wz;     // witness: the point that set the value
  double R;              // upper bound of the step's value in any later state (< 0: never inserts)
  double rho;            // radius within which the state decides this result (inf: any change may)
  long long arg;         // argmin (provisional sphere numbering)
  int t;                 // step index
  unsigned short flags;  // result word without LOST_WITNESS
  unsigned char insert;  // 1: the result joins the samples
  unsigned char pad;
};

// Device-side counters of the insertion rounds (read back once per round).
struct InsMisc {
  int npend;                 // valid window slots
  int next;                  // next step not yet in the window
  int ncommit;               // steps committed by the last round
  int nnew;                  // spheres inserted by the last round
  int ndyn;                  // spheres inserted since the last rebuild (the dynamic list)
  int ndyn_start;            // ndyn before the last round's commits (its new spheres follow)
  unsigned nlost;            // spheres that lost their last survivor in the last round
  unsigned err;              // bit 0: walk stack overflow, bit 1: dynamic list overflow
  int ninserted;             // spheres inserted by this call so far
  // step-query work over the call: spheres evaluated exactly in FP64, spheres
  // screened in FP32, survivors evaluated exactly, survivors screened
  unsigned long long work[4];
};

struct InsertArgs {
  // spheres in the hierarchy (sid: provisional index), plus the ones inserted
  // since the last rebuild (dyn_ids); step t's sphere has provisional index
  // n0 + t until the call renumbers the inserted spheres consecutively
  const float4* sph;
  const int* sid;
  Tree st;
  int n0;
  const int* dyn_ids;
  float4* dyn_f4;       // FP32 (x, y, z, value) of the dynamic list's spheres (sign class kept)
  int* near_list;       // per new sphere of a round: dynamic-list spheres that reach it
  int* near_cnt;
  D4* sph64;            // by provisional index
  double* witness64;    // witness point per sphere (inserted spheres)
  int* counts;          // live survivors per sphere
  int* maxrem;          // largest step that removed one of the sphere's survivors
  // survivors: hierarchies with tombstone bits, plus the candidates and
  // witnesses of the spheres inserted since the rebuild: KS slots per
  // dynamic-list sphere (slot d * KS + k), a tombstone word each (1: culled
  // at insertion or covered since)
  const float4* surv[2];
  Tree vt[2];
  uint32_t* tomb[2];
  float4* dsurv[2];
  uint32_t* dtomb[2];
  const double* U64;
  int K, KS;
  double tol;
  int box_cull, clamp_opp;
  const BuildConsts* bc;
  const double* y;
  const double* known;  // nullable: per-point known value (its sign fixes the class)
  int64_t T;
  double* s_out;
  int64_t* arg_out;
  uint16_t* fl_out;
  // the window of pending steps
  int* slot_t;           // step of each slot, in step order
  InsSlot* slots;
  unsigned char* cbuf;   // commit decisions, 2 x window capacity (passes alternate halves)
  int wcap;              // window capacity
  int* new_ids;          // provisional indices of the spheres inserted by the round
  int* lost_list;        // spheres that lost their last survivor in the round
  int* inserted;            // per step: 1 when it joined the samples
  unsigned char* codes;     // per step: result code (for the final renumbering of the argmins)
  int* dyn_ids_w;        // writable view of dyn_ids
  InsMisc* misc;
};

// one round of the insertion: speculative queries of the window's nslots
// steps, then the commit passes and the commit itself (window compaction and
// refill up to wnext slots); the host reads InsMisc afterwards
cudaError_t launch_ins_query(const InsertArgs& a, int nslots, cudaStream_t st);
cudaError_t launch_ins_commit(const InsertArgs& a, int nslots, int passes, int wnext, cudaStream_t st);
// state update of the spheres the last round inserted (nnew of them)
// (ndyn_start: spheres of the dynamic list before the round's commits)
cudaError_t launch_ins_update(const InsertArgs& a, int nnew, int ndyn_start, cudaStream_t st);
cudaError_t launch_ins_counts(const float4* s0, unsigned n0, const float4* s1, unsigned n1, const D4* sph64, int KS,
                              int* counts, cudaStream_t st);
cudaError_t launch_ins_compact(const float4* ssurv, const uint32_t* tomb, unsigned ns, const float4* dsurv,
                               const uint32_t* dtomb, unsigned nd, float4* out, unsigned* count, cudaStream_t st);
// renumbering after the call: newid[n0 + t] = n0 + (inserted steps before t)
cudaError_t launch_ins_renumber(const InsertArgs& a, const int* newid, D4* sph_out, double* wit_out,
                                cudaStream_t st);
cudaError_t launch_ins_remap_survivors(float4* items, unsigned n, const int* newid, int n0, int KS, cudaStream_t st);
cudaError_t exclusive_scan_i32(void* temp, size_t& bytes, const int* in, int* out, int64_t n,
                              cudaStream_t st);
cudaError_t launch_gather_d4(const D4* src, const int* ids, int64_t n, D4* dst, cudaStream_t st);
cudaError_t launch_remap_sid(int* sid, const int* ids, int64_t n, cudaStream_t st);
// kernels the insertion file has launched in this process
unsigned long long insert_launch_count();

struct GradArgs {
  const double* x64;
  const float* x32;
  int64_t m;
  const float* s;
  const int64_t* arg;
  const uint16_t* flags;
  const float* grad_s;
  float* grad_x;
  const D4* sph64;
  const double* U64;
  const double* witness64;
  int K, KS;
  long long* acc_p;  // 3n fixed-point accumulators
  long long* acc_s;  // n fixed-point accumulators
};

cudaError_t launch_copy_inputs(const double* p, const double* s, int64_t n, D4* sph64, cudaStream_t st);
cudaError_t launch_keys_d4(const D4* sph64, int64_t n, uint32_t* keys, int* vals, unsigned int* bound_bits,
                           BuildConsts* bc, cudaStream_t st);
cudaError_t sort_pairs(void* temp, size_t& temp_bytes, const uint32_t* kin, uint32_t* kout, const int* vin,
                       int* vout, int64_t n, cudaStream_t st);
cudaError_t sort_keys_u32(void* temp, size_t& temp_bytes, const uint32_t* kin, uint32_t* kout, int64_t n,
                          cudaStream_t st);
cudaError_t launch_gather_spheres(const D4* sph64, const int* order, int64_t n, const BuildConsts* bc, float tol32,
                                  double tol, float4* sph, float4* thr, int* sid, cudaStream_t st);
// scratch (spheres only, may be null): 3 * (nodes above the leaves) unsigned
// words for tightening the internal bounding balls; null skips it
cudaError_t launch_build_tree(const float4* items, int is_sphere, float A, Tree& T, unsigned* scratch,
                              cudaStream_t st);
cudaError_t launch_query_keys(const double* x64, const float* x32, int64_t m, uint32_t* keys, int* vals,
                              cudaStream_t st);
cudaError_t launch_point_keys(const float4* items, int64_t n, uint32_t* keys, int* vals, cudaStream_t st);
cudaError_t launch_gather_points(const float4* src, const int* order, int64_t n, float4* dst, cudaStream_t st);
cudaError_t launch_cull(const CullArgs& a, cudaStream_t st);
// the query in two kernels: phase 1 (sphere pass, state to a.state), phase 2
// (survivor pass, exact re-evaluation, flags, outputs)
cudaError_t launch_query_spheres(const QueryArgs& a, cudaStream_t st);
cudaError_t launch_query_finish(const QueryArgs& a, cudaStream_t st);
cudaError_t launch_query_exact(const QueryArgs& a, int all, cudaStream_t st);
cudaError_t launch_grad(const GradArgs& a, int64_t n, float* grad_p, float* grad_sv, cudaStream_t st);
cudaError_t launch_collect_ids(const float4* s0, unsigned int n0, const float4* s1, unsigned int n1, const D4* sph64,
                               int KS, uint32_t* out, unsigned int* count, cudaStream_t st);
void launch_counts(unsigned long long* own, unsigned long long* sorts);
cudaError_t launch_widen_ids(const uint32_t* in, int64_t n, int64_t* out, cudaStream_t st);

cudaError_t launch_batch_copy(const ShapeDesc* d, const int64_t* off, int ns, int64_t N, D4* sph64,
                              unsigned long long* keys, int* vals, unsigned int* bits, BuildConsts* bc,
                              cudaStream_t st);
cudaError_t sort_pairs64(void* temp, size_t& bytes, const unsigned long long* kin, unsigned long long* kout,
                         const int* vin, int* vout, int64_t n, int end_bit, cudaStream_t st);
cudaError_t launch_batch_gather(const D4* sph64, const int* order, const int64_t* off, int ns, int64_t N,
                                const BuildConsts* bc, float tol32, double tol, float4* sph, float4* thr, int* sid,
                                cudaStream_t st);
cudaError_t launch_batch_tree_level(const Tree* trees, const int64_t* prefix, int64_t total, int ns, int level,
                                    const float4* items_base, const int64_t* item_off, const BuildConsts* bc,
                                    int is_sphere, cudaStream_t st);
cudaError_t launch_batch_hist(const uint16_t* shape, unsigned n, unsigned* counts, cudaStream_t st);
cudaError_t launch_batch_surv_keys(const float4* items, const uint16_t* shape, unsigned n, unsigned long long* keys,
                                   int* vals, cudaStream_t st);
cudaError_t launch_batch_gather_points(const float4* src, const int* order, unsigned n, float4* dst, cudaStream_t st);
cudaError_t launch_batch_qkeys(const ShapeDesc* d, const int64_t* off, int ns, int64_t M, unsigned long long* keys,
                               int* vals, cudaStream_t st);
// phase 1: the sphere pass of every (shape, 32 points) item, phase 2: the rest
// (reset ctr between the two launches)
// cull over a group of shapes, one block per (shape, k, tile spheres) item
// (tile 64, 128 or 256): bprefix holds each shape's first item, nblocks the
// total
cudaError_t launch_batch_cull_blocks(const CullArgs* views, const int64_t* bprefix, int ns, int64_t nblocks, int tile,
                                     cudaStream_t st);
cudaError_t launch_batch_query(const QueryArgs* views, const int64_t* wprefix, int ns, int64_t limit,
                               unsigned long long* ctr, int grid, int phase, cudaStream_t st);
// the survivor forest of one class laid out and built on the device from the
// cull's counts (capacity cap survivor slots, node_cap nodes, nlev levels;
// the query views' survivor pointers and trees are patched; overflow sets a
// status bit); no host synchronisation
cudaError_t launch_batch_surv_forest(const uint16_t* shape, const float4* raw, const Counters* cnt, int cls,
                                     unsigned cap, int ns, unsigned* hist, unsigned long long* kin,
                                     unsigned long long* kout, int* vin, int* vout, void* sort_temp,
                                     size_t sort_bytes, int end_bit, float4* sorted, int64_t node_cap, float4* lo,
                                     float4* hi, Tree* trees, int64_t* prefix, int nlev, int64_t* soff,
                                     QueryArgs* views, unsigned* status, cudaStream_t st);

}  // namespace gfs
