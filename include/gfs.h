/*
 * gfs.h -- C ABI of the GB300 consistent signed-distance library.
 *
 * The library evaluates the data-parallel hot path of "Greed for the
 * Spheres" (consistent signed distance interpolation):
 *
 *  P build  -- every sample (p_i, s_i) is a sphere of radius |s_i| and sign
 *              sign(s_i) (Sec. 3.1).  Candidate surface points are placed on
 *              every sphere at the vertices of a geodesic icosphere of depth
 *              tau, q_ik = p_i + |s_i| u_k, and a candidate survives when it
 *              lies in the domain box [-1,1]^3 (App. B) and no other ball,
 *              shrunk by tol, contains it (the "uncovered points" of
 *              Prop. 1 (ii); the discrete stand-in for the grow-to points
 *              T, U, D of Def. 1).
 *  query    -- at a new point x: the sign from the balls containing x
 *              (Sec. 4.3), the distance to the nearest surviving candidate
 *              of that sign, clamped by the nearest tangent point of an
 *              opposite-sign sphere (Def. 1 T; Sec. 4.3 upper bound), and
 *              the Sec. 4.3 bound checks as flags.  This is the discrete
 *              counterpart of the minimum valid radius of Prop. 2 / Sec. 6.
 *  backward -- d s*(x) / d(x, p_i, s_i) through the argmin.
 *  insert   -- the greedy sequential refinement loop (Sec. 4): each new
 *              value is computed against the inputs and all values inserted
 *              before it, then joins the sample set.
 * and, beyond that path: the same-sign tangent points of Def. 1 as extra
 * query candidates (gfs_query_tangent), the point q* behind each value
 * (gfs_query_points), the exact coverage of each sphere (Prop. 1 (ii),
 * gfs_sphere_uncovered) and the flood-fill refinement order of Sec. 4.2
 * (gfs_cell_coverage, gfs_flood_order).
 *
 * Conventions shared by every call:
 *  - Positions are FP64 (x, y, z) triples stored row-major (n x 3); values
 *    are FP64.  Query points may be FP64 or FP32 triples.
 *  - Every buffer argument is a DEVICE pointer unless the name ends in
 *    `_host`; the caller owns all input and output buffers.  The library
 *    owns the sphere/survivor hierarchies and scratch inside the context.
 *  - All work is enqueued on the context's CUDA stream (cudaStream_t passed
 *    as void*; NULL = legacy default stream).  A call returns once the work
 *    is enqueued, except where noted (gfs_build reads back one counter).
 *  - Return value: GFS_OK (0) or a GFS_ERR_* code; gfs_strerror() names it.
 *    Per-query anomalies are flags, not errors.  There is no CPU fallback:
 *    without a CUDA device every compute call fails with GFS_ERR_CUDA.
 *  - Candidate ids: g = i * (K + 1) + k, K = 10 * 4^tau + 2, i the sphere's
 *    index in input order (inserted spheres continue the numbering), k < K an
 *    icosphere vertex; slot k = K holds an inserted sphere's witness point.
 */
#ifndef GFS_H
#define GFS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define GFS_OK 0
#define GFS_ERR_ARG 1        /* invalid argument (null, negative size, bad option) */
#define GFS_ERR_OOM 2        /* device allocation failed */
#define GFS_ERR_CUDA 3       /* CUDA runtime error (no device, launch failure) */
#define GFS_ERR_STATE 4      /* call order violated (e.g. query before build) */
#define GFS_ERR_TIMEOUT 5    /* a capped device loop ran out of iterations */
#define GFS_ERR_TOO_LARGE 6  /* sizes exceed the library's index ranges */

/* ---- per-query result word (uint16) ------------------------------------ */
/* low 4 bits: result code */
#define GFS_CODE_SURVIVOR 0  /* value = distance to nearest surviving candidate; argmin = g */
#define GFS_CODE_OPPOSITE 1  /* value = distance to nearest opposite tangent point; argmin = sphere */
#define GFS_CODE_SAMPLE 2    /* x equals an input position; value = its sample; argmin = sphere */
#define GFS_CODE_OUTSIDE 3   /* x lies in no (shrunk) ball: value 0; argmin = -1 */
#define GFS_CODE_INVALID 4   /* x lies in balls of both signs: value NaN; argmin = -1 */
#define GFS_CODE_LOWER 5     /* no candidate at all: value = lower bound; argmin = sphere */
#define GFS_CODE_TANGENT 6   /* gfs_query_tangent: value = distance to an uncovered same-sign tangent point;
                                argmin = 2 * sphere + side (0 near, 1 far) */
/* violation bits (Sec. 4.3 bound checks) */
#define GFS_FLAG_LB_VIOL 0x10     /* |s| < LB - tol  (LB: nearest-tangent bound of the containing spheres) */
#define GFS_FLAG_FAR_VIOL 0x20    /* |s| > FAR + tol (FAR: nearest far tangent point of any sphere) */
#define GFS_FLAG_OPP_VIOL 0x40    /* |s| > UB_opp + tol (only possible with clamp_opp = 0) */
#define GFS_FLAG_LOST_WITNESS 0x80 /* insertion: some sphere lost its last surviving candidate */
#define GFS_FLAG_NONCONSERVATIVE 0x100 /* insertion with known values: |value| < |known| - tol */
#define GFS_FLAG_SCORE_FALLBACK 0x200 /* gfs_query_scored: no valid candidate, the minimum value kept */

/* ---- options ------------------------------------------------------------ */
typedef struct {
  int tau;          /* icosphere subdivision depth, 0..6 (K = 10*4^tau + 2 candidates per sphere) */
  double tol;       /* coverage tolerance: q is covered by j iff |q-p_j| < |s_j| - tol (App. B: 1e-6) */
  int box_cull;     /* 1: drop candidates outside [-1,1]^3 (App. B) */
  int clamp_opp;    /* 1: clamp by the nearest opposite-sign tangent point (Sec. 4.3 upper bound) */
  int precision;    /* 0: FP32 bulk arithmetic, predicates near a boundary re-decided in FP64;
                       1: FP64 throughout (same results, slower) */
  int timing;       /* 1: record CUDA events around each phase (read back by gfs_stats) */
  int reserved[6];  /* must be zero */
} gfs_options;

/* Fill *opt with the defaults: tau 3, tol 1e-6, box_cull 1, clamp_opp 1, precision 0. */
void gfs_default_options(gfs_options* opt);

typedef struct gfs_ctx gfs_ctx; /* opaque, library-owned */

/* Create a context bound to the current CUDA device and the given stream.
 * Errors: GFS_ERR_ARG (bad options), GFS_ERR_CUDA (no device), GFS_ERR_OOM. */
int gfs_create(gfs_ctx** out, const gfs_options* opt, void* cuda_stream);

/* Change the stream later calls are enqueued on. */
int gfs_set_stream(gfs_ctx* ctx, void* cuda_stream);

/* P build (Def. 1 discretised; Prop. 1 (ii) uncovered points).
 * p_xyz: device, n*3 FP64, row-major sample positions.
 * s:     device, n FP64 signed distance samples.
 * Builds the sphere hierarchy, culls all n*K candidates and builds the
 * survivor hierarchies.  Inputs are copied; the caller may free them after
 * the call returns.  Synchronises the stream twice (the coordinate bound
 * that sets the hierarchy's rounding slack, and the survivor count).
 * Errors: GFS_ERR_ARG (n < 1, null), GFS_ERR_TOO_LARGE (n*(K+1) >= 2^32, or
 * more than 2^30 survivors of one sign class), GFS_ERR_OOM, GFS_ERR_CUDA. */
int gfs_build(gfs_ctx* ctx, const double* p_xyz, const double* s, int64_t n);

/* Consistent value at m query points (Prop. 2 / Sec. 6 minimum radius,
 * discretised; Sec. 4.3 sign inference, bounds and checks).
 * x:         device, m*3 FP64 (x_is_fp32 = 0) or FP32 (x_is_fp32 = 1) points.
 * s_out:     device, m FP32 values (nullable).
 * s64_out:   device, m FP64 values (nullable).
 * argmin_out:device, m int64 (nullable): candidate id or sphere index, per code.
 * flags_out: device, m uint16 result words (nullable).
 * Runs as two kernels (the pass over the spheres, then the pass over the
 * survivors and the exact re-evaluations) plus, for points outside the FP32
 * error model's coordinate range, the FP64 kernel.  Grows library-owned
 * scratch when m grows (Morton keys and order, 48 B of state per point).
 * No host synchronisation.
 * Errors: GFS_ERR_STATE (no build), GFS_ERR_ARG, GFS_ERR_TOO_LARGE
 * (m >= 2^32), GFS_ERR_OOM, GFS_ERR_CUDA. */
int gfs_query(gfs_ctx* ctx, const void* x, int x_is_fp32, int64_t m, float* s_out, double* s64_out,
              int64_t* argmin_out, uint16_t* flags_out);

/* Same-sign tangent augmentation of a gfs_query result (Def. 1: the grow-to
 * points T include the tangent points of the spheres in the direction of x;
 * Sec. 6 min_valid_radius takes them as candidates).  For every point whose
 * code is SURVIVOR, OPPOSITE or LOWER, the candidate set is extended by the
 * near and far tangent points t = p_j +- |s_j| (x - p_j)/|x - p_j| of every
 * sphere j of x's sign class (none when x = p_j), kept when no other ball,
 * shrunk by tol, contains t and (box_cull) t lies in [-1,1]^3.  The nearest
 * candidate (squared distances; a survivor wins a tie, then the lowest
 * 2j + side) sets the value, clamped by UB_opp as in gfs_query, with the same
 * bound checks; a tangent winner gets code GFS_CODE_TANGENT and argmin
 * 2j + side (side 0 near, 1 far).  Other points are left unchanged.
 * Decisions are taken in FP64 (one thread per point; slower than gfs_query).
 * x, m:       the points of the preceding gfs_query on this context.
 * argmin_out, flags_out: that call's outputs (device, required): read, then
 *             rewritten in place where a tangent point wins.
 * s_out, s64_out: its value outputs (device, nullable), rewritten likewise.
 * gfs_query_backward differentiates TANGENT results as distances to the
 * moving tangent point (d|x - t|/dx = +-(x - p_j)/|x - p_j|).
 * Points are processed in Morton order (library-owned key and order
 * buffers grow when m grows, as in gfs_query).  No host synchronisation.
 * Errors: GFS_ERR_STATE (no build), GFS_ERR_ARG, GFS_ERR_TOO_LARGE
 * (m >= 2^32), GFS_ERR_OOM, GFS_ERR_CUDA. */
int gfs_query_tangent(gfs_ctx* ctx, const void* x, int x_is_fp32, int64_t m, float* s_out, double* s64_out,
                      int64_t* argmin_out, uint16_t* flags_out);

/* Scored value of a gfs_query result (Sec. 3.3: score_for_radius,
 * interpolate_sdf_to): instead of the minimum valid radius, the best-scoring
 * valid one over the grow-to points -- the survivors (standing in for the
 * intersection points U, D of Def. 1) and the near and far tangent points of
 * every sphere that no other shrunk ball covers (with box_cull, inside the
 * box), each with the sphere i it lies on, for both signs of r = |x - q|.
 * Order: type class (tangency point whose normals agree > intersection point
 * that agrees > intersection point that disagrees > tangency point that
 * disagrees; the normals sign * (x - q) and sign(s_i) * (p_i - q) agree when
 * their dot product is positive), then sign score * r (1 for positive, 2 for
 * negative values), then the lower candidate key (survivor id; tangent
 * points after every survivor), then the negative sign.  Valid: no ball of
 * the opposite sign intersected (not UB < r - tol), no sphere other than i
 * loses all its survivors to the new ball shrunk by tol, no sphere strictly
 * inside it (not r > FAR + tol).  Result codes: SURVIVOR (argmin g) or
 * TANGENT (argmin 2j + side), value sign * r, LB_VIOL as in gfs_query.  SAMPLE
 * and INVALID results are kept; where no candidate is valid the query's
 * result is kept with GFS_FLAG_SCORE_FALLBACK.
 * x, m: the points of the preceding gfs_query on this context (with
 * clamp_opp = 1 that result is the minimum valid value the paper falls back
 * to).  argmin_out, flags_out: that call's outputs (device, required), read
 * and rewritten; s_out, s64_out: its values (device, nullable), rewritten.
 * The first call after a build or an insertion sorts the survivor ids into
 * per-sphere lists (library-owned, synchronises the stream); one thread per
 * point in Morton order, decisions in FP64.
 * Errors: GFS_ERR_STATE (no build), GFS_ERR_ARG, GFS_ERR_TOO_LARGE
 * (m >= 2^32), GFS_ERR_OOM, GFS_ERR_CUDA. */
int gfs_query_scored(gfs_ctx* ctx, const void* x, int x_is_fp32, int64_t m, float* s_out, double* s64_out,
                     int64_t* argmin_out, uint16_t* flags_out);

/* The point q* that sets each value of a gfs_query / gfs_query_tangent
 * result (Prop. 2: the nearest valid grow-to point), from its argmin and
 * result word: SURVIVOR: the candidate p_i + |s_i| u_k (or an inserted
 * sphere's witness); OPPOSITE and LOWER j: the point of sphere j nearest to
 * x, p_j + |s_j| (x - p_j)/|x - p_j|; TANGENT 2j + side: that tangent point
 * (side 1: p_j - ...); OUTSIDE, and OPPOSITE / LOWER with argmin -1: x
 * itself (value 0); SAMPLE and INVALID: NaN (no point sets the value), and
 * NaN where x = p_j.  FP64, the expressions of the candidates and tangent
 * points, so |x - q*| reproduces the value.
 * x, m: the query points; argmin, flags: that query's outputs (device).
 * qstar_out: device, m*3 FP64.  No host synchronisation, no allocation.
 * Errors: GFS_ERR_STATE (no build), GFS_ERR_ARG, GFS_ERR_CUDA. */
int gfs_query_points(gfs_ctx* ctx, const void* x, int x_is_fp32, int64_t m, const int64_t* argmin,
                     const uint16_t* flags, double* qstar_out);

/* Adjoint of gfs_query through the argmin (the paper has no gradients; the
 * value is piecewise a distance to a point or a sphere, differentiated here).
 * argmin/flags/s: the forward outputs for the same x (device).
 * grad_s: device, m FP32 upstream gradient.
 * grad_x: device, m*3 FP32 output (nullable), overwritten.
 * grad_p: device, n*3 FP32 output (nullable), overwritten.
 * grad_sv:device, n FP32 output (nullable), overwritten.
 * Per-sample sums are accumulated in 64-bit fixed point, so the result does
 * not depend on scheduling order.  Errors: GFS_ERR_STATE, GFS_ERR_ARG. */
int gfs_query_backward(gfs_ctx* ctx, const void* x, int x_is_fp32, int64_t m, const float* s,
                       const int64_t* argmin, const uint16_t* flags, const float* grad_s, float* grad_x,
                       float* grad_p, float* grad_sv);

/* Greedy sequential insertion (Sec. 4 refinement loop; Sec. 6 repair
 * inserts the removed samples the same way).  For t = 0..T-1 in order: the
 * consistent value at y_t is computed against the current samples (inputs
 * and every earlier insertion) and survivors, exactly as gfs_query defines it
 * (FP64 decisions); unless the code is SAMPLE, OUTSIDE or INVALID, (y_t,
 * value) then joins the samples as sphere n+j (j = number inserted so far):
 * survivors inside its shrunk ball are dropped, its K candidates and its
 * witness (the point that set the value, candidate slot K) are culled against
 * every other sphere and join the survivors.  LOST_WITNESS is set on step t
 * when some sphere loses its last survivor.
 * y:          device, T*3 FP64 points, processed in order.
 * s_out:      device, T FP64 values (nullable).
 * argmin_out: device, T int64 (nullable); flags_out: device, T uint16 (nullable).
 * The context's state is updated: later gfs_query / gfs_survivors calls see
 * the inserted samples (numbered n, n+1, ... in step order).
 * Execution: deterministic parallel rounds with the sequential results.  A
 * round evaluates a window of the first pending steps against the state at
 * its start (one block per step) and commits every step that no earlier
 * pending step can influence or be influenced by: the ball of an earlier
 * step t, whose radius in any later state is at most its nearest opposite
 * tangent distance R_t (or exactly its value when t commits in the same
 * round), must stay more than a margin away from the region that decides the
 * later step's result (its value around its point).  The first pending step
 * always commits.  The window grows while most of it commits and shrinks when
 * little does; far-apart points commit many steps per round, points within
 * each other's reach one.  Synchronises the stream once per round.
 * Errors: GFS_ERR_STATE (no build), GFS_ERR_ARG,
 * GFS_ERR_TOO_LARGE ((n+T+1)*(K+1) >= 2^32), GFS_ERR_OOM, GFS_ERR_CUDA,
 * GFS_ERR_TIMEOUT (more rounds than steps: cannot happen unless the device
 * state is corrupted). */
/* As gfs_insert, with a known value per point (Sec. 6 repair: the removed
 * samples are re-inserted knowing their own sample values).
 * known: device, T FP64 values (nullable: then this is gfs_insert).  The sign
 * of known[t] fixes y_t's sign class instead of containment (0 or NaN: the
 * class is inferred as in gfs_query), so a known step is never OUTSIDE or
 * INVALID; LOWER with no sphere of that class has value 0, argmin -1.
 * GFS_FLAG_NONCONSERVATIVE marks an inserted step whose |value| is below
 * |known[t]| - tol.  Errors: as gfs_insert. */
int gfs_insert_known(gfs_ctx* ctx, const double* y, const double* known, int64_t T, double* s_out,
                     int64_t* argmin_out, uint16_t* flags_out);

int gfs_insert(gfs_ctx* ctx, const double* y, int64_t T, double* s_out, int64_t* argmin_out,
               uint16_t* flags_out);

/* Same computation and outputs as gfs_query_backward, for callers that must
 * not allocate device memory: code running while a CUDA graph is captured
 * (allocation is not allowed during capture), and runtimes that reserve all
 * device memory at start-up and forbid later allocation.  gfs_query_backward
 * grows a context-owned accumulator buffer on demand; this variant instead
 * uses one library-wide array in static device memory of
 * 4 * GFS_NOALLOC_MAX_SPHERES 64-bit words (8 MiB), which every GPU that
 * loads the library holds until the process exits.  The paper has no
 * counterpart of this call.
 *  - Limit: the context's sphere count n must be <= GFS_NOALLOC_MAX_SPHERES,
 *    else GFS_ERR_TOO_LARGE (nothing is launched).
 *  - The array is shared by every call on a device and keeps the last call's
 *    contents; each call clears the part it uses first.  Calls whose work
 *    overlaps on the GPU (different streams, or different contexts on the
 *    same device) race on it and must be ordered by the caller.
 *  - The first call on a device looks up the array's device address (no
 *    allocation); make that first call before any stream capture.  The
 *    address is kept for the life of the process: it stays valid while the
 *    device's primary context lives (after cudaDeviceReset the library must
 *    not be used without reloading it).
 * Arguments and other errors: as gfs_query_backward. */
#define GFS_NOALLOC_MAX_SPHERES 262144
int gfs_query_backward_noalloc(gfs_ctx* ctx, const void* x, int x_is_fp32, int64_t m, const float* s,
                               const int64_t* argmin, const uint16_t* flags, const float* grad_s, float* grad_x,
                               float* grad_p, float* grad_sv);

/* Copy the surviving candidate ids, ascending, into g_out (device, capacity
 * cap); *count_host receives the number of survivors (host pointer).
 * Errors: GFS_ERR_STATE, GFS_ERR_ARG (cap too small: *count_host still set). */
int gfs_survivors(gfs_ctx* ctx, int64_t* g_out, int64_t cap, int64_t* count_host);

/* ---- exact coverage of each sample sphere (Prop. 1 (ii)) ------------------ */
/* out[i] for every sphere of the context's current state (input order, n
 * bytes, device): 1 when some point of sphere i lies in no other ball shrunk
 * by tol, 0 when every point is covered, 2 when not decided (the certificate
 * below outgrew its 512 members).  Exact in the sense of Def. 1: the test
 * points are the circles where the other shrunk balls cut the sphere (two
 * points each) and the points where two of them meet on it (the D points),
 * each tested against every ball but the ones it was built from, in FP64; a
 * sample with s_i = 0 is the point p_i.  Rather than every pair of the balls
 * that meet the sphere, each sphere grows a certificate: a set of those
 * balls, started from the ones holding six probe points, whose test points
 * are checked first against the set and then against all balls; a ball that
 * holds a point joins the set, a point no ball holds decides "uncovered",
 * and a set whose every test point is held by another member covers the
 * sphere (the boundary argument of Prop. 1 applied to its caps).
 * witness (device, 3n doubles, or null): for out[i] = 1 the uncovered test
 * point (p_i for a zero sample, p_i + (|s_i|, 0, 0) when no ball meets the
 * sphere), NaN otherwise.  The icosphere survivors are a subset: a sphere
 * with a survivor is uncovered.  One thread per sphere.  No host
 * synchronisation, no allocation.  Errors: GFS_ERR_STATE (no build),
 * GFS_ERR_ARG, GFS_ERR_CUDA. */
int gfs_sphere_uncovered(gfs_ctx* ctx, uint8_t* out, double* witness);

/* ---- uncovered intersection circles and points (Sec. 4.1, Def. 1) --------- */
/* The U and D precomputation of Sec. 4.1 for the context's current state,
 * over the spheres S_i = (p_i, |s_i|) with |s_i| > 0 (input indices):
 *  circles: the pairs i < j whose spheres cut in a circle with a point in no
 *    other ball shrunk by tol -- the circles whose points D of Def. 1 a
 *    query at any x may grow to;
 *  points (U of Def. 1): the points shared by three spheres i < j < m (two
 *    per triple: side 0 and 1 of the trilateration in the frame of p_i, p_j,
 *    p_m) that lie in no ball but those three shrunk by tol.
 * Where the paper finds candidate pairs and triples by rasterising the
 * contour of the union of spheres, the library starts from the spheres
 * that gfs_sphere_uncovered finds uncovered (a circle or point of a covered
 * sphere is covered), walks the sphere hierarchy for the spheres that cut
 * each, decides each circle with a growing certificate of covering balls
 * (its extreme points and its crossings with the members' shrunk spheres,
 * the same test points and tests as a full enumeration) and, on an
 * uncovered circle, tests the points shared with every sphere that crosses
 * it.  Outputs (device, sorted lexicographically): circles_out 2 int64 per
 * circle (i, j); quads_out 4 int64 per point (i, j, m, side); points_out 3
 * doubles per point.  counts_host (host, 3 int64): the numbers of circles
 * and points, and a status word (bit 0: a circle's certificate outgrew 512
 * members and the circle was taken as uncovered).  Synchronises the
 * context's stream and allocates scratch on the device.
 * Errors: GFS_ERR_STATE (no build), GFS_ERR_ARG (null pointers, negative
 * capacities, or counts above the capacities: counts_host still set, nothing
 * written), GFS_ERR_TOO_LARGE (2^31 entries or more), GFS_ERR_CUDA. */
int gfs_uncovered_intersections(gfs_ctx* ctx, int64_t cap_circles, int64_t* circles_out, int64_t cap_points,
                                int64_t* quads_out, double* points_out, int64_t* counts_host);

/* ---- exact minimum valid radius (Sec. 6, over T u U u D) ------------------ */
/* rmin_out[q] (device, m doubles) = the least distance from x[q] (device,
 * m*3 doubles) to a grow-to point of Def. 1 that no other ball shrunk by tol
 * holds, for the sign sigma[q] (device, m int8: +1, -1, or 0 for no sign
 * filter) -- the minimum valid radius for a known sign of Sec. 6
 * (min_valid_radius_for_known_sign), exactly, not over icosphere
 * candidates: the uncovered points U shared by three spheres none of whose
 * signs is opposite to sigma, the points of their uncovered circles nearest
 * to and farthest from x (D), and the near and far tangent points of every
 * sphere (T), in the box when the context culls by it; INFINITY when no
 * candidate exists.  U and the uncovered circles come from the state's U
 * and D precomputation (gfs_uncovered_intersections, computed on the first
 * call for a state: that call synchronises the stream and allocates);
 * every point is then built and tested in FP64 as Def. 1 states.  One warp
 * per point scans every uncovered point, circle and sphere, so this is for
 * moderate inputs (thousands of spheres) and for checking the discrete
 * values against the exact ones.  Errors: GFS_ERR_STATE (no build),
 * GFS_ERR_ARG, GFS_ERR_CUDA. */
int gfs_exact_rmin(gfs_ctx* ctx, const double* x, const int8_t* sigma, int64_t m, double* rmin_out);

/* ---- refinement order (Sec. 4.2) ------------------------------------------ */
/* The greedy refinement depends on the order of the new points.  The paper
 * orders the interesting cells by a flood fill that starts at the least
 * covered cell, with coverage estimated from regularly spaced points.
 *
 * gfs_cell_coverage: for each cell c with integer coordinates
 * (i, j, k) = cells[3c .. 3c+2], its sub^3 points
 *   origin + h * ((i, j, k) + ((a, b, c) + 1/2) / sub),  a, b, c < sub
 * (each coordinate rounded per operation in that order) are tested for
 * containment in the balls of the context's current samples, of either
 * sign, shrunk by tol (the cull's coverage predicate, decided in FP64);
 * counts_out[c] = the number contained (the covered area ratio times sub^3).
 * cells: device, ncells*3 int32.  origin_host: host, 3 FP64.  h > 0.
 * 1 <= sub <= 64.  counts_out: device, ncells uint32.  One warp per cell; no
 * host synchronisation, no allocation.  Errors: GFS_ERR_STATE (no build),
 * GFS_ERR_ARG, GFS_ERR_CUDA. */
int gfs_cell_coverage(gfs_ctx* ctx, const int32_t* cells, int64_t ncells, const double* origin_host, double h,
                      int sub, uint32_t* counts_out);

/* gfs_flood_order (host computation, no device needed): the flood-fill
 * order of ncells cells (cells_host: ncells*3 int32 coordinates, each
 * within +-(2^20 - 2); counts_host: their covered counts).  Start at the
 * cell with the lowest count; repeatedly take the queued cell with the
 * lowest count (ties: lower index), emit it and queue its not yet queued
 * neighbours among the listed cells (cells sharing a face, an edge or a
 * corner); when the queue is empty, start again at the lowest-count cell
 * not yet emitted.  order_out_host: host, ncells int64 indices in emission
 * order.  Errors: GFS_ERR_ARG (null, negative count, a cell listed twice),
 * GFS_ERR_TOO_LARGE (coordinates out of range). */
int gfs_flood_order(const int32_t* cells_host, const uint32_t* counts_host, int64_t ncells, int64_t* order_out_host);

/* ---- batched shapes ------------------------------------------------------ */
/* One independent shape of a batched call: its samples, its query points and
 * its outputs (all device pointers; outputs nullable).  Layout and meaning
 * are those of gfs_build / gfs_query. */
typedef struct {
  const double* p_xyz;  /* n*3 FP64 sample positions */
  const double* s;      /* n FP64 samples */
  int64_t n;
  const void* x;        /* m*3 query points, FP64 or FP32 */
  int x_is_fp32;
  int64_t m;
  float* s_out;         /* m FP32 values */
  double* s64_out;      /* m FP64 values */
  int64_t* argmin_out;  /* m candidate ids (local to the shape) or sphere indices */
  uint16_t* flags_out;  /* m result words */
} gfs_shape;

/* P build of many shapes at once: one cull launch covers every shape's
 * candidates, a block per (shape, direction, 128 spheres) item (the library
 * keeps the shape table; the caller keeps the buffers alive until the last
 * gfs_batch_query).  Results per shape are those of gfs_build on that shape
 * alone.  Sizes every buffer (the survivor capacity is grown and the cull
 * rerun until the counts fit) and uploads the shape table, so that
 * gfs_batch_rebuild can later repeat the build without the host.  The first
 * build also picks the persistent query's grid size by timing a few
 * candidates (autotuning).  Synchronises the stream.  Errors: GFS_ERR_ARG (nshapes < 1 or > 65535, a
 * shape with n < 1), GFS_ERR_TOO_LARGE, GFS_ERR_OOM, GFS_ERR_CUDA. */
int gfs_batch_build(gfs_ctx* ctx, const gfs_shape* shapes_host, int nshapes);

/* Rebuild of the last gfs_batch_build's shapes from the current contents of
 * their sample buffers (the same shape table: same pointers and sample and
 * query counts; new positions and values): the whole build -- inputs copied
 * and Morton-sorted, sample forest, cull, survivor forests laid out from the
 * device-side survivor counts, query views -- issues no host
 * synchronisation, no allocation and no host-to-device copy, so it can be
 * captured in a CUDA graph together with gfs_batch_query and replayed.
 * Capacities are the first build's: survivors beyond the survivor capacity
 * are dropped and set a status bit (read with gfs_batch_status; the
 * results of that rebuild are then not valid -- call gfs_batch_build again,
 * which sizes the capacity for the new counts).
 * Errors: GFS_ERR_STATE (no batch build), GFS_ERR_CUDA. */
int gfs_batch_rebuild(gfs_ctx* ctx);

/* Status bits of the batched builds since the last call (then cleared):
 * 1 and 2 -- survivors of the positive / negative class exceeded the
 * capacity; 4 -- a survivor forest exceeded its node capacity.  0: every
 * build was complete.  Synchronises the stream.
 * Errors: GFS_ERR_ARG (null), GFS_ERR_STATE (no batch build), GFS_ERR_CUDA. */
int gfs_batch_status(gfs_ctx* ctx, unsigned* status_host);

/* Queries of every shape of the last gfs_batch_build in two persistent
 * launches (the sphere pass of every point, then the rest), into each
 * shape's outputs.  Issues no host synchronisation and no
 * allocation, so it can be captured in a CUDA graph and replayed (with new
 * point coordinates written into the same buffers).
 * Errors: GFS_ERR_STATE (no batch build), GFS_ERR_CUDA. */
int gfs_batch_query(gfs_ctx* ctx);

/* Same-sign tangent augmentation (as gfs_query_tangent) of the outputs of
 * the last gfs_batch_query, shape by shape; every shape with points needs
 * its argmin and flags outputs.  One launch per shape, in the Morton order
 * of that gfs_batch_query; no host synchronisation and no allocation.
 * Errors: GFS_ERR_STATE (no batch build), GFS_ERR_ARG (a shape without
 * argmin or flags outputs; nothing is launched), GFS_ERR_CUDA. */
int gfs_batch_query_tangent(gfs_ctx* ctx);

/* Surviving candidate ids of one shape of the batch, ascending (device
 * g_out, capacity cap; *count_host set).  Errors as gfs_survivors. */
int gfs_batch_survivors(gfs_ctx* ctx, int shape, int64_t* g_out, int64_t cap, int64_t* count_host);

/* Counters of the last build/query (host struct). */
typedef struct {
  int64_t n_spheres;        /* spheres in the current state */
  int64_t n_candidates;     /* n * K generated by the last build */
  int64_t n_survivors;      /* survivors (unique ids) */
  int64_t n_survivors_pos;  /* survivors on positive or zero spheres */
  int64_t n_survivors_neg;  /* survivors on negative or zero spheres */
  int64_t cull_fp64_rechecks;  /* coverage predicates re-decided in FP64 by the build */
  int64_t query_fp64_rechecks; /* predicates re-decided in FP64 by the last query */
  int64_t query_deferred;      /* queries finished by the FP64 path in the last query */
  int64_t tree_levels;         /* levels of the sphere hierarchy */
  int64_t query_sphere_node_tests; /* child-node bound tests of the last query's sphere pass (sum over points) */
  int64_t query_sphere_items;  /* spheres tested by the last query */
  int64_t query_surv_node_tests;   /* child-node bound tests of the last query's survivor pass */
  int64_t query_band_passes;   /* FP64 passes over an error band that settled near-ties */
  int64_t query_surv_items;    /* survivors tested by the last query */
  /* phase times of the last build / query in ms (timing = 1 only, else 0) */
  double ms_build_total;       /* whole gfs_build */
  double ms_build_cull;        /* candidate culling kernel */
  double ms_query_fast;        /* FP32 query kernel */
  double ms_query_exact;       /* FP64 kernel for queries outside the FP32 error model */
  int64_t kernel_launches;     /* kernels this library has launched in this process (cumulative) */
  int64_t sort_calls;          /* radix-sort calls (each launches a few library-sort kernels) */
  int64_t cull_node_tests;     /* child-node coverage tests of the last build (sum over open candidates) */
  int64_t cull_items;          /* sphere coverage tests of the last build (sum over open candidates) */
  double ms_query_spheres;     /* first of the query's two FP32 kernels (the pass over the spheres); part of
                                  ms_query_fast (timing = 1 only) */
  int64_t insert_rounds;       /* rounds of the last gfs_insert / gfs_insert_known call */
  int64_t insert_steps;        /* steps it committed (its T) */
  int64_t insert_rebuilds;     /* hierarchy rebuilds between its rounds */
  double insert_ms_total;      /* host wall time of that call */
  double insert_ms_rebuild;    /* of which in the rebuilds between rounds */
  double insert_ms_final;      /* of which in the final renumbering and rebuild */
  double insert_ms_query;      /* device time of its step queries (timing = 1 only) */
  double insert_ms_commit;     /* device time of its commit tests and commits (timing = 1 only) */
  double insert_ms_update;     /* device time of its state updates (timing = 1 only) */
  int64_t insert_slots;        /* step queries it evaluated (window slots over all rounds) */
  int64_t insert_sph_exact;    /* spheres its step queries evaluated exactly in FP64 */
  int64_t insert_sph_tested;   /* spheres they screened in FP32 */
  int64_t insert_surv_exact;   /* survivors they evaluated exactly in FP64 */
  int64_t insert_surv_tested;  /* survivors they screened in FP32 */
  int64_t batch_sphere_items;  /* (point, sphere) tests of the last gfs_batch_query */
  int64_t batch_sphere_node_tests; /* its child-node bound tests of the sphere pass */
  int64_t batch_surv_items;    /* its (point, survivor) tests */
  int64_t batch_cull_tile[3];  /* autotuned cull tile (spheres per block) of the batch's shapes with < 32k,
                                  < 256k and more samples (0: no such shape) */
  int64_t batch_query_grid;    /* autotuned grid of the persistent batched query (blocks) */
} gfs_stats_t;

/* Synchronises the stream and fills *out (host). */
int gfs_stats(gfs_ctx* ctx, gfs_stats_t* out);

/* Whole path from HOST buffers: copies p_host (n*3 FP64) and s_host (n FP64)
 * and x_host (m*3, FP64 or FP32) to library-owned device memory, runs
 * gfs_build and gfs_query, and copies the FP32 values, argmins and result
 * words back into s_out_host / argmin_out_host / flags_out_host (each
 * nullable).  Host buffers should be page-locked for asynchronous copies.
 * The upload of x runs on a second stream the context owns and overlaps
 * the build.
 * Returns after the results are in host memory (synchronises the stream).
 * Errors: as gfs_build / gfs_query. */
int gfs_solve_host(gfs_ctx* ctx, const double* p_host, const double* s_host, int64_t n, const void* x_host,
                   int x_is_fp32, int64_t m, float* s_out_host, int64_t* argmin_out_host,
                   uint16_t* flags_out_host);

/* ---- measurement ----------------------------------------------------------- */
/* Arithmetic peak probe (not part of the method): one launch of
 * blocks_per_sm x (SM count) blocks of 256 threads, each thread running 16
 * independent fused multiply-add chains for iters x 8 steps in FP32
 * (fp64 = 0) or FP64 (fp64 = 1), on the given stream.  The path's kernels
 * are bound by these pipes; their roofline fractions divide by the rate this
 * launch reaches (time it with events on the same stream).
 * sink: device buffer of at least blocks x 256 elements of the chosen type
 * (sink_bytes), overwritten.  *flops_host (host) receives the launch's flop
 * count (2 per multiply-add).  No synchronisation, no allocation.
 * Errors: GFS_ERR_ARG (iters < 1, blocks_per_sm outside 1..8, sink too small,
 * null pointers), GFS_ERR_CUDA. */
int gfs_fma_probe(int fp64, int64_t iters, int blocks_per_sm, void* sink, int64_t sink_bytes, void* cuda_stream,
                  double* flops_host);

/* The icosphere direction table the library uses (host computation, no
 * device needed): writes K = 10*4^tau+2 rows of FP64 (x,y,z) into out_host
 * (capacity cap_rows).  Returns K, or -1 on bad arguments. */
int gfs_icosphere(int tau, double* out_host, int64_t cap_rows);

const char* gfs_strerror(int status);

/* Release the context and all library-owned device memory. */
void gfs_destroy(gfs_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* GFS_H */
