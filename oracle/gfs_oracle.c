/*
 * gfs_oracle.c -- plain FP64 CPU oracle for the consistent-SDF hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library links, includes or calls
 * this file; only the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg load it.  It shares no code, header or table generator
 * with the CUDA library.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fPIC -shared
 * (-ffp-contract=off matters: every product and sum below must be rounded on
 * its own, in the order written, so that the device's FP64 re-decision path
 * can reproduce each value bit for bit).
 *
 * What it computes (the method of "Greed for the Spheres", discretised):
 *  - Sec. 3.1: a sample (p_i, s_i) is a sphere of radius |s_i| and sign
 *    sign(s_i); the surface never enters the open ball.
 *  - Prop. 1 (ii): every sphere keeps an "uncovered" point, i.e. a point not
 *    inside any other ball.  Def. 1 / Prop. 2: the minimum valid radius at x
 *    is the distance from x to the nearest uncovered point of the contour of
 *    the spheres of x's sign (the closest valid grow-to point).
 *  - Discretisation: the grow-to points T/U/D of Def. 1 are replaced by the
 *    vertices of a geodesic icosphere of depth tau placed on every sphere
 *    ("candidates"); a candidate survives when it lies in the domain box
 *    [-1,1]^3 (App. B) and no other ball, shrunk by tol = 1e-6 (App. B),
 *    contains it.
 *  - Sec. 4.3 heuristic bounds: LB = largest near-tangent distance over the
 *    spheres containing x; UB = nearest tangent point of an opposite sphere;
 *    far bound = nearest far tangent point of any sphere.
 *  - Sec. 6 (min_valid_radius_for_known_sign): the exact T/U/D enumeration,
 *    kept here by brute force for tiny inputs only (orc_exact_rmin).
 *  - Prop. 1 (ii) exactly: whether each sphere keeps a point outside every
 *    other ball, from the circle and triple points of Def. 1
 *    (orc_sphere_uncovered).
 *  - The U and D precomputation of Sec. 4.1: the intersection circles with
 *    an uncovered point and the uncovered points shared by three spheres
 *    (orc_uncovered_intersections).
 *  - Sec. 4.2 refinement order: the covered area ratio of grid cells from
 *    regularly spaced sub-points (orc_cell_coverage); the flood-fill order
 *    itself is plain Python in oracle.py.
 *  - The same-sign tangent points of Def. 1 as extra query candidates
 *    (orc_query_aug, orc_query_aug_lazy) and the point behind each value
 *    (orc_argmin_points).
 *  - Sec. 3.3 scored value (score_for_radius, interpolate_sdf_to): the
 *    best-scoring valid grow-to radius (orc_query_scored).
 *
 * Readings where the paper is silent are listed in the design notes; the
 * ones that fix arithmetic are repeated at each function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_INF (1.0 / 0.0)

/* result codes (low 4 bits of a flag word) */
#define CODE_SURVIVOR 0  /* value = distance to the nearest surviving candidate */
#define CODE_OPPOSITE 1  /* value = distance to the nearest opposite tangent point */
#define CODE_SAMPLE 2    /* x is an input position: value = its sample */
#define CODE_OUTSIDE 3   /* x lies in no ball: value 0 (Prop. 2 proof) */
#define CODE_INVALID 4   /* x lies in balls of both signs (input violates Prop. 1) */
#define CODE_LOWER 5     /* no candidate at all: value = lower bound LB */
#define CODE_TANGENT 6   /* augmented query: value = distance to an uncovered same-sign tangent point */
/* violation bits (shifted by 4) */
#define FLAG_LB_VIOL (1 << 4)
#define FLAG_FAR_VIOL (1 << 5)
#define FLAG_OPP_VIOL (1 << 6)
#define FLAG_LOST_WITNESS (1 << 7)
#define FLAG_NONCONSERVATIVE (1 << 8) /* repair: |value| < |known value| - tol */

/* ------------------------------------------------------------------------ */
/* elementary FP64 pieces, each written in the one order the device repeats */
/* ------------------------------------------------------------------------ */

static double dist2(const double* a, const double* b) {
  double dx = a[0] - b[0];
  double dy = a[1] - b[1];
  double dz = a[2] - b[2];
  return dx * dx + dy * dy + dz * dz; /* ((dx*dx + dy*dy) + dz*dz) */
}

static int sgn(double v) { return v > 0.0 ? 1 : (v < 0.0 ? -1 : 0); }

/* cov(q, j): q lies in the open ball of sphere j shrunk by tol (Sec. 3.1
 * "does not penetrate the open ball"; App. B tolerance 1e-6). */
static int covers(const double* q, const double* pj, double sj, double tol) {
  double r = fabs(sj);
  if (!(r > tol)) return 0;
  double rt = r - tol;
  return dist2(q, pj) < rt * rt;
}

static int inbox(const double* q) {
  return fabs(q[0]) <= 1.0 && fabs(q[1]) <= 1.0 && fabs(q[2]) <= 1.0;
}

/* candidate (i,k): q = p_i + |s_i| * u_k, per component, product then sum */
static void cand_pos(const double* p, double s, const double* u, double* q) {
  double r = fabs(s);
  q[0] = p[0] + r * u[0];
  q[1] = p[1] + r * u[1];
  q[2] = p[2] + r * u[2];
}

/* ------------------------------------------------------------------------ */
/* geodesic icosphere (directions u_k, k < K = 10*4^tau + 2)                 */
/* ------------------------------------------------------------------------ */
/* Construction (not in the paper; fixed here so that the vertex table is a
 * single well-defined list):
 *  1. the 12 icosahedron vertices are the cyclic permutations of
 *     (+-1, +-phi, 0) in the order listed below, each divided by its norm;
 *  2. the 20 faces are every triple a<b<c of mutually adjacent vertices
 *     (unnormalised squared distance 4), in lexicographic order, turned so
 *     that (b-a)x(c-a) points away from the origin (else b and c swap);
 *  3. each level walks the faces in order; for a face (a,b,c) it looks up
 *     the midpoints of edges ab, bc, ca in that order, creating a new vertex
 *     (v_a + v_b) / |v_a + v_b| at the end of the list on first sight of the
 *     edge, and emits the faces (a,ab,ca), (b,bc,ab), (c,ca,bc), (ab,bc,ca).
 * Vertices never move, so the table at depth tau is a prefix of the table at
 * depth tau+1. */

static double norm3(const double* v) { return sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }

typedef struct { int64_t key; int val; } orc_edge;

static int edge_lookup(orc_edge* tab, int64_t cap, int a, int b, int* created, double* V, int* nv) {
  int lo = a < b ? a : b, hi = a < b ? b : a;
  int64_t key = (int64_t)lo * 1000003LL + hi;
  uint64_t h = (uint64_t)key * 0x9E3779B97F4A7C15ULL;
  int64_t slot = (int64_t)(h % (uint64_t)cap);
  while (tab[slot].key >= 0) {
    if (tab[slot].key == key) { *created = 0; return tab[slot].val; }
    slot = (slot + 1) % cap;
  }
  int idx = (*nv)++;
  double m[3] = {V[3 * a + 0] + V[3 * b + 0], V[3 * a + 1] + V[3 * b + 1], V[3 * a + 2] + V[3 * b + 2]};
  double nm = norm3(m);
  V[3 * idx + 0] = m[0] / nm;
  V[3 * idx + 1] = m[1] / nm;
  V[3 * idx + 2] = m[2] / nm;
  tab[slot].key = key;
  tab[slot].val = idx;
  *created = 1;
  return idx;
}

/* Returns K = 10*4^tau+2 and writes the K*3 table, or -1 on bad arguments. */
int orc_icosphere(int tau, double* out, int64_t cap_rows) {
  if (tau < 0 || tau > 7) return -1;
  int64_t K = 10LL * (1LL << (2 * tau)) + 2;
  if (cap_rows < K) return -1;
  const double phi = (1.0 + sqrt(5.0)) / 2.0;
  const double base[12][3] = {{-1, phi, 0}, {1, phi, 0}, {-1, -phi, 0}, {1, -phi, 0},
                              {0, -1, phi}, {0, 1, phi}, {0, -1, -phi}, {0, 1, -phi},
                              {phi, 0, -1}, {phi, 0, 1}, {-phi, 0, -1}, {-phi, 0, 1}};
  double* V = out;
  for (int v = 0; v < 12; ++v) {
    double n = norm3(base[v]);
    V[3 * v + 0] = base[v][0] / n;
    V[3 * v + 1] = base[v][1] / n;
    V[3 * v + 2] = base[v][2] / n;
  }
  /* faces of the icosahedron from adjacency of the unnormalised vertices */
  int64_t fcap = 20LL * (1LL << (2 * tau));
  int* F = (int*)malloc(sizeof(int) * 3 * fcap);
  int* G = (int*)malloc(sizeof(int) * 3 * fcap);
  int nf = 0;
  for (int a = 0; a < 12; ++a)
    for (int b = a + 1; b < 12; ++b)
      for (int c = b + 1; c < 12; ++c) {
        double dab = dist2(base[a], base[b]), dbc = dist2(base[b], base[c]), dca = dist2(base[c], base[a]);
        if (fabs(dab - 4.0) < 1e-9 && fabs(dbc - 4.0) < 1e-9 && fabs(dca - 4.0) < 1e-9) {
          double e1[3] = {base[b][0] - base[a][0], base[b][1] - base[a][1], base[b][2] - base[a][2]};
          double e2[3] = {base[c][0] - base[a][0], base[c][1] - base[a][1], base[c][2] - base[a][2]};
          double nrm[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
          double cen[3] = {base[a][0] + base[b][0] + base[c][0], base[a][1] + base[b][1] + base[c][1],
                           base[a][2] + base[b][2] + base[c][2]};
          double o = nrm[0] * cen[0] + nrm[1] * cen[1] + nrm[2] * cen[2];
          F[3 * nf + 0] = a;
          F[3 * nf + 1] = o > 0 ? b : c;
          F[3 * nf + 2] = o > 0 ? c : b;
          ++nf;
        }
      }
  if (nf != 20) { free(F); free(G); return -1; }
  int nv = 12;
  int64_t ecap = 4 * (30LL * (1LL << (2 * tau))) + 17;
  orc_edge* tab = (orc_edge*)malloc(sizeof(orc_edge) * ecap);
  for (int level = 0; level < tau; ++level) {
    for (int64_t e = 0; e < ecap; ++e) tab[e].key = -1;
    int ng = 0;
    for (int f = 0; f < nf; ++f) {
      int a = F[3 * f], b = F[3 * f + 1], c = F[3 * f + 2], cr;
      int ab = edge_lookup(tab, ecap, a, b, &cr, V, &nv);
      int bc = edge_lookup(tab, ecap, b, c, &cr, V, &nv);
      int ca = edge_lookup(tab, ecap, c, a, &cr, V, &nv);
      int kids[4][3] = {{a, ab, ca}, {b, bc, ab}, {c, ca, bc}, {ab, bc, ca}};
      for (int t = 0; t < 4; ++t) {
        G[3 * ng + 0] = kids[t][0];
        G[3 * ng + 1] = kids[t][1];
        G[3 * ng + 2] = kids[t][2];
        ++ng;
      }
    }
    int* tmp = F; F = G; G = tmp;
    nf = ng;
  }
  free(tab);
  free(F);
  free(G);
  return nv == K ? (int)K : -1;
}

/* ------------------------------------------------------------------------ */
/* P build: keep(i,k)                                                        */
/* ------------------------------------------------------------------------ */

/* keep(i,k) <=> (box_cull => q in [-1,1]^3) and no j != i covers q. */
int orc_keep_one(const double* p, const double* s, int64_t n, const double* U, int K, double tol,
                 int box_cull, int64_t i, int k) {
  double q[3];
  (void)K;
  cand_pos(p + 3 * i, s[i], U + 3 * k, q);
  if (box_cull && !inbox(q)) return 0;
  for (int64_t j = 0; j < n; ++j) {
    if (j == i) continue;
    if (covers(q, p + 3 * j, s[j], tol)) return 0;
  }
  return 1;
}

void orc_keep_all(const double* p, const double* s, int64_t n, const double* U, int K, double tol,
                  int box_cull, uint8_t* keep) {
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < K; ++k) keep[i * K + k] = (uint8_t)orc_keep_one(p, s, n, U, K, tol, box_cull, i, k);
}

/* candidate list (g, sphere, q) of all kept candidates; g = i*(K+1) + k */
int64_t orc_collect(const double* p, const double* s, int64_t n, const double* U, int K, const uint8_t* keep,
                    int64_t* g_out, int64_t* sph_out, double* q_out) {
  int64_t c = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < K; ++k)
      if (keep[i * K + k]) {
        if (g_out) {
          g_out[c] = i * (int64_t)(K + 1) + k;
          sph_out[c] = i;
          cand_pos(p + 3 * i, s[i], U + 3 * k, q_out + 3 * c);
        }
        ++c;
      }
  return c;
}

/* ------------------------------------------------------------------------ */
/* query: the consistent value at x                                          */
/* ------------------------------------------------------------------------ */

typedef struct {
  double value;   /* signed value s*(x) (NaN for INVALID) */
  int64_t argmin; /* candidate id g, sphere index j, or -1 (per code) */
  int32_t flags;  /* code | violation bits */
  double gap;     /* second-nearest minus nearest candidate distance */
} orc_result;

/* Sign and containment (Prop. 2 proof; Sec. 4.3 known-sign inference):
 * C_+ / C_- = spheres of that sign whose shrunk open ball holds x.
 * Both empty -> OUTSIDE (value 0); both non-empty -> INVALID. */
static int classify(const double* p, const double* s, int64_t n, double tol, const double* x, int* sigma) {
  int anyP = 0, anyN = 0;
  for (int64_t j = 0; j < n; ++j)
    if (covers(x, p + 3 * j, s[j], tol)) {
      if (s[j] > 0) anyP = 1;
      else if (s[j] < 0) anyN = 1;
    }
  if (anyP && anyN) return CODE_INVALID;
  if (!anyP && !anyN) return CODE_OUTSIDE;
  *sigma = anyP ? 1 : -1;
  return -1;
}

/* Finish a query once the nearest survivor (d2 best, id bestg) is known:
 * UB_opp (nearest opposite tangent point, Sec. 4.3 / Def. 1 T), the value,
 * and the Sec. 4.3 bound checks. */
static orc_result finish(const double* p, const double* s, int64_t n, double tol, int clamp_opp,
                         const double* x, int sigma, double bestd2, int64_t bestg, double second_d2) {
  orc_result R;
  double ub = ORC_INF, ub2 = ORC_INF, lb = -ORC_INF, far = ORC_INF;
  int64_t ubj = -1, lbj = -1;
  for (int64_t j = 0; j < n; ++j) {
    double r = fabs(s[j]);
    double d = sqrt(dist2(x, p + 3 * j));
    int c = sgn(s[j]);
    if (c == -sigma) {
      double a = d - r;
      if (a < ub) { ub2 = ub; ub = a; ubj = j; }
      else if (a < ub2) ub2 = a;
    }
    if (c == sigma) {
      double b = r - d;
      if (b > lb) { lb = b; lbj = j; }
    }
    double f = d + r;
    if (f < far) far = f;
  }
  double dS = bestg >= 0 ? sqrt(bestd2) : ORC_INF;
  double m;
  int code;
  if (bestg >= 0 && (!clamp_opp || dS <= ub)) {
    code = CODE_SURVIVOR;
    m = dS;
    R.argmin = bestg;
  } else if (clamp_opp && ubj >= 0) {
    code = CODE_OPPOSITE;
    m = ub;
    R.argmin = ubj;
  } else {
    code = CODE_LOWER;
    m = lb;
    R.argmin = lbj;
  }
  if (m < 0.0) m = 0.0;
  int flags = code;
  if (m < lb - tol) flags |= FLAG_LB_VIOL;
  if (m > far + tol) flags |= FLAG_FAR_VIOL;
  if (ubj >= 0 && ub < m - tol) flags |= FLAG_OPP_VIOL;
  R.value = sigma > 0 ? m : -m;
  R.flags = flags;
  /* gap between the two nearest candidates (survivors and opposite tangent
   * points together); used by tests to stay away from argmin switches */
  double c1 = dS, c2 = second_d2 < ORC_INF ? sqrt(second_d2) : ORC_INF;
  double cand[4] = {c1, c2, clamp_opp ? ub : ORC_INF, clamp_opp ? ub2 : ORC_INF};
  double b1 = ORC_INF, b2 = ORC_INF;
  for (int t = 0; t < 4; ++t) {
    if (cand[t] < b1) { b2 = b1; b1 = cand[t]; }
    else if (cand[t] < b2) b2 = cand[t];
  }
  R.gap = b2 - b1;
  return R;
}

static int64_t sample_index(const double* p, int64_t n, const double* x) {
  for (int64_t i = 0; i < n; ++i)
    if (p[3 * i] == x[0] && p[3 * i + 1] == x[1] && p[3 * i + 2] == x[2]) return i;
  return -1;
}

/* known: 0 = infer the sign from containment; +1 / -1 = the sign is given
 * (Sec. 6 min_valid_radius_for_known_sign: the repair knows each removed
 * sample's sign), so no OUTSIDE / INVALID outcome */
static orc_result query_one(const double* p, const double* s, int64_t n, const int64_t* sg, const int64_t* ssph,
                            const double* sq, int64_t ns, double tol, int clamp_opp, const double* x, int known) {
  orc_result R;
  R.gap = ORC_INF;
  int64_t si = sample_index(p, n, x);
  if (si >= 0) { /* input values are reproduced exactly */
    R.value = s[si];
    R.argmin = si;
    R.flags = CODE_SAMPLE;
    return R;
  }
  int sigma = known;
  int code = known ? -1 : classify(p, s, n, tol, x, &sigma);
  if (code >= 0) {
    R.value = code == CODE_OUTSIDE ? 0.0 : (0.0 / 0.0);
    R.argmin = -1;
    R.flags = code;
    return R;
  }
  /* d_S: nearest surviving candidate on a sphere of x's sign (or of a zero
   * sample); ties go to the lowest candidate id. */
  double best = ORC_INF, second = ORC_INF;
  int64_t bestg = -1;
  for (int64_t t = 0; t < ns; ++t) {
    int c = sgn(s[ssph[t]]);
    if (c != sigma && c != 0) continue;
    double d2 = dist2(x, sq + 3 * t);
    if (d2 < best || (d2 == best && sg[t] < bestg)) {
      second = best;
      best = d2;
      bestg = sg[t];
    } else if (d2 < second) {
      second = d2;
    }
  }
  return finish(p, s, n, tol, clamp_opp, x, sigma, best, bestg, second);
}

void orc_query(const double* p, const double* s, int64_t n, const int64_t* sg, const int64_t* ssph,
               const double* sq, int64_t ns, double tol, int clamp_opp, const double* x, int64_t m,
               double* value, int64_t* argmin, int32_t* flags, double* gap) {
  for (int64_t t = 0; t < m; ++t) {
    orc_result R = query_one(p, s, n, sg, ssph, sq, ns, tol, clamp_opp, x + 3 * t, 0);
    value[t] = R.value;
    argmin[t] = R.argmin;
    flags[t] = R.flags;
    if (gap) gap[t] = R.gap;
  }
}

/* Query with same-sign tangent augmentation (the tangent points T of
 * Def. 1 of the spheres of x's own sign, Sec. 3.2 / Sec. 6): besides the
 * surviving candidates, the candidate set holds, for every sphere j with
 * sign(s_j) = sign of x and |s_j| > 0, its near and far tangent points in
 * the direction of x, t = p_j +- |s_j| (x - p_j)/|x - p_j| (none when
 * x = p_j), kept when they lie in no ball but j's own (shrunk by tol) and,
 * with box_cull, in the box.  The nearest candidate (squared distances;
 * survivors win ties, then the lowest 2j + side, side 0 near, 1 far) gives
 * the value, clamped by UB_opp exactly as in orc_query; a tangent winner has
 * code TANGENT and argmin 2j + side.  Brute force: O(n^2) per point. */
void orc_query_aug(const double* p, const double* s, int64_t n, const int64_t* sg, const int64_t* ssph,
                   const double* sq, int64_t ns, double tol, int clamp_opp, int box_cull, const double* x,
                   int64_t m, double* value, int64_t* argmin, int32_t* flags) {
  for (int64_t t = 0; t < m; ++t) {
    const double* xq = x + 3 * t;
    orc_result R = query_one(p, s, n, sg, ssph, sq, ns, tol, clamp_opp, xq, 0);
    const int code = R.flags & 15;
    if (code != CODE_SURVIVOR && code != CODE_OPPOSITE && code != CODE_LOWER) {
      value[t] = R.value;
      argmin[t] = R.argmin;
      flags[t] = R.flags;
      continue;
    }
    int sig = 0; /* x's class, from containment (the value may be 0) */
    classify(p, s, n, tol, xq, &sig);
    /* the nearest uncovered same-sign tangent point */
    double tbest = ORC_INF;
    int64_t tid = -1;
    for (int64_t j = 0; j < n; ++j) {
      if (sgn(s[j]) != sig) continue;
      const double r = fabs(s[j]);
      const double* pj = p + 3 * j;
      double v[3] = {xq[0] - pj[0], xq[1] - pj[1], xq[2] - pj[2]};
      const double dv = norm3(v);
      if (!(dv > 0.0)) continue;
      for (int side = 0; side < 2; ++side) {
        const double sgnr = side == 0 ? r : -r;
        double tp[3];
        for (int c = 0; c < 3; ++c) tp[c] = pj[c] + sgnr * (v[c] / dv);
        if (box_cull && !inbox(tp)) continue;
        int cov = 0;
        for (int64_t k = 0; k < n && !cov; ++k)
          if (k != j && covers(tp, p + 3 * k, s[k], tol)) cov = 1;
        if (cov) continue;
        const double d2 = dist2(xq, tp);
        const int64_t id = 2 * j + side;
        if (d2 < tbest || (d2 == tbest && id < tid)) {
          tbest = d2;
          tid = id;
        }
      }
    }
    /* survivors first: recompute their nearest (d2, g) for the comparison */
    double sbest = ORC_INF;
    int64_t sgbest = -1;
    for (int64_t u = 0; u < ns; ++u) {
      int c = sgn(s[ssph[u]]);
      if (c != sig && c != 0) continue;
      double d2 = dist2(xq, sq + 3 * u);
      if (d2 < sbest || (d2 == sbest && sg[u] < sgbest)) {
        sbest = d2;
        sgbest = sg[u];
      }
    }
    if (tid >= 0 && tbest < sbest) {
      /* a tangent point is the nearest candidate: same clamp and checks */
      orc_result T = finish(p, s, n, tol, clamp_opp, xq, sig, tbest, 0, ORC_INF);
      if ((T.flags & 15) == CODE_SURVIVOR) {
        T.flags = (T.flags & ~15) | CODE_TANGENT;
        T.argmin = tid;
      }
      R = T;
    }
    value[t] = R.value;
    argmin[t] = R.argmin;
    flags[t] = R.flags;
  }
}

/* ------------------------------------------------------------------------ */
/* scored value (Sec. 3.3: score_for_radius, interpolate_sdf_to)            */
/* ------------------------------------------------------------------------ */
#define FLAG_SCORE_FALLBACK (1 << 9) /* scored value: no valid candidate, minimum value kept */

/* The paper scores every grow-to point q (with the input sphere i it lies
 * on) for both signs of the radius |x - q| and returns the best-scoring
 * value that keeps the samples valid.  Discrete form, with readings:
 *  - grow-to points: the survivors S_tau (standing in for the intersection
 *    points U, D) and the near and far tangent points of every sphere
 *    (x != p_j, |s_j| > 0) that no other shrunk ball covers and, with the
 *    box cull, that lie in the box (T of Def. 1);
 *  - validity of the new sample (x, sign * r), Prop. 1 discretely:
 *      (V1) no ball of the opposite sign is intersected: not
 *           UB < r - tol, UB the nearest opposite tangent distance (the
 *           query's OPP_VIOL test);
 *      (V2) no other sphere with survivors loses all of them: for each
 *           sphere j != i with survivors, some survivor lies outside the
 *           new ball shrunk by tol (the cull's coverage predicate); sphere
 *           i keeps the grow-to point q, on the new sphere;
 *      (V3) no sphere lies strictly inside the new ball: not
 *           r > FAR + tol (the query's FAR_VIOL test);
 *    a sign is possible only where x is not inside a ball of the other
 *    sign (V1 then fails for every r >= 0);
 *  - normals_agree (undefined in the paper): the normals the two spheres
 *    give the surface at q, sign * (x - q) and sign(s_i) * (p_i - q), have
 *    a positive dot product;
 *  - max_possible_radius (undefined): any bound above twice every valid
 *    radius makes the type score dominate; the order is then (type class:
 *    tangency agreeing 3 > intersection agreeing 2 > intersection
 *    disagreeing 1 > tangency disagreeing 0; then sign score * r with sign
 *    score 1 for positive and 2 for negative radii);
 *  - ties (the paper's sort is unspecified): the lower candidate key
 *    (survivor id g; tangent points 2^40 + 2j + side), then the negative
 *    sign;
 *  - a sample position keeps its sample (SAMPLE), both-sign containment is
 *    INVALID; with no valid candidate the minimum value of the plain query
 *    is kept (the paper's fallback to the minimum valid radius) with
 *    FLAG_SCORE_FALLBACK.
 * Result codes: SURVIVOR (argmin g) or TANGENT (argmin 2j + side); the value
 * is sign * r; LB_VIOL is set as in the query. */
#define SCORE_TKEY ((int64_t)1 << 40)

/* some ball other than j's, shrunk by tol, contains t */
static int covered_by_other(const double* p, const double* s, int64_t n, double tol, const double* t, int64_t j) {
  for (int64_t k = 0; k < n; ++k)
    if (k != j && covers(t, p + 3 * k, s[k], tol)) return 1;
  return 0;
}

typedef struct {
  int cls;     /* type class 0..3 */
  double sr;   /* sign score * r */
  int64_t key; /* candidate key */
  int sign;    /* +1 / -1 */
  double r;
} orc_score;

static int score_better(const orc_score* a, const orc_score* b) {
  if (a->cls != b->cls) return a->cls > b->cls;
  if (a->sr != b->sr) return a->sr > b->sr;
  if (a->key != b->key) return a->key < b->key;
  return a->sign < b->sign;
}

void orc_query_scored(const double* p, const double* s, int64_t n, const int64_t* sg, const int64_t* ssph,
                      const double* sq, int64_t ns, double tol, int box_cull, const double* x, int64_t m,
                      double* value, int64_t* argmin, int32_t* flags) {
  double* maxd2 = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int64_t t = 0; t < m; ++t) {
    const double* xq = x + 3 * t;
    const orc_result R = query_one(p, s, n, sg, ssph, sq, ns, tol, 1, xq, 0);
    const int code = R.flags & 15;
    if (code == CODE_SAMPLE || code == CODE_INVALID) {
      value[t] = R.value;
      argmin[t] = R.argmin;
      flags[t] = R.flags;
      continue;
    }
    int sig = 0;
    classify(p, s, n, tol, xq, &sig);
    /* bounds: nearest opposite tangent distance per sign, far bound, and the
     * deepest containment per sign (for LB_VIOL) */
    double ub[2] = {ORC_INF, ORC_INF}; /* [0]: for a positive value (negative spheres), [1]: negative */
    double far = ORC_INF, lb[2] = {-ORC_INF, -ORC_INF};
    for (int64_t j = 0; j < n; ++j) {
      const double d = sqrt(dist2(xq, p + 3 * j));
      const double r = fabs(s[j]);
      if (d + r < far) far = d + r;
      if (s[j] < 0.0 && d - r < ub[0]) ub[0] = d - r;
      if (s[j] > 0.0 && d - r < ub[1]) ub[1] = d - r;
      if (covers(xq, p + 3 * j, s[j], tol)) {
        if (s[j] > 0.0 && r - d > lb[0]) lb[0] = r - d;
        if (s[j] < 0.0 && r - d > lb[1]) lb[1] = r - d;
      }
    }
    /* (V2) per sphere, the farthest survivor's squared distance; the two
     * smallest over spheres with survivors */
    for (int64_t j = 0; j < n; ++j) maxd2[j] = -1.0;
    for (int64_t g = 0; g < ns; ++g) {
      const double d2 = dist2(xq, sq + 3 * g);
      if (d2 > maxd2[ssph[g]]) maxd2[ssph[g]] = d2;
    }
    double m1 = ORC_INF, m2 = ORC_INF;
    int64_t j1 = -1;
    for (int64_t j = 0; j < n; ++j) {
      if (maxd2[j] < 0.0) continue;
      if (maxd2[j] < m1) {
        m2 = m1;
        m1 = maxd2[j];
        j1 = j;
      } else if (maxd2[j] < m2) {
        m2 = maxd2[j];
      }
    }
    orc_score best;
    best.cls = -1;
    int have = 0;
    /* one candidate q on sphere i, of type tan (1) or intersection (0);
     * UNCOVERED: whether q keeps out of every other ball, evaluated only for
     * a candidate that would become the best (the result is the same) */
#define TRY_CANDIDATE(QPTR, I, TAN, KEY, UNCOVERED)                                       \
    do {                                                                                  \
      const double* q_ = (QPTR);                                                          \
      const int64_t i_ = (I);                                                             \
      const double r_ = sqrt(dist2(xq, q_));                                              \
      const double dn_ = (xq[0] - q_[0]) * (p[3 * i_] - q_[0]) + (xq[1] - q_[1]) * (p[3 * i_ + 1] - q_[1]) + \
                         (xq[2] - q_[2]) * (p[3 * i_ + 2] - q_[2]);                       \
      for (int sgi = 0; sgi < 2; ++sgi) {                                                 \
        const int sign_ = sgi == 0 ? 1 : -1;                                              \
        if (sig != 0 && sign_ != sig) continue;                                           \
        if (ub[sgi] < r_ - tol) continue;                           /* V1 */              \
        if (r_ > far + tol) continue;                               /* V3 */              \
        if (r_ > tol) {                                             /* V2 */              \
          const double rt_ = r_ - tol;                                                    \
          const double eff_ = (i_ == j1) ? m2 : m1;                                       \
          if (eff_ < rt_ * rt_) continue;                                                 \
        }                                                                                 \
        const int agree_ = (double)(sign_ * sgn(s[i_])) * dn_ > 0.0;                     \
        orc_score c_;                                                                     \
        c_.cls = (TAN) ? (agree_ ? 3 : 0) : (agree_ ? 2 : 1);                             \
        c_.sr = sign_ > 0 ? r_ : 2.0 * r_;                                                \
        c_.key = (KEY);                                                                   \
        c_.sign = sign_;                                                                  \
        c_.r = r_;                                                                        \
        if ((!have || score_better(&c_, &best)) && (UNCOVERED)) {                         \
          best = c_;                                                                      \
          have = 1;                                                                       \
        }                                                                                 \
      }                                                                                   \
    } while (0)
    for (int64_t g = 0; g < ns; ++g) TRY_CANDIDATE(sq + 3 * g, ssph[g], 0, sg[g], 1);
    for (int64_t j = 0; j < n; ++j) {
      const double r = fabs(s[j]);
      if (!(r > 0.0)) continue;
      const double* pj = p + 3 * j;
      double v[3] = {xq[0] - pj[0], xq[1] - pj[1], xq[2] - pj[2]};
      const double dv = norm3(v);
      if (!(dv > 0.0)) continue;
      for (int side = 0; side < 2; ++side) {
        const double sgnr = side == 0 ? r : -r;
        double tp[3];
        for (int c = 0; c < 3; ++c) tp[c] = pj[c] + sgnr * (v[c] / dv);
        if (box_cull && !inbox(tp)) continue;
        TRY_CANDIDATE(tp, j, 1, SCORE_TKEY + 2 * j + side, !covered_by_other(p, s, n, tol, tp, j));
      }
    }
#undef TRY_CANDIDATE
    if (!have) {
      value[t] = R.value;
      argmin[t] = R.argmin;
      flags[t] = R.flags | FLAG_SCORE_FALLBACK;
      continue;
    }
    const int tan = best.key >= SCORE_TKEY;
    value[t] = best.sign * best.r;
    argmin[t] = tan ? best.key - SCORE_TKEY : best.key;
    int fl = tan ? CODE_TANGENT : CODE_SURVIVOR;
    const double lbv = lb[best.sign > 0 ? 0 : 1];
    if (best.r < lbv - tol) fl |= FLAG_LB_VIOL;
    flags[t] = fl;
  }
  free(maxd2);
}

/* Lazy variant for single queries on large inputs: the same result as
 * orc_query on the full survivor list, with keep decisions evaluated only for
 * candidates that could be the nearest.  It uses two facts:
 *  - a candidate nearer to x than LB - tol is covered (LB = r_j - |x - p_j|
 *    for the sphere j that attains it: |q - p_j| <= |q - x| + |x - p_j| <
 *    r_j - tol; a candidate of sphere j itself is never that near);
 *  - any point of sphere i is at least | |x - p_i| - r_i | away from x.
 * Candidates in the shell LB - tol <= |x - q| <= R are collected, sorted by
 * (distance^2, id), and keep-tested in that order; the first kept one is the
 * nearest survivor.  R starts just above LB and grows until a survivor is
 * found, R passes UB_opp (the value is then the opposite tangent point), or R
 * passes every candidate.  Margins of 1e-9 relative keep rounding on the
 * safe side.  The gap output is not computed here (NaN). */
typedef struct { double d2; int64_t g; } orc_cd;
static int cmp_cd(const void* a, const void* b) {
  const orc_cd* x = (const orc_cd*)a;
  const orc_cd* y = (const orc_cd*)b;
  if (x->d2 < y->d2) return -1;
  if (x->d2 > y->d2) return 1;
  return x->g < y->g ? -1 : (x->g > y->g);
}

void orc_query_lazy(const double* p, const double* s, int64_t n, const double* U, int K, double tol, int box_cull,
                    int clamp_opp, const double* x, int64_t m, double* value, int64_t* argmin, int32_t* flags,
                    double* gap) {
  size_t cap = 1 << 16;
  orc_cd* buf = (orc_cd*)malloc(sizeof(orc_cd) * cap);
  double* lbs = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int64_t t = 0; t < m; ++t) {
    const double* xq = x + 3 * t;
    orc_result R;
    int64_t si = sample_index(p, n, xq);
    int sigma = 0, code = -1;
    if (si >= 0) {
      R.value = s[si];
      R.argmin = si;
      R.flags = CODE_SAMPLE;
    } else if ((code = classify(p, s, n, tol, xq, &sigma)) >= 0) {
      R.value = code == CODE_OUTSIDE ? 0.0 : (0.0 / 0.0);
      R.argmin = -1;
      R.flags = code;
    } else {
      double lbv = -ORC_INF, ub = ORC_INF, dmax = 0;
      int64_t lbj = -1;
      for (int64_t j = 0; j < n; ++j) {
        double d = sqrt(dist2(xq, p + 3 * j)), r = fabs(s[j]);
        int c = sgn(s[j]);
        if (c == sigma && r - d > lbv) { lbv = r - d; lbj = j; }
        if (c == -sigma && d - r < ub) ub = d - r;
        lbs[j] = fabs(d - r);
        if (d + r > dmax) dmax = d + r;
      }
      double skip = lbv - tol - 1e-9 * (1.0 + fabs(lbv));
      double skip2 = skip > 0 ? skip * skip : -1.0;
      double width = 1e-4 + 1e-3 * fabs(lbv);
      double best = ORC_INF;
      int64_t bestg = -1;
      for (;;) {
        double lim = (lbv > 0 ? lbv : 0) + width;
        int last = 0;
        if (clamp_opp && ub < ORC_INF && lim >= ub) { lim = ub; last = 1; }
        if (lim >= dmax) { lim = dmax; last = 1; }
        double limm = lim * (1.0 + 1e-9) + 1e-12, lim2 = limm * limm;
        size_t nc = 0;
        for (int64_t i = 0; i < n; ++i) {
          int c = sgn(s[i]);
          if ((c != sigma && c != 0) || lbs[i] > limm) continue;
          for (int k = 0; k < K; ++k) {
            double q[3];
            cand_pos(p + 3 * i, s[i], U + 3 * k, q);
            if (box_cull && !inbox(q)) continue;
            double d2 = dist2(xq, q);
            if (d2 > lim2 || (i != lbj && d2 < skip2)) continue;
            if (nc == cap) {
              cap *= 2;
              buf = (orc_cd*)realloc(buf, sizeof(orc_cd) * cap);
            }
            buf[nc].d2 = d2;
            buf[nc].g = i * (int64_t)(K + 1) + k;
            ++nc;
          }
        }
        qsort(buf, nc, sizeof(orc_cd), cmp_cd);
        for (size_t u = 0; u < nc; ++u) {
          int64_t i = buf[u].g / (K + 1);
          int k = (int)(buf[u].g % (K + 1));
          if (orc_keep_one(p, s, n, U, K, tol, box_cull, i, k)) {
            best = buf[u].d2;
            bestg = buf[u].g;
            break;
          }
        }
        if (bestg >= 0 || last) break;
        width *= 8.0;
      }
      R = finish(p, s, n, tol, clamp_opp, xq, sigma, best, bestg, ORC_INF);
    }
    value[t] = R.value;
    argmin[t] = R.argmin;
    flags[t] = R.flags;
    if (gap) gap[t] = 0.0 / 0.0;
  }
  free(buf);
  free(lbs);
}

/* ------------------------------------------------------------------------ */
/* gradient of s*(x) through the argmin (analytic, FP64)                     */
/* ------------------------------------------------------------------------ */
/* SURVIVOR g=(i,k): s = sigma |x - p_i - r_i u_k|, v = (x - q)/|x - q|:
 *   ds/dx = sigma v, ds/dp_i = -sigma v, ds/ds_i = -sigma sign(s_i) (v . u_k).
 * OPPOSITE j: s = sigma (|x - p_j| - r_j), w = (x - p_j)/|x - p_j|:
 *   ds/dx = sigma w, ds/dp_j = -sigma w, ds/ds_j = -sigma sign(s_j).
 * LOWER j: s = sigma (r_j - |x - p_j|): ds/dx = -sigma w, ds/dp_j = sigma w,
 *   ds/ds_j = sigma sign(s_j).
 * TANGENT 2j+side (augmented query): s = sigma |d - e r_j|, d = |x - p_j|,
 *   e = +1 (near) / -1 (far), h = sign(d - e r_j): ds/dx = sigma h w,
 *   ds/dp_j = -sigma h w, ds/ds_j = -sigma e h sign(s_j).
 * SAMPLE i: ds/ds_i = 1.  OUTSIDE / INVALID / zero distance: 0. */
void orc_grad(const double* p, const double* s, int64_t n, const double* U, int K, const double* x, int64_t m,
              const double* value, const int64_t* argmin, const int32_t* flags, const double* gup, double* gx,
              double* gp, double* gs) {
  (void)n;
  for (int64_t t = 0; t < m; ++t) {
    const double* xq = x + 3 * t;
    int code = flags[t] & 15;
    double g = gup[t];
    gx[3 * t] = gx[3 * t + 1] = gx[3 * t + 2] = 0.0;
    double sigma = value[t] > 0 ? 1.0 : (value[t] < 0 ? -1.0 : 0.0);
    if (code == CODE_SAMPLE) {
      gs[argmin[t]] += g;
      continue;
    }
    if (sigma == 0.0) continue;
    if (code == CODE_SURVIVOR) {
      int64_t i = argmin[t] / (K + 1);
      int k = (int)(argmin[t] % (K + 1));
      double q[3];
      cand_pos(p + 3 * i, s[i], U + 3 * k, q);
      double v[3] = {xq[0] - q[0], xq[1] - q[1], xq[2] - q[2]};
      double d = norm3(v);
      if (!(d > 0)) continue;
      v[0] /= d; v[1] /= d; v[2] /= d;
      double si = (double)sgn(s[i]);
      const double* u = U + 3 * k;
      double vu = v[0] * u[0] + v[1] * u[1] + v[2] * u[2];
      for (int c = 0; c < 3; ++c) {
        gx[3 * t + c] = g * sigma * v[c];
        gp[3 * i + c] += -g * sigma * v[c];
      }
      gs[i] += -g * sigma * si * vu;
    } else if (code == CODE_OPPOSITE || code == CODE_LOWER) {
      int64_t j = argmin[t];
      double w[3] = {xq[0] - p[3 * j], xq[1] - p[3 * j + 1], xq[2] - p[3 * j + 2]};
      double d = norm3(w);
      if (!(d > 0)) continue;
      w[0] /= d; w[1] /= d; w[2] /= d;
      double sj = (double)sgn(s[j]);
      double dir = code == CODE_OPPOSITE ? 1.0 : -1.0;
      for (int c = 0; c < 3; ++c) {
        gx[3 * t + c] = g * sigma * dir * w[c];
        gp[3 * j + c] += -g * sigma * dir * w[c];
      }
      gs[j] += -g * sigma * dir * sj;
    } else if (code == CODE_TANGENT) {
      /* value sigma * |x - t|, t = p_j + e r (x - p_j)/|x - p_j| (e = +1 near,
       * -1 far): |x - t| = |d - e r| with d = |x - p_j|, so with
       * w = (x - p_j)/d and h = sign(d - e r) it moves as h w in x, -h w in
       * p_j and -e h in r = |s_j| */
      int64_t j = argmin[t] / 2;
      double e = (argmin[t] % 2) ? -1.0 : 1.0;
      double w[3] = {xq[0] - p[3 * j], xq[1] - p[3 * j + 1], xq[2] - p[3 * j + 2]};
      double d = norm3(w);
      if (!(d > 0)) continue;
      w[0] /= d; w[1] /= d; w[2] /= d;
      double r = fabs(s[j]);
      double h = d - e * r >= 0.0 ? 1.0 : -1.0;
      double sj = (double)sgn(s[j]);
      for (int c = 0; c < 3; ++c) {
        gx[3 * t + c] = g * sigma * h * w[c];
        gp[3 * j + c] += -g * sigma * h * w[c];
      }
      gs[j] += g * sigma * (-e * h) * sj;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* greedy sequential insertion (Sec. 4: each new value is consistent with   */
/* the inputs and every value generated before it)                           */
/* ------------------------------------------------------------------------ */
/* For t = 0..T-1 in the given order:
 *   value_t = query(y_t) against the current spheres and survivors;
 *   if the code is SURVIVOR / OPPOSITE / LOWER the sample (y_t, value_t)
 *   joins as sphere n+t:
 *     - survivors inside its shrunk ball are dropped;
 *     - its K candidates are culled against every current sphere but itself;
 *     - its witness (the point that set the value) becomes candidate K of
 *       the new sphere, culled the same way;
 *     - LOST_WITNESS is raised when a sphere that had a survivor has none.
 * Candidate ids: g = sphere * (K+1) + k.  The state after the loop can be
 * read back with orc_insert_state. */
typedef struct {
  int64_t nsph, cap_sph, ns, cap_s;
  double *p, *s;
  int64_t *g, *sph;
  double* q;
  int64_t* count; /* survivors per sphere */
} orc_state;

static orc_state g_state = {0};

static void st_free(void) {
  free(g_state.p); free(g_state.s); free(g_state.g); free(g_state.sph); free(g_state.q); free(g_state.count);
  memset(&g_state, 0, sizeof(g_state));
}

static void st_push_surv(int64_t g, int64_t sph, const double* q) {
  if (g_state.ns == g_state.cap_s) {
    g_state.cap_s = g_state.cap_s ? 2 * g_state.cap_s : 1024;
    g_state.g = (int64_t*)realloc(g_state.g, sizeof(int64_t) * g_state.cap_s);
    g_state.sph = (int64_t*)realloc(g_state.sph, sizeof(int64_t) * g_state.cap_s);
    g_state.q = (double*)realloc(g_state.q, sizeof(double) * 3 * g_state.cap_s);
  }
  g_state.g[g_state.ns] = g;
  g_state.sph[g_state.ns] = sph;
  memcpy(g_state.q + 3 * g_state.ns, q, sizeof(double) * 3);
  g_state.ns++;
  g_state.count[sph]++;
}

static int uncovered_except(const double* q, int64_t self, double tol) {
  for (int64_t j = 0; j < g_state.nsph; ++j) {
    if (j == self) continue;
    if (covers(q, g_state.p + 3 * j, g_state.s[j], tol)) return 0;
  }
  return 1;
}

int64_t orc_insert(const double* p, const double* s, int64_t n, const double* U, int K, double tol, int box_cull,
                   int clamp_opp, const double* y, const double* known, int64_t T, double* value, int64_t* argmin,
                   int32_t* flags) {
  st_free();
  g_state.cap_sph = n + T;
  g_state.p = (double*)malloc(sizeof(double) * 3 * (g_state.cap_sph + 1));
  g_state.s = (double*)malloc(sizeof(double) * (g_state.cap_sph + 1));
  g_state.count = (int64_t*)calloc((size_t)(g_state.cap_sph + 1), sizeof(int64_t));
  memcpy(g_state.p, p, sizeof(double) * 3 * n);
  memcpy(g_state.s, s, sizeof(double) * n);
  g_state.nsph = n;
  uint8_t* keep = (uint8_t*)malloc((size_t)(n * K > 0 ? n * K : 1));
  orc_keep_all(p, s, n, U, K, tol, box_cull, keep);
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < K; ++k)
      if (keep[i * K + k]) {
        double q[3];
        cand_pos(p + 3 * i, s[i], U + 3 * k, q);
        st_push_surv(i * (int64_t)(K + 1) + k, i, q);
      }
  free(keep);
  int64_t inserted = 0;
  for (int64_t t = 0; t < T; ++t) {
    const double* x = y + 3 * t;
    const int ks = known ? sgn(known[t]) : 0;
    orc_result R = query_one(g_state.p, g_state.s, g_state.nsph, g_state.g, g_state.sph, g_state.q, g_state.ns, tol,
                             clamp_opp, x, ks);
    int code = R.flags & 15;
    /* repair (Sec. 6): a value below the removed sample's own by more than
     * tol is flagged (the inserted ball is smaller than the input's) */
    if (ks && (code == CODE_SURVIVOR || code == CODE_OPPOSITE || code == CODE_LOWER) &&
        fabs(R.value) < fabs(known[t]) - tol)
      R.flags |= FLAG_NONCONSERVATIVE;
    value[t] = R.value;
    argmin[t] = R.argmin;
    flags[t] = R.flags;
    if (!(code == CODE_SURVIVOR || code == CODE_OPPOSITE || code == CODE_LOWER)) continue;
    /* witness point (x itself when no sphere sets the value) */
    double wq[3];
    if (code == CODE_SURVIVOR) {
      int64_t at = -1;
      for (int64_t u = 0; u < g_state.ns; ++u)
        if (g_state.g[u] == R.argmin) { at = u; break; }
      memcpy(wq, g_state.q + 3 * at, sizeof(wq));
    } else if (R.argmin < 0) {
      memcpy(wq, x, sizeof(wq));
    } else {
      const double* pj = g_state.p + 3 * R.argmin;
      double rj = fabs(g_state.s[R.argmin]);
      double w[3] = {x[0] - pj[0], x[1] - pj[1], x[2] - pj[2]};
      double d = norm3(w);
      for (int c = 0; c < 3; ++c) wq[c] = pj[c] + rj * (w[c] / d);
    }
    int64_t j = g_state.nsph++;
    memcpy(g_state.p + 3 * j, x, sizeof(double) * 3);
    g_state.s[j] = R.value;
    ++inserted;
    /* drop survivors covered by the new ball */
    int lost = 0;
    int64_t w = 0;
    for (int64_t u = 0; u < g_state.ns; ++u) {
      if (covers(g_state.q + 3 * u, x, R.value, tol)) {
        int64_t o = g_state.sph[u];
        if (--g_state.count[o] == 0) lost = 1;
        continue;
      }
      g_state.g[w] = g_state.g[u];
      g_state.sph[w] = g_state.sph[u];
      memcpy(g_state.q + 3 * w, g_state.q + 3 * u, sizeof(double) * 3);
      ++w;
    }
    g_state.ns = w;
    if (lost) flags[t] |= FLAG_LOST_WITNESS;
    /* the new sphere's candidates and its witness */
    for (int k = 0; k <= K; ++k) {
      double q[3];
      if (k < K) cand_pos(x, R.value, U + 3 * k, q);
      else memcpy(q, wq, sizeof(q));
      if (box_cull && !inbox(q)) continue;
      if (!uncovered_except(q, j, tol)) continue;
      st_push_surv(j * (int64_t)(K + 1) + k, j, q);
    }
  }
  return inserted;
}

/* read back the state after orc_insert (spheres and survivors) */
int64_t orc_insert_state(double* p_out, double* s_out, int64_t* g_out, int64_t* sph_out, double* q_out,
                         int64_t* nsph_out) {
  if (nsph_out) *nsph_out = g_state.nsph;
  if (p_out) memcpy(p_out, g_state.p, sizeof(double) * 3 * g_state.nsph);
  if (s_out) memcpy(s_out, g_state.s, sizeof(double) * g_state.nsph);
  if (g_out) {
    memcpy(g_out, g_state.g, sizeof(int64_t) * g_state.ns);
    memcpy(sph_out, g_state.sph, sizeof(int64_t) * g_state.ns);
    memcpy(q_out, g_state.q, sizeof(double) * 3 * g_state.ns);
  }
  return g_state.ns;
}

/* ------------------------------------------------------------------------ */
/* exact minimum valid radius (Sec. 6, min_valid_radius_for_known_sign)      */
/* ------------------------------------------------------------------------ */
/* Brute force over the grow-to points of Def. 1 for tiny inputs:
 *  U: the two intersection points of every triple of spheres of sign sigma
 *     (or zero); D: the closest and farthest points to x on the intersection
 *     circle of every pair of such spheres; T: both tangent points of every
 *     sphere (any sign) in the direction of x.  The result is the distance to
 *     the nearest of these points that is uncovered (and inside the domain
 *     box when box_cull).  A circle's projections are only kept when
 *     uncovered, which is the "partially uncovered circles" policy the paper
 *     uses for repair. */

/* uncovered by every ball except the (up to three) spheres the point was
 * constructed on: a grow-to point lies on those spheres by construction, and
 * with a zero tolerance rounding alone would decide whether they "cover" it */
static int uncovered_but(const double* p, const double* s, int64_t n, double tol, const double* q, int64_t a,
                         int64_t b, int64_t c) {
  for (int64_t j = 0; j < n; ++j) {
    if (j == a || j == b || j == c) continue;
    if (covers(q, p + 3 * j, s[j], tol)) return 0;
  }
  return 1;
}

static void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* intersection points of three spheres (trilateration); returns count */
static int tri_intersect(const double* p1, double r1, const double* p2, double r2, const double* p3, double r3,
                         double* out) {
  double ex[3] = {p2[0] - p1[0], p2[1] - p1[1], p2[2] - p1[2]};
  double d = norm3(ex);
  if (!(d > 1e-12)) return 0;
  for (int c = 0; c < 3; ++c) ex[c] /= d;
  double t13[3] = {p3[0] - p1[0], p3[1] - p1[1], p3[2] - p1[2]};
  double i = dot3(ex, t13);
  double ey[3] = {t13[0] - i * ex[0], t13[1] - i * ex[1], t13[2] - i * ex[2]};
  double ny = norm3(ey);
  if (!(ny > 1e-12)) return 0;
  for (int c = 0; c < 3; ++c) ey[c] /= ny;
  double ez[3];
  cross3(ex, ey, ez);
  double j = dot3(ey, t13);
  double X = (r1 * r1 - r2 * r2 + d * d) / (2 * d);
  double Y = (r1 * r1 - r3 * r3 + i * i + j * j) / (2 * j) - (i / j) * X;
  double z2 = r1 * r1 - X * X - Y * Y;
  if (z2 < 0) return 0;
  double Z = sqrt(z2);
  for (int c = 0; c < 3; ++c) {
    out[c] = p1[c] + X * ex[c] + Y * ey[c] + Z * ez[c];
    out[3 + c] = p1[c] + X * ex[c] + Y * ey[c] - Z * ez[c];
  }
  return 2;
}

/* closest and farthest points to x on the intersection circle of 2 spheres */
static int circle_points(const double* p1, double r1, const double* p2, double r2, const double* x, double* out) {
  double mu[3] = {p2[0] - p1[0], p2[1] - p1[1], p2[2] - p1[2]};
  double d = norm3(mu);
  if (!(d > 1e-12) || d >= r1 + r2 || d <= fabs(r1 - r2)) return 0;
  for (int c = 0; c < 3; ++c) mu[c] /= d;
  double a = (d * d + r1 * r1 - r2 * r2) / (2 * d);
  double rho2 = r1 * r1 - a * a;
  if (!(rho2 > 0)) return 0;
  double rho = sqrt(rho2);
  double zeta[3] = {p1[0] + a * mu[0], p1[1] + a * mu[1], p1[2] + a * mu[2]};
  double v[3] = {x[0] - zeta[0], x[1] - zeta[1], x[2] - zeta[2]};
  double vm = dot3(v, mu);
  double t[3] = {v[0] - vm * mu[0], v[1] - vm * mu[1], v[2] - vm * mu[2]};
  double nt = norm3(t);
  if (!(nt > 1e-12)) { /* x on the axis: every circle point is equidistant */
    double e[3] = {1, 0, 0};
    if (fabs(mu[0]) > 0.9) { e[0] = 0; e[1] = 1; }
    double em = dot3(e, mu);
    for (int c = 0; c < 3; ++c) t[c] = e[c] - em * mu[c];
    nt = norm3(t);
  }
  for (int c = 0; c < 3; ++c) {
    out[c] = zeta[c] + rho * t[c] / nt;
    out[3 + c] = zeta[c] - rho * t[c] / nt;
  }
  return 2;
}

double orc_exact_rmin(const double* p, const double* s, int64_t n, double tol, int box_cull, const double* x,
                      int sigma) {
  double rmin = ORC_INF;
  double pts[6];
#define ORC_TRY(q, a, b, c)                                                     \
  do {                                                                          \
    if ((!box_cull || inbox(q)) && uncovered_but(p, s, n, tol, (q), a, b, c)) { \
      double dd = sqrt(dist2(x, (q)));                                          \
      if (dd < rmin) rmin = dd;                                                 \
    }                                                                           \
  } while (0)
  for (int64_t i = 0; i < n; ++i) {
    if (sigma * sgn(s[i]) < 0) continue;
    for (int64_t j = i + 1; j < n; ++j) {
      if (sigma * sgn(s[j]) < 0) continue;
      for (int64_t k = j + 1; k < n; ++k) {
        if (sigma * sgn(s[k]) < 0) continue;
        if (tri_intersect(p + 3 * i, fabs(s[i]), p + 3 * j, fabs(s[j]), p + 3 * k, fabs(s[k]), pts) == 2) {
          ORC_TRY(pts, i, j, k);
          ORC_TRY(pts + 3, i, j, k);
        }
      }
      if (circle_points(p + 3 * i, fabs(s[i]), p + 3 * j, fabs(s[j]), x, pts) == 2) {
        ORC_TRY(pts, i, j, -1);
        ORC_TRY(pts + 3, i, j, -1);
      }
    }
  }
  for (int64_t i = 0; i < n; ++i) {
    double w[3] = {x[0] - p[3 * i], x[1] - p[3 * i + 1], x[2] - p[3 * i + 2]};
    double d = norm3(w);
    if (!(d > 0)) continue;
    double r = fabs(s[i]);
    for (int c = -1; c <= 1; c += 2) {
      double q[3] = {p[3 * i] + c * r * w[0] / d, p[3 * i + 1] + c * r * w[1] / d, p[3 * i + 2] + c * r * w[2] / d};
      ORC_TRY(q, i, -1, -1);
    }
  }
#undef ORC_TRY
  return rmin;
}

/* ------------------------------------------------------------------------ */
/* refinement order (Sec. 4.2): covered area ratio of grid cells             */
/* ------------------------------------------------------------------------ */
/* Each cell c (integer coordinates i, j, k in cells[3c..3c+2]) is sampled at
 * sub^3 regularly spaced points, the centres of a sub x sub x sub split of
 * the cell: coordinate origin + h * (i + (a + 1/2) / sub), a < sub, each
 * operation rounded on its own in that order.  counts[c] = number of these
 * points inside some ball, of either sign, shrunk by tol (the cull's
 * coverage predicate).  The covered area ratio is counts[c] / sub^3. */
void orc_cell_coverage(const double* p, const double* s, int64_t n, double tol, const int32_t* cells,
                       int64_t ncells, const double* origin, double h, int sub, uint32_t* counts) {
  for (int64_t c = 0; c < ncells; ++c) {
    uint32_t cnt = 0;
    for (int a = 0; a < sub; ++a)
      for (int b = 0; b < sub; ++b)
        for (int e = 0; e < sub; ++e) {
          const int idx[3] = {a, b, e};
          double x[3];
          for (int d = 0; d < 3; ++d)
            x[d] = origin[d] + h * ((double)cells[3 * c + d] + ((double)idx[d] + 0.5) / (double)sub);
          for (int64_t j = 0; j < n; ++j)
            if (covers(x, p + 3 * j, s[j], tol)) {
              ++cnt;
              break;
            }
        }
    counts[c] = cnt;
  }
}

/* Lazy variant of orc_query_aug for single points on large inputs: the same
 * result, with the plain part from orc_query_lazy and the tangent part
 * restricted to the points that can matter:
 *  - a tangent point only changes the result when it is nearer than the
 *    plain result's candidate (squared distance below the survivor's;
 *    distance at most UB_opp for an OPPOSITE result; anything for LOWER);
 *  - a point nearer to x than LB - tol (LB = r_j - |x - p_j| for the sphere
 *    j of x's class that attains it) lies in j's shrunk ball, so it is
 *    covered (the fact orc_query_lazy uses for candidates); j's own points
 *    are kept regardless.
 * The rest are sorted by (squared distance, id) and coverage-tested in that
 * order; the first uncovered one is the nearest kept tangent point. */
void orc_query_aug_lazy(const double* p, const double* s, int64_t n, const double* U, int K, double tol,
                        int box_cull, int clamp_opp, const double* x, int64_t m, double* value, int64_t* argmin,
                        int32_t* flags) {
  size_t cap = 1 << 12;
  orc_cd* buf = (orc_cd*)malloc(sizeof(orc_cd) * cap);
  for (int64_t t = 0; t < m; ++t) {
    const double* xq = x + 3 * t;
    double v0;
    int64_t a0;
    int32_t f0;
    orc_query_lazy(p, s, n, U, K, tol, box_cull, clamp_opp, xq, 1, &v0, &a0, &f0, NULL);
    value[t] = v0;
    argmin[t] = a0;
    flags[t] = f0;
    const int code = f0 & 15;
    if (code != CODE_SURVIVOR && code != CODE_OPPOSITE && code != CODE_LOWER) continue;
    int sig = 0;
    classify(p, s, n, tol, xq, &sig);
    double lbv = -ORC_INF, ub = ORC_INF;
    int64_t lbj = -1;
    for (int64_t j = 0; j < n; ++j) {
      double d = sqrt(dist2(xq, p + 3 * j)), r = fabs(s[j]);
      int c = sgn(s[j]);
      if (c == sig && r - d > lbv) { lbv = r - d; lbj = j; }
      if (c == -sig && d - r < ub) ub = d - r;
    }
    double sbest = ORC_INF;
    if (code == CODE_SURVIVOR) {
      double q[3];
      cand_pos(p + 3 * (a0 / (K + 1)), s[a0 / (K + 1)], U + 3 * (a0 % (K + 1)), q);
      sbest = dist2(xq, q);
    }
    const double skip = lbv - tol - 1e-9 * (1.0 + fabs(lbv));
    size_t nc = 0;
    for (int64_t j = 0; j < n; ++j) {
      if (sgn(s[j]) != sig) continue;
      const double r = fabs(s[j]);
      const double* pj = p + 3 * j;
      double v[3] = {xq[0] - pj[0], xq[1] - pj[1], xq[2] - pj[2]};
      const double dv = norm3(v);
      if (!(dv > 0.0)) continue;
      for (int side = 0; side < 2; ++side) {
        const double sgnr = side == 0 ? r : -r;
        double tp[3];
        for (int c = 0; c < 3; ++c) tp[c] = pj[c] + sgnr * (v[c] / dv);
        if (box_cull && !inbox(tp)) continue;
        const double d2 = dist2(xq, tp);
        if (code == CODE_SURVIVOR && !(d2 < sbest)) continue;
        if (code == CODE_OPPOSITE && !(sqrt(d2) <= ub)) continue;
        if (j != lbj && skip > 0 && sqrt(d2) < skip) continue;
        if (nc == cap) {
          cap *= 2;
          buf = (orc_cd*)realloc(buf, sizeof(orc_cd) * cap);
        }
        buf[nc].d2 = d2;
        buf[nc].g = 2 * j + side;
        ++nc;
      }
    }
    qsort(buf, nc, sizeof(orc_cd), cmp_cd);
    for (size_t u = 0; u < nc; ++u) {
      const int64_t j = buf[u].g / 2;
      const double r = fabs(s[j]);
      const double* pj = p + 3 * j;
      double v[3] = {xq[0] - pj[0], xq[1] - pj[1], xq[2] - pj[2]};
      const double dv = norm3(v);
      const double sgnr = buf[u].g % 2 == 0 ? r : -r;
      double tp[3];
      for (int c = 0; c < 3; ++c) tp[c] = pj[c] + sgnr * (v[c] / dv);
      int cov = 0;
      for (int64_t k = 0; k < n && !cov; ++k)
        if (k != j && covers(tp, p + 3 * k, s[k], tol)) cov = 1;
      if (cov) continue;
      orc_result T = finish(p, s, n, tol, clamp_opp, xq, sig, buf[u].d2, 0, ORC_INF);
      if ((T.flags & 15) == CODE_SURVIVOR) {
        T.flags = (T.flags & ~15) | CODE_TANGENT;
        T.argmin = buf[u].g;
      }
      value[t] = T.value;
      argmin[t] = T.argmin;
      flags[t] = T.flags;
      break;
    }
  }
  free(buf);
}

/* ------------------------------------------------------------------------ */
/* exact uncovered test per sphere (Prop. 1 (ii); the U and D points of      */
/* Def. 1 on each sphere)                                                   */
/* ------------------------------------------------------------------------ */
/* out[i] = 1 when some point of sphere i lies in no other ball shrunk by tol
 * (for |s_i| = 0: when p_i does).  Let N_i be the spheres k != i with
 * rho_k = |s_k| - tol > 0 whose shrunk open ball meets sphere i,
 * | |p_i - p_k| - |s_i| | < rho_k.  With N_i empty the sphere is uncovered.
 * Otherwise the uncovered set U of sphere i, if not empty, is a closed proper
 * subset of the sphere, so it has a boundary point, on some circle
 * C_k = S_i with the sphere (p_k, rho_k); on C_k, U is either the whole
 * circle or closed arcs whose ends lie on a third sphere (p_m, rho_m).  So it
 * suffices to test, against every ball but i and the spheres they were
 * built from: two points of every circle C_k (its points nearest and
 * farthest from a fixed reference point) and the two points shared by
 * sphere i and the spheres (p_k, rho_k), (p_m, rho_m) for every pair k < m
 * in N_i. */
static int in_list_meets(const double* p, const double* s, int64_t i, int64_t k, double tol) {
  const double rho = fabs(s[k]) - tol;
  if (!(rho > 0.0)) return 0;
  const double d = sqrt(dist2(p + 3 * i, p + 3 * k));
  return fabs(d - fabs(s[i])) < rho;
}

void orc_sphere_uncovered(const double* p, const double* s, int64_t n, double tol, uint8_t* out) {
  const double e_ref[3] = {0.36, 0.48, 0.8};
  int64_t* N = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) {
    const double* pi = p + 3 * i;
    const double ri = fabs(s[i]);
    if (ri == 0.0) {
      out[i] = (uint8_t)uncovered_but(p, s, n, tol, pi, i, -1, -1);
      continue;
    }
    int64_t nn = 0;
    for (int64_t k = 0; k < n; ++k)
      if (k != i && in_list_meets(p, s, i, k, tol)) N[nn++] = k;
    if (nn == 0) {
      out[i] = 1;
      continue;
    }
    int found = 0;
    double ref[3];
    for (int c = 0; c < 3; ++c) ref[c] = pi[c] + (ri + 1.0) * e_ref[c];
    for (int64_t a = 0; a < nn && !found; ++a) {
      const int64_t k = N[a];
      double pts[6];
      if (circle_points(pi, ri, p + 3 * N[a], fabs(s[k]) - tol, ref, pts) == 2)
        found = uncovered_but(p, s, n, tol, pts, i, k, -1) || uncovered_but(p, s, n, tol, pts + 3, i, k, -1);
      for (int64_t b = a + 1; b < nn && !found; ++b) {
        const int64_t m = N[b];
        if (tri_intersect(pi, ri, p + 3 * k, fabs(s[k]) - tol, p + 3 * m, fabs(s[m]) - tol, pts) == 2)
          found = uncovered_but(p, s, n, tol, pts, i, k, m) || uncovered_but(p, s, n, tol, pts + 3, i, k, m);
      }
    }
    out[i] = (uint8_t)found;
  }
  free(N);
}

/* ------------------------------------------------------------------------ */
/* uncovered intersection circles and points (Def. 1 U and the circles of D; */
/* the U and D precomputation of Sec. 4.1)                                  */
/* ------------------------------------------------------------------------ */
/* Over the spheres S_i = (p_i, |s_i|) with |s_i| > 0:
 *  circles: the pairs i < j whose spheres cut in a circle C_ij (the
 *    construction of circle_points) that has a point in no ball but i and j
 *    shrunk by tol.  The uncovered part of C_ij is closed; if it is not
 *    empty and not the whole circle, its ends lie where C_ij crosses some
 *    sphere (p_m, |s_m| - tol), m != i, j.  So the test points are the two
 *    points of C_ij nearest to and farthest from p_i + (|s_i| + 1) e,
 *    e = (0.36, 0.48, 0.8), and, for every m with |s_m| - tol > 0, the two
 *    points shared by S_i, S_j and the sphere (p_m, |s_m| - tol), each tested
 *    against every ball but i, j and the m it was built from.
 *  points (U): for every triple i < j < m, the two points shared by S_i, S_j
 *    and S_m (the trilateration's order: side 0, side 1) that lie in no ball
 *    but i, j, m shrunk by tol.
 * Outputs in lexicographic order: circles as (i, j) pairs, points as
 * (i, j, m, side) quadruples with their coordinates.  Returns the number of
 * circles; *n_points receives the number of points; entries past the
 * capacities are counted, not written. */
int64_t orc_uncovered_intersections(const double* p, const double* s, int64_t n, double tol, int64_t* circles,
                                    int64_t cap_circles, int64_t* quads, double* pts, int64_t cap_points,
                                    int64_t* n_points) {
  const double e_ref[3] = {0.36, 0.48, 0.8};
  int64_t nc = 0, np = 0;
  for (int64_t i = 0; i < n; ++i) {
    const double ri = fabs(s[i]);
    if (!(ri > 0.0)) continue;
    const double* pi = p + 3 * i;
    double ref[3];
    for (int c = 0; c < 3; ++c) ref[c] = pi[c] + (ri + 1.0) * e_ref[c];
    for (int64_t j = i + 1; j < n; ++j) {
      const double rj = fabs(s[j]);
      if (!(rj > 0.0)) continue;
      const double* pj = p + 3 * j;
      double q[6];
      if (circle_points(pi, ri, pj, rj, ref, q) != 2) continue;
      int found = uncovered_but(p, s, n, tol, q, i, j, -1) || uncovered_but(p, s, n, tol, q + 3, i, j, -1);
      for (int64_t m = 0; m < n && !found; ++m) {
        if (m == i || m == j) continue;
        const double rho = fabs(s[m]) - tol;
        if (!(rho > 0.0)) continue;
        if (tri_intersect(pi, ri, pj, rj, p + 3 * m, rho, q) == 2)
          found = uncovered_but(p, s, n, tol, q, i, j, m) || uncovered_but(p, s, n, tol, q + 3, i, j, m);
      }
      if (found) {
        if (nc < cap_circles) {
          circles[2 * nc] = i;
          circles[2 * nc + 1] = j;
        }
        ++nc;
      }
      for (int64_t m = j + 1; m < n; ++m) {
        const double rm = fabs(s[m]);
        if (!(rm > 0.0)) continue;
        if (tri_intersect(pi, ri, pj, rj, p + 3 * m, rm, q) != 2) continue;
        for (int side = 0; side < 2; ++side) {
          if (!uncovered_but(p, s, n, tol, q + 3 * side, i, j, m)) continue;
          if (np < cap_points) {
            quads[4 * np] = i;
            quads[4 * np + 1] = j;
            quads[4 * np + 2] = m;
            quads[4 * np + 3] = side;
            for (int c = 0; c < 3; ++c) pts[3 * np + c] = q[3 * side + c];
          }
          ++np;
        }
      }
    }
  }
  *n_points = np;
  return nc;
}

/* ------------------------------------------------------------------------ */
/* the point that sets each value (q* of the query)                          */
/* ------------------------------------------------------------------------ */
/* From a query's argmin and code: SURVIVOR g = (i, k): the candidate
 * p_i + |s_i| u_k; OPPOSITE and LOWER j: the near tangent point
 * p_j + |s_j| (x - p_j)/|x - p_j| (for OPPOSITE the point of the opposite
 * sphere nearest to x, for LOWER the point where x's deepest containing ball
 * is nearest to x); TANGENT 2j + side: that tangent point (side 1: far);
 * OUTSIDE, and LOWER with no sphere (argmin -1): x itself (value 0);
 * SAMPLE and INVALID: NaN (no point defines the value).  Where x = p_j the
 * direction is undefined: NaN.  Same expressions, in the same order, as the
 * candidates and the tangent points of the queries. */
void orc_argmin_points(const double* p, const double* s, const double* U, int K, const double* x, int64_t m,
                       const int64_t* argmin, const int32_t* flags, double* out) {
  const double nan = 0.0 / 0.0;
  for (int64_t t = 0; t < m; ++t) {
    const double* xq = x + 3 * t;
    double* o = out + 3 * t;
    const int code = flags[t] & 15;
    const int64_t a = argmin[t];
    o[0] = o[1] = o[2] = nan;
    if (code == CODE_SURVIVOR) {
      cand_pos(p + 3 * (a / (K + 1)), s[a / (K + 1)], U + 3 * (a % (K + 1)), o);
    } else if (code == CODE_OUTSIDE || ((code == CODE_LOWER || code == CODE_OPPOSITE) && a < 0)) {
      o[0] = xq[0];
      o[1] = xq[1];
      o[2] = xq[2];
    } else if (code == CODE_OPPOSITE || code == CODE_LOWER || code == CODE_TANGENT) {
      const int64_t j = code == CODE_TANGENT ? a / 2 : a;
      const double r = fabs(s[j]);
      const double sgnr = (code == CODE_TANGENT && a % 2 == 1) ? -r : r;
      const double* pj = p + 3 * j;
      double v[3] = {xq[0] - pj[0], xq[1] - pj[1], xq[2] - pj[2]};
      const double dv = norm3(v);
      if (dv > 0.0)
        for (int c = 0; c < 3; ++c) o[c] = pj[c] + sgnr * (v[c] / dv);
    }
  }
}
