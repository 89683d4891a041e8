"""ctypes front end of the FP64 CPU oracle (``gfs_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the package's smoke
check and by the benchmark's CPU-baseline leg.  The CUDA library never
imports, links or executes anything here, and nothing here calls the library.

Every function takes and returns numpy arrays in FP64 (positions (n,3)
row-major, values (n,)).  Candidate ids are ``g = i * (K + 1) + k``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gfs_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libgfs_oracle.so")

TOL = 1e-6  # App. B: "all other tolerances are 1e-6"

CODE_SURVIVOR, CODE_OPPOSITE, CODE_SAMPLE, CODE_OUTSIDE, CODE_INVALID, CODE_LOWER, CODE_TANGENT = range(7)
FLAG_LB_VIOL, FLAG_FAR_VIOL, FLAG_OPP_VIOL, FLAG_LOST_WITNESS = 16, 32, 64, 128
FLAG_NONCONSERVATIVE = 256
FLAG_SCORE_FALLBACK = 512


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off) and return the path."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.orc_icosphere.argtypes = [i32, P, i64]
        L.orc_icosphere.restype = i32
        L.orc_keep_one.argtypes = [P, P, i64, P, i32, f64, i32, i64, i32]
        L.orc_keep_one.restype = i32
        L.orc_keep_all.argtypes = [P, P, i64, P, i32, f64, i32, P]
        L.orc_keep_all.restype = None
        L.orc_collect.argtypes = [P, P, i64, P, i32, P, P, P, P]
        L.orc_collect.restype = i64
        L.orc_query.argtypes = [P, P, i64, P, P, P, i64, f64, i32, P, i64, P, P, P, P]
        L.orc_query_aug.argtypes = [P, P, i64, P, P, P, i64, f64, i32, i32, P, i64, P, P, P]
        L.orc_query_scored.argtypes = [P, P, i64, P, P, P, i64, f64, i32, P, i64, P, P, P]
        L.orc_query_scored.restype = None
        L.orc_query.restype = None
        L.orc_query_lazy.argtypes = [P, P, i64, P, i32, f64, i32, i32, P, i64, P, P, P, P]
        L.orc_query_lazy.restype = None
        L.orc_grad.argtypes = [P, P, i64, P, i32, P, i64, P, P, P, P, P, P, P]
        L.orc_grad.restype = None
        L.orc_insert.argtypes = [P, P, i64, P, i32, f64, i32, i32, P, P, i64, P, P, P]
        L.orc_insert.restype = i64
        L.orc_insert_state.argtypes = [P, P, P, P, P, P]
        L.orc_insert_state.restype = i64
        L.orc_exact_rmin.argtypes = [P, P, i64, f64, i32, P, i32]
        L.orc_exact_rmin.restype = f64
        L.orc_query_aug_lazy.argtypes = [P, P, i64, P, i32, f64, i32, i32, P, i64, P, P, P]
        L.orc_query_aug_lazy.restype = None
        L.orc_argmin_points.argtypes = [P, P, P, i32, P, i64, P, P, P]
        L.orc_argmin_points.restype = None
        L.orc_sphere_uncovered.argtypes = [P, P, i64, f64, P]
        L.orc_sphere_uncovered.restype = None
        L.orc_uncovered_intersections.argtypes = [P, P, i64, f64, P, i64, P, P, i64, P]
        L.orc_uncovered_intersections.restype = i64
        L.orc_cell_coverage.argtypes = [P, P, i64, f64, P, i64, P, f64, i32, P]
        L.orc_cell_coverage.restype = None
        _lib = L
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None and a.size else None


def icosphere(tau: int) -> np.ndarray:
    K = 10 * 4 ** tau + 2
    out = np.zeros((K, 3), dtype=np.float64)
    k = lib().orc_icosphere(tau, _ptr(out), K)
    if k != K:
        raise ValueError(f"icosphere construction failed for tau={tau}")
    return out


def keep_one(p, s, U, i, k, tol=TOL, box_cull=True) -> bool:
    p, s, U = _c(p, np.float64), _c(s, np.float64), _c(U, np.float64)
    return bool(lib().orc_keep_one(_ptr(p), _ptr(s), s.shape[0], _ptr(U), U.shape[0], tol, int(box_cull), i, k))


def keep_all(p, s, U, tol=TOL, box_cull=True) -> np.ndarray:
    """(n, K) uint8 keep mask of every candidate (brute force, O(n^2 K))."""
    p, s, U = _c(p, np.float64), _c(s, np.float64), _c(U, np.float64)
    n, K = s.shape[0], U.shape[0]
    keep = np.zeros((n, K), dtype=np.uint8)
    if n:
        lib().orc_keep_all(_ptr(p), _ptr(s), n, _ptr(U), K, tol, int(box_cull), _ptr(keep))
    return keep


def collect(p, s, U, keep):
    """Survivor list (g, sphere, q) in ascending g from a keep mask."""
    p, s, U, keep = _c(p, np.float64), _c(s, np.float64), _c(U, np.float64), _c(keep, np.uint8)
    n, K = s.shape[0], U.shape[0]
    c = int(keep.sum())
    g = np.zeros(c, np.int64)
    sph = np.zeros(c, np.int64)
    q = np.zeros((c, 3), np.float64)
    if c:
        lib().orc_collect(_ptr(p), _ptr(s), n, _ptr(U), K, _ptr(keep), _ptr(g), _ptr(sph), _ptr(q))
    return g, sph, q


def query(p, s, surv, x, tol=TOL, clamp_opp=True):
    """Brute-force consistent value at every row of x against the survivor
    list ``surv = (g, sphere, q)``.  Returns (value, argmin, flags, gap)."""
    p, s, x = _c(p, np.float64), _c(s, np.float64), _c(x, np.float64)
    g, sph, q = (_c(surv[0], np.int64), _c(surv[1], np.int64), _c(surv[2], np.float64))
    m = x.shape[0]
    val = np.zeros(m, np.float64)
    arg = np.zeros(m, np.int64)
    fl = np.zeros(m, np.int32)
    gap = np.zeros(m, np.float64)
    if m:
        lib().orc_query(_ptr(p), _ptr(s), s.shape[0], _ptr(g), _ptr(sph), _ptr(q), g.shape[0], tol,
                        int(clamp_opp), _ptr(x), m, _ptr(val), _ptr(arg), _ptr(fl), _ptr(gap))
    return val, arg, fl, gap


def query_aug(p, s, surv, x, tol=TOL, clamp_opp=True, box_cull=True):
    """As ``query``, with the candidate set augmented by the uncovered near
    and far tangent points of the spheres of x's own sign (code TANGENT,
    argmin 2j + side).  Returns (value, argmin, flags)."""
    p, s, x = _c(p, np.float64), _c(s, np.float64), _c(x, np.float64)
    g, sph, q = (_c(surv[0], np.int64), _c(surv[1], np.int64), _c(surv[2], np.float64))
    m = x.shape[0]
    val = np.zeros(m, np.float64)
    arg = np.zeros(m, np.int64)
    fl = np.zeros(m, np.int32)
    if m:
        lib().orc_query_aug(_ptr(p), _ptr(s), s.shape[0], _ptr(g), _ptr(sph), _ptr(q), g.shape[0], tol,
                            int(clamp_opp), int(box_cull), _ptr(x), m, _ptr(val), _ptr(arg), _ptr(fl))
    return val, arg, fl


def query_scored(p, s, surv, x, tol=TOL, box_cull=True):
    """Sec. 3.3 scored value at every row of x against the survivor list
    ``surv = (g, sphere, q)``: the best-scoring valid grow-to radius over the
    survivors and the uncovered tangent points (codes SURVIVOR / TANGENT),
    SAMPLE / INVALID as in ``query``, and the plain query's result with
    FLAG_SCORE_FALLBACK where no candidate is valid.  Returns (value,
    argmin, flags)."""
    p, s, x = _c(p, np.float64), _c(s, np.float64), _c(x, np.float64)
    g, sph, q = (_c(surv[0], np.int64), _c(surv[1], np.int64), _c(surv[2], np.float64))
    m = x.shape[0]
    val = np.zeros(m, np.float64)
    arg = np.zeros(m, np.int64)
    fl = np.zeros(m, np.int32)
    if m:
        lib().orc_query_scored(_ptr(p), _ptr(s), s.shape[0], _ptr(g), _ptr(sph), _ptr(q), g.shape[0], tol,
                               int(box_cull), _ptr(x), m, _ptr(val), _ptr(arg), _ptr(fl))
    return val, arg, fl


def query_aug_lazy(p, s, U, x, tol=TOL, box_cull=True, clamp_opp=True):
    """Same result as ``query_aug`` on the full survivor list, for a few
    points on large inputs (tangent points coverage-tested only where they
    can change the result).  Returns (value, argmin, flags)."""
    p, s, U, x = _c(p, np.float64), _c(s, np.float64), _c(U, np.float64), _c(x, np.float64)
    m = x.shape[0]
    val = np.zeros(m, np.float64)
    arg = np.zeros(m, np.int64)
    fl = np.zeros(m, np.int32)
    if m:
        lib().orc_query_aug_lazy(_ptr(p), _ptr(s), s.shape[0], _ptr(U), U.shape[0], tol, int(box_cull),
                                 int(clamp_opp), _ptr(x), m, _ptr(val), _ptr(arg), _ptr(fl))
    return val, arg, fl


def query_lazy(p, s, U, x, tol=TOL, box_cull=True, clamp_opp=True):
    """Same result as ``query`` on the full survivor list, computing keep
    decisions only for candidates that could be nearest (large inputs)."""
    p, s, U, x = _c(p, np.float64), _c(s, np.float64), _c(U, np.float64), _c(x, np.float64)
    m = x.shape[0]
    val = np.zeros(m, np.float64)
    arg = np.zeros(m, np.int64)
    fl = np.zeros(m, np.int32)
    gap = np.zeros(m, np.float64)
    if m:
        lib().orc_query_lazy(_ptr(p), _ptr(s), s.shape[0], _ptr(U), U.shape[0], tol, int(box_cull),
                             int(clamp_opp), _ptr(x), m, _ptr(val), _ptr(arg), _ptr(fl), _ptr(gap))
    return val, arg, fl, gap


def grad(p, s, U, x, value, argmin, flags, gup):
    """Analytic gradient through the argmin: (grad_x (m,3), grad_p (n,3),
    grad_s (n,)) for upstream gradient ``gup`` (m,)."""
    p, s, U, x = _c(p, np.float64), _c(s, np.float64), _c(U, np.float64), _c(x, np.float64)
    value, argmin = _c(value, np.float64), _c(argmin, np.int64)
    flags, gup = _c(flags, np.int32), _c(gup, np.float64)
    m, n = x.shape[0], s.shape[0]
    gx = np.zeros((m, 3), np.float64)
    gp = np.zeros((n, 3), np.float64)
    gs = np.zeros(n, np.float64)
    if m:
        lib().orc_grad(_ptr(p), _ptr(s), n, _ptr(U), U.shape[0], _ptr(x), m, _ptr(value), _ptr(argmin),
                       _ptr(flags), _ptr(gup), _ptr(gx), _ptr(gp), _ptr(gs))
    return gx, gp, gs


def insert(p, s, U, y, tol=TOL, box_cull=True, clamp_opp=True, known=None):
    """Sequential greedy insertion of the rows of y.  known (optional, T
    values): the sign of known[t] fixes y_t's sign class (0: inferred from
    containment), and NONCONSERVATIVE marks |value| < |known[t]| - tol (the
    Sec. 6 repair of removed samples).  Returns (value, argmin, flags) per
    insertion and the final state dict."""
    p, s, U, y = _c(p, np.float64), _c(s, np.float64), _c(U, np.float64), _c(y, np.float64)
    T = y.shape[0]
    val = np.zeros(T, np.float64)
    arg = np.zeros(T, np.int64)
    fl = np.zeros(T, np.int32)
    kn = None if known is None else _c(known, np.float64)
    L = lib()
    L.orc_insert(_ptr(p), _ptr(s), s.shape[0], _ptr(U), U.shape[0], tol, int(box_cull), int(clamp_opp),
                 _ptr(y), _ptr(kn) if kn is not None else None, T, _ptr(val), _ptr(arg), _ptr(fl))
    nsph = ctypes.c_int64(0)
    ns = L.orc_insert_state(None, None, None, None, None, ctypes.byref(nsph))
    P = np.zeros((nsph.value, 3))
    S = np.zeros(nsph.value)
    g = np.zeros(ns, np.int64)
    sph = np.zeros(ns, np.int64)
    q = np.zeros((ns, 3))
    L.orc_insert_state(_ptr(P), _ptr(S), _ptr(g) if ns else None, _ptr(sph) if ns else None,
                       _ptr(q) if ns else None, None)
    order = np.argsort(g, kind="stable")
    state = {"p": P, "s": S, "g": g[order], "sph": sph[order], "q": q[order]}
    return val, arg, fl, state


def exact_rmin(p, s, x, sigma, tol=TOL, box_cull=False) -> float:
    """Exact minimum valid radius (T/U/D grow-to points, brute force)."""
    p, s, x = _c(p, np.float64), _c(s, np.float64), _c(x, np.float64)
    return float(lib().orc_exact_rmin(_ptr(p), _ptr(s), s.shape[0], tol, int(box_cull), _ptr(x), int(sigma)))


def solve(p, s, tau, x, tol=TOL, box_cull=True, clamp_opp=True):
    """Whole path on small inputs: icosphere, P build, query."""
    U = icosphere(tau)
    keep = keep_all(p, s, U, tol, box_cull)
    surv = collect(p, s, U, keep)
    return keep, surv, query(p, s, surv, x, tol, clamp_opp)


# ----------------------------------------------------------------------------
# refinement order (Sec. 4.2)
# ----------------------------------------------------------------------------

def cell_coverage(p, s, cells, origin, h, sub=8, tol=TOL):
    """Covered sub-point count of each cell (cells: (c, 3) integer cell
    coordinates; points origin + h * (ijk + (abc + 1/2) / sub)): how many of
    the cell's sub^3 points lie in some ball shrunk by tol."""
    p, s = _c(p, np.float64), _c(s, np.float64)
    cells = _c(cells, np.int32)
    origin = _c(origin, np.float64)
    out = np.zeros(cells.shape[0], np.uint32)
    if cells.shape[0]:
        lib().orc_cell_coverage(_ptr(p), _ptr(s), s.shape[0], tol, _ptr(cells), cells.shape[0], _ptr(origin),
                                float(h), int(sub), _ptr(out))
    return out


NEIGHBOURS = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1) if (a, b, c) != (0, 0, 0)]


def flood_order(cells, counts):
    """Flood-fill refinement order of Sec. 4.2 (reading: priorities are the
    covered counts, lowest first, ties to the lower list index; neighbours
    are the cells of the list that share a face, an edge or a corner).
    Start from the least covered cell; repeatedly pop the least covered
    queued cell, emit it and queue its not yet queued neighbours; when the
    queue runs dry, start again from the least covered cell not yet
    emitted.  Returns the list indices in emission order."""
    import heapq
    cells = [tuple(int(v) for v in c) for c in np.asarray(cells)]
    counts = [int(v) for v in np.asarray(counts)]
    where = {c: i for i, c in enumerate(cells)}
    seeds = sorted(range(len(cells)), key=lambda i: (counts[i], i))
    queued = [False] * len(cells)
    heap, order, nxt = [], [], 0
    while len(order) < len(cells):
        if not heap:
            while queued[seeds[nxt]]:
                nxt += 1
            queued[seeds[nxt]] = True
            heap.append((counts[seeds[nxt]], seeds[nxt]))
        _, i = heapq.heappop(heap)
        order.append(i)
        ci = cells[i]
        for d in NEIGHBOURS:
            j = where.get((ci[0] + d[0], ci[1] + d[1], ci[2] + d[2]))
            if j is not None and not queued[j]:
                queued[j] = True
                heapq.heappush(heap, (counts[j], j))
    return order


def sphere_uncovered(p, s, tol=TOL):
    """Exact uncovered test per sphere (Prop. 1 (ii)): 1 where some point of
    the sphere lies in no other ball shrunk by tol."""
    p, s = _c(p, np.float64), _c(s, np.float64)
    out = np.zeros(s.shape[0], np.uint8)
    if s.shape[0]:
        lib().orc_sphere_uncovered(_ptr(p), _ptr(s), s.shape[0], tol, _ptr(out))
    return out


def uncovered_intersections(p, s, tol=TOL):
    """Sec. 4.1 U and D precomputation (Def. 1): the pairs i < j whose
    intersection circle has a point in no other ball shrunk by tol, (c, 2)
    int64; the uncovered points shared by three spheres, (u, 4) int64
    (i, j, m, side) and (u, 3) float64 positions; lexicographic order."""
    p, s = _c(p, np.float64), _c(s, np.float64)
    cap_c, cap_p = 1024, 1024
    while True:
        circ = np.zeros((cap_c, 2), np.int64)
        quads = np.zeros((cap_p, 4), np.int64)
        pts = np.zeros((cap_p, 3), np.float64)
        npt = ctypes.c_int64(0)
        nc = lib().orc_uncovered_intersections(_ptr(p), _ptr(s), s.shape[0], tol, _ptr(circ), cap_c, _ptr(quads),
                                               _ptr(pts), cap_p, ctypes.byref(npt))
        if nc <= cap_c and npt.value <= cap_p:
            return circ[:nc], quads[:npt.value], pts[:npt.value]
        cap_c, cap_p = max(cap_c, int(nc)), max(cap_p, int(npt.value))


def argmin_points(p, s, U, x, argmin, flags):
    """The point q* that sets each query value (from the argmin and code);
    (m, 3), NaN where no point defines the value (SAMPLE, INVALID)."""
    p, s, U, x = _c(p, np.float64), _c(s, np.float64), _c(U, np.float64), _c(x, np.float64)
    argmin, flags = _c(argmin, np.int64), _c(flags, np.int32)
    out = np.zeros((x.shape[0], 3), np.float64)
    if x.shape[0]:
        lib().orc_argmin_points(_ptr(p), _ptr(s), _ptr(U), U.shape[0], _ptr(x), x.shape[0], _ptr(argmin),
                                _ptr(flags), _ptr(out))
    return out
