"""Device routines compiled as host C++, against the oracle (CPU, no GPU
needed): the tangent pass, the cell coverage count of the refinement order,
the exact uncovered test per sphere and the points q* that set the values.

`csrc/gfs_tangent.cuh` holds the whole per-point logic of gfs_query_tangent:
the FP64 pass over the sphere hierarchy, the tangent-point search with its
pruning and its skip of points covered by the deepest containing ball, and
the coverage walks.  `tests/host_emu/` supplies a stand-in CUDA header and a
hierarchy built on the host with the library's layout (Morton-ordered, or
shuffled so that nodes overlap heavily), and the routines refine the
oracle's plain query results in place.  Every output must equal the oracle's
augmented query bit for bit.  This checks the traversal logic on the CPU;
the GPU tests check the compiled kernel.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2605_01919_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def host(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("needs g++")
    out = str(tmp_path_factory.mktemp("tangent_host") / "tangent_host.so")
    cmd = [cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-I", os.path.join(ROOT, "tests", "host_emu"), "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(ROOT, "paper_2605_01919_gb300", "csrc"),
           os.path.join(ROOT, "tests", "host_emu", "tangent_host.cpp"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    L = ctypes.CDLL(out)
    P = ctypes.c_void_p
    L.tangent_host.argtypes = [P, P, ctypes.c_int64, P, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                               P, ctypes.c_int64, P, P, P, ctypes.c_uint]
    L.tangent_host.restype = ctypes.c_int
    L.coverage_host.argtypes = [P, P, ctypes.c_int64, ctypes.c_double, P, ctypes.c_int64, P, ctypes.c_double,
                                ctypes.c_int, P, ctypes.c_uint]
    L.coverage_host.restype = ctypes.c_int
    L.uncovered_host.argtypes = [P, P, ctypes.c_int64, ctypes.c_double, P, P, ctypes.c_uint]
    L.uncovered_host.restype = ctypes.c_int
    L.intersections_host.argtypes = [P, P, ctypes.c_int64, ctypes.c_double, ctypes.c_int64, P, ctypes.c_int64, P,
                                     P, P, P, ctypes.c_uint]
    L.intersections_host.restype = ctypes.c_int
    L.exact_rmin_host.argtypes = [P, P, ctypes.c_int64, ctypes.c_double, ctypes.c_int, P, P, ctypes.c_int64, P,
                                  ctypes.c_uint]
    L.exact_rmin_host.restype = ctypes.c_int
    L.points_host.argtypes = [P, P, ctypes.c_int64, P, ctypes.c_int, P, ctypes.c_int64, P, P, P]
    L.points_host.restype = ctypes.c_int
    L.scored_host.argtypes = [P, P, ctypes.c_int64, P, ctypes.c_int, ctypes.c_double, ctypes.c_int, P, P, P,
                              ctypes.c_int64, P, ctypes.c_int64, P, P, P, ctypes.c_uint]
    L.scored_host.restype = ctypes.c_int
    return L


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def check(host, orc, p, s, tau, x, box_cull=True, clamp_opp=True, tol=1e-6, orders=(0, 5)):
    p, s, x = (np.ascontiguousarray(a, np.float64) for a in (p, s, x))
    U = orc.icosphere(tau)
    surv = orc.collect(p, s, U, orc.keep_all(p, s, U, tol=tol, box_cull=box_cull))
    v0, a0, f0, _ = orc.query(p, s, surv, x, tol=tol, clamp_opp=clamp_opp)
    v1, a1, f1 = orc.query_aug(p, s, surv, x, tol=tol, clamp_opp=clamp_opp, box_cull=box_cull)
    for order in orders:
        val, arg, fl = v0.copy(), a0.copy(), f0.astype(np.uint16)
        assert host.tangent_host(_ptr(p), _ptr(s), p.shape[0], _ptr(U), U.shape[0], tol, int(clamp_opp),
                                 int(box_cull), _ptr(x), x.shape[0], _ptr(val), _ptr(arg), _ptr(fl), order) == 0
        bad = np.nonzero(~((val == v1) | (np.isnan(val) & np.isnan(v1))) | (arg != a1) |
                         (fl.astype(np.int32) != f1))[0]
        assert bad.size == 0, f"order {order}: {bad.size} points differ, first {bad[:5]}"
    return int(np.sum((f1 & 15) == orc.CODE_TANGENT))


def test_host_sphere_grid(host, orc):
    """10^3 sphere grid, tau = 2, every 19^3 point."""
    w = W.sphere_grid(N=10, up=2, tau=2)
    assert check(host, orc, w.p, w.s, w.tau, w.make_queries()) > 500


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (7, 2), (37, 3), (100, 4), (257, 5)])
def test_host_tiny_random(host, orc, n, seed):
    p, s = W.tiny_random(n, seed, valid=(seed % 3 != 0), spread=0.9)
    rng = np.random.default_rng(1000 + seed)
    x = np.concatenate([rng.uniform(-1, 1, size=(300, 3)), p[: min(n, 20)],
                        rng.uniform(-1.5, 1.5, size=(20, 3))])
    for tau in (0, 1, 3):
        for box_cull, clamp in [(True, True), (False, True), (True, False)]:
            check(host, orc, p, s, tau, x, box_cull, clamp)
    # tol = 0 (touching balls share boundary points)
    check(host, orc, p, s, 1, x, tol=0.0)


def test_host_degenerate(host, orc):
    p = np.array([[0.0, 0, 0], [0.0, 0, 0], [0.5, 0, 0], [0.2, 0.1, 0], [0.2, 0.1, 0.0],
                  [-0.4, 0.3, 0.2], [-0.4, 0.3, 0.2], [0.7, 0.7, 0.7]])
    s = np.array([0.3, 0.3, 0.2, 0.0, 0.05, -0.25, -0.1, 0.5])
    rng = np.random.default_rng(9)
    x = np.concatenate([p, rng.uniform(-1, 1, size=(500, 3)), [[0.3, 0.0, 0.0], [0.25, 0.0, 0.0],
                                                               [-0.219, 0.164, 0.109]]])
    for tau in (1, 2):
        assert check(host, orc, p, s, tau, x) > 0


def test_host_union_grid(host, orc):
    """12^3 union grid, tau = 3: sampled 4x upsampled points and samples."""
    w = W.union_grid(N=12, up=4)
    xq = w.make_queries()
    sel = np.random.default_rng(2).choice(xq.shape[0], 1200, replace=False)
    assert check(host, orc, w.p, w.s, w.tau, np.concatenate([xq[sel], w.p[::11]]), orders=(0,)) > 50


def test_host_torus_fp32_points(host, orc):
    w = W.torus_grid(N=14, m=600)
    assert check(host, orc, w.p, w.s, w.tau, w.make_queries().astype(np.float64), orders=(0,)) > 20


def _coverage(host, p, s, cells, origin, h, sub, tol, order):
    p, s = np.ascontiguousarray(p, np.float64), np.ascontiguousarray(s, np.float64)
    cells = np.ascontiguousarray(cells, np.int32)
    origin = np.ascontiguousarray(origin, np.float64)
    out = np.zeros(cells.shape[0], np.uint32)
    assert host.coverage_host(_ptr(p), _ptr(s), p.shape[0], tol, _ptr(cells), cells.shape[0], _ptr(origin), h, sub,
                              _ptr(out), order) == 0
    return out


@pytest.mark.parametrize("sub", [1, 3, 8])
def test_host_cell_coverage(host, orc, sub):
    """Covered sub-point counts of the surface cells of a 12^3 union grid and
    of random cells, against the oracle's brute force."""
    w = W.union_grid(N=12, up=4)
    N = 12
    S = w.s.reshape(N, N, N)
    near = np.abs(S) < 0.5 * np.sqrt(3) * w.h
    cell = near[:-1, :-1, :-1] | near[1:, 1:, 1:] | near[1:, :-1, :-1] | near[:-1, 1:, 1:]
    cells = np.argwhere(cell).astype(np.int32)
    rng = np.random.default_rng(sub)
    cells = np.concatenate([cells[rng.choice(cells.shape[0], min(150, cells.shape[0]), replace=False)],
                            rng.integers(-2, N + 1, size=(40, 3)).astype(np.int32)])
    origin = np.array([-1.0, -1.0, -1.0])
    want = orc.cell_coverage(w.p, w.s, cells, origin, w.h, sub)
    assert 0 < want.sum() < cells.shape[0] * sub ** 3
    for order in (0, 5):
        got = _coverage(host, w.p, w.s, cells, origin, w.h, sub, 1e-6, order)
        assert np.array_equal(got, want)


def test_host_cell_coverage_lattice_shells(host, orc):
    """The oracle's shell-count pins hold for the device routine too."""
    h = 0.05
    origin = np.array([-1.0, -1.0, -1.0])
    cell = np.array([[2, -1, 3]])
    centre = origin + h * (cell[0] + 0.5)
    for R2, count in [(2.0, 0), (7.0, 8), (15.0, 32), (23.0, 56), (31.0, 88), (150.0, 512)]:
        s = np.array([-h / 16 * np.sqrt(R2)])
        assert _coverage(host, centre[None], s, cell, origin, h, 8, 0.0, 0)[0] == count


def _uncovered(host, p, s, tol, order):
    p, s = np.ascontiguousarray(p, np.float64), np.ascontiguousarray(s, np.float64)
    out = np.zeros(s.shape[0], np.uint8)
    wit = np.full((s.shape[0], 3), np.nan)
    assert host.uncovered_host(_ptr(p), _ptr(s), s.shape[0], tol, _ptr(out), _ptr(wit), order) == 0
    return out, wit


def check_witnesses(p, s, tol, out, wit):
    """Each uncovered sphere's witness lies on the sphere and in no other
    shrunk ball beyond rounding (it is a test point built on up to two other
    spheres, which the test leaves out)."""
    for i in np.nonzero(out == 1)[0]:
        t = wit[i]
        assert abs(np.linalg.norm(t - p[i]) - abs(s[i])) <= 1e-9 * (1 + abs(s[i]))
        d = np.linalg.norm(p - t, axis=1)
        rho = np.abs(s) - tol
        inside = (d < rho - 1e-9) & (rho > 0)
        inside[i] = False
        assert not inside.any(), (i, np.nonzero(inside)[0][:4])


def test_host_sphere_uncovered(host, orc):
    """Octahedral caps around the threshold rho = 0.919401, the 8^3 sphere
    grid inflated by 1.2 (covered spheres), and valid and invalid tiny
    random inputs, for tol = 0 and 1e-6, and grids of exactly touching SDF
    samples (sphere, CSG: a few covered spheres among many that are not)
    for tol = 1e-6: equal to the oracle sphere by sphere, in eight hierarchy
    orders, and every witness valid."""
    e = np.eye(3)
    cases = []
    for rho in (0.91, 0.9194, 0.9195, 0.93):
        cases.append((np.concatenate([np.zeros((1, 3)), e, -e]), np.array([1.0] + [rho] * 6)))
    w = W.sphere_grid(N=8, up=2, tau=2)
    cases.append((w.p, 1.2 * w.s))
    # grids of SDF samples touch exactly: with tol = 0 some spheres keep only
    # tangency points, where rounding decides; compared at the method's tol
    exact_touch = [(w.p, w.s)]
    for N in (6, 8):
        w = W.csg_pseudo_grid(N=N, tau=1)
        exact_touch.append((w.p, w.s))
    for seed in range(4):
        cases.append(W.tiny_random(40, seed, valid=(seed % 2 == 0), spread=0.35))
    p = np.array([[0.0, 0, 0], [0.1, 0, 0], [0.9, 0, 0], [0.0, 0, 0]])
    cases.append((p, np.array([0.5, 0.0, 0.0, 0.5])))      # zero samples, a duplicated ball
    cases.append((np.array([[0.0, 0, 0], [0.3, 0, 0]]), np.array([0.25, 0.25])))   # one circle each
    for (p, s), tols in [(c, (0.0, 1e-6)) for c in cases] + [(c, (1e-6,)) for c in exact_touch]:
        for tol in tols:
            want = orc.sphere_uncovered(p, s, tol=tol)
            for order in range(8):
                got, wit = _uncovered(host, p, s, tol, order)
                assert np.array_equal(got, want), (np.nonzero(got != want)[0][:8], got[got != want][:8])
                check_witnesses(p, s, tol, got, wit)
                assert np.all(np.isnan(wit[got != 1]))


def test_host_sphere_uncovered_csg10(host, orc):
    """The 10^3 CSG pseudo-SDF grid: 117 of 1,000 spheres are exactly
    covered; the certificate decides every sphere as the full enumeration
    does, in eight hierarchy orders."""
    w = W.csg_pseudo_grid(N=10, tau=1)
    want = orc.sphere_uncovered(w.p, w.s)
    for order in range(8):
        got, wit = _uncovered(host, w.p, w.s, 1e-6, order)
        assert np.array_equal(got, want)
    assert int(np.sum(want == 0)) == 117
    check_witnesses(w.p, w.s, 1e-6, got, wit)


def _intersections(host, p, s, tol, order):
    p, s = np.ascontiguousarray(p, np.float64), np.ascontiguousarray(s, np.float64)
    cap = 200000
    circ = np.zeros((cap, 2), np.int64)
    quad = np.zeros((cap, 4), np.int64)
    pts = np.zeros((cap, 3), np.float64)
    cnt = np.zeros(2, np.uint64)
    status = np.zeros(1, np.uint32)
    assert host.intersections_host(_ptr(p), _ptr(s), s.shape[0], tol, cap, _ptr(circ), cap, _ptr(quad), _ptr(pts),
                                   _ptr(cnt), _ptr(status), order) == 0
    nc, npt = int(cnt[0]), int(cnt[1])
    assert nc <= cap and npt <= cap and status[0] == 0
    circ, quad, pts = circ[:nc], quad[:npt], pts[:npt]
    oc = np.lexsort((circ[:, 1], circ[:, 0]))
    oq = np.lexsort((quad[:, 3], quad[:, 2], quad[:, 1], quad[:, 0]))
    return circ[oc], quad[oq], pts[oq]


def test_host_uncovered_intersections(host, orc):
    """Uncovered circles and points: the triangle and octahedral cases, the
    inflated sphere grid and valid and invalid tiny random inputs for tol 0
    and 1e-6, grids of exactly touching SDF samples (sphere, CSG) for tol
    1e-6, eight hierarchy orders: the same sorted lists as the oracle,
    points bit for bit."""
    h = np.sqrt(3) / 2
    cases = [(np.array([[0.0, 0, 0], [1.0, 0, 0], [0.5, h, 0], [0.5, h / 3, 1.3]]), np.array([1.0, 1, 1, 0.6]))]
    e = np.eye(3)
    for rho in (0.91, 0.93):
        cases.append((np.concatenate([np.zeros((1, 3)), e, -e]), np.array([1.0] + [rho] * 6)))
    w = W.sphere_grid(N=6, up=2, tau=2)
    cases += [(w.p, 1.2 * w.s)]
    exact_touch = [(w.p, w.s)]
    w = W.csg_pseudo_grid(N=6, tau=1)
    exact_touch.append((w.p, w.s))
    for seed in range(4):
        cases.append(W.tiny_random(40, seed, valid=(seed % 2 == 0), spread=0.35))
    for (p, s), tols in [(c, (0.0, 1e-6)) for c in cases] + [(c, (1e-6,)) for c in exact_touch]:
        for tol in tols:
            wc, wq, wp = orc.uncovered_intersections(p, s, tol=tol)
            for order in range(8):
                gc, gq, gp = _intersections(host, p, s, tol, order)
                assert np.array_equal(gc, wc), (len(gc), len(wc))
                assert np.array_equal(gq, wq), (len(gq), len(wq))
                assert np.array_equal(gp, wp)


def _exact_rmin(host, p, s, tol, box, x, sig, order):
    p, s, x = (np.ascontiguousarray(v, np.float64) for v in (p, s, x))
    sig = np.ascontiguousarray(sig, np.int8)
    out = np.zeros(x.shape[0])
    assert host.exact_rmin_host(_ptr(p), _ptr(s), s.shape[0], tol, int(box), _ptr(x), _ptr(sig), x.shape[0],
                                _ptr(out), order) == 0
    return out


def test_host_exact_rmin(host, orc):
    """Exact minimum valid radius over T, U, D (Sec. 6) from the uncovered
    circles and points: equal to the oracle's brute force bit for bit, for
    both signs and no sign, with and without the box, tol 0 and 1e-6."""
    cases = [W.tiny_random(n, seed, valid=(seed % 2 == 0), spread=0.35) for n, seed in ((12, 0), (25, 1), (40, 2))]
    h = np.sqrt(3) / 2
    cases.append((np.array([[0.0, 0, 0], [1.0, 0, 0], [0.5, h, 0], [0.5, h / 3, 1.3]]) * 0.5,
                  np.array([0.5, 0.5, 0.5, -0.3])))
    rng = np.random.default_rng(31)
    for p, s in cases:
        x = rng.uniform(-0.8, 0.8, size=(12, 3))
        for tol in (0.0, 1e-6):
            for box in (False, True):
                for sg in (1, -1, 0):
                    sig = np.full(x.shape[0], sg, np.int8)
                    want = np.array([orc.exact_rmin(p, s, x[t], sg, tol=tol, box_cull=box) for t in range(len(x))])
                    for order in (0, 5):
                        got = _exact_rmin(host, p, s, tol, box, x, sig, order)
                        assert np.array_equal(got, want), (tol, box, sg, got[got != want], want[got != want])


def test_host_argmin_points(host, orc):
    """q* from the plain and the augmented query's outputs, bit for bit
    against the oracle (NaN where no point sets the value)."""
    for seed in range(4):
        p, s = W.tiny_random(40, seed, valid=(seed % 2 == 0), spread=0.6)
        rng = np.random.default_rng(70 + seed)
        x = np.ascontiguousarray(np.concatenate([rng.uniform(-1.2, 1.2, size=(300, 3)), p[:5]]))
        U = orc.icosphere(2)
        surv = orc.collect(p, s, U, orc.keep_all(p, s, U))
        for _, arg, fl in (orc.query(p, s, surv, x)[:3], orc.query_aug(p, s, surv, x)):
            want = orc.argmin_points(p, s, U, x, arg, fl)
            got = np.zeros_like(want)
            fl16 = np.ascontiguousarray(fl.astype(np.uint16))
            arg = np.ascontiguousarray(arg)
            assert host.points_host(_ptr(p), _ptr(s), p.shape[0], _ptr(U), U.shape[0], _ptr(x), x.shape[0],
                                    _ptr(arg), _ptr(fl16), _ptr(got)) == 0
            assert np.array_equal(got, want, equal_nan=True)


def _scored_check(host, orc, p, s, tau, x, box_cull=True, orders=(0, 5)):
    p, s, x = (np.ascontiguousarray(a, np.float64) for a in (p, s, x))
    U = orc.icosphere(tau)
    surv = orc.collect(p, s, U, orc.keep_all(p, s, U, box_cull=box_cull))
    g, sph, q = (np.ascontiguousarray(surv[0], np.int64), np.ascontiguousarray(surv[1], np.int64),
                 np.ascontiguousarray(surv[2], np.float64))
    v0, a0, f0, _ = orc.query(p, s, surv, x)
    v1, a1, f1 = orc.query_scored(p, s, surv, x, box_cull=box_cull)
    for order in orders:
        val, arg, fl = v0.copy(), a0.copy(), f0.astype(np.uint16)
        assert host.scored_host(_ptr(p), _ptr(s), p.shape[0], _ptr(U), U.shape[0], 1e-6, int(box_cull), _ptr(g),
                                _ptr(sph), _ptr(q), g.shape[0], _ptr(x), x.shape[0], _ptr(val), _ptr(arg),
                                _ptr(fl), order) == 0
        bad = np.nonzero(~((val == v1) | (np.isnan(val) & np.isnan(v1))) | (arg != a1) |
                         (fl.astype(np.int32) != f1))[0]
        assert bad.size == 0, (f"order {order}: {bad.size} points differ, first {bad[:5]}: host {val[bad[:3]]} "
                               f"{arg[bad[:3]]} {fl[bad[:3]]} oracle {v1[bad[:3]]} {a1[bad[:3]]} {f1[bad[:3]]}")
    return f1


def test_host_scored_sphere_grid(host, orc):
    w = W.sphere_grid(N=8, up=2, tau=2)
    f = _scored_check(host, orc, w.p, w.s, w.tau, w.make_queries())
    assert np.sum((f & 15) == orc.CODE_TANGENT) > 50


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (9, 2), (60, 3), (200, 4)])
def test_host_scored_tiny_random(host, orc, n, seed):
    p, s = W.tiny_random(n, seed)
    x = np.random.default_rng(200 + seed).uniform(-1.1, 1.1, size=(200, 3))
    for tau in (0, 2):
        for box in (True, False):
            _scored_check(host, orc, p, s, tau, x, box_cull=box)


def test_host_scored_union_grid(host, orc):
    w = W.union_grid(N=10, up=2, tau=1)
    _scored_check(host, orc, w.p, w.s, w.tau, w.make_queries())
