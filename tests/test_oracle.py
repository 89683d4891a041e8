"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these checks re-types an oracle formula: each compares the oracle
with a closed form, an invariant, a special case or brute force of a
different formulation, chosen so that a dropped term, a wrong sign or index,
or a transposed operand fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest

from paper_2605_01919_gb300 import workloads as W

PHI = (1 + 5 ** 0.5) / 2


# ----------------------------------------------------------------------------
# icosphere (candidate directions)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("tau", range(0, 6))
def test_icosphere_counts_and_norms(orc, tau):
    U = orc.icosphere(tau)
    assert U.shape == (10 * 4 ** tau + 2, 3)          # 12, 42, 162, 642, ...
    assert np.abs(np.linalg.norm(U, axis=1) - 1).max() < 4e-16


def test_icosphere_base_is_regular_icosahedron(orc):
    U = orc.icosphere(0)
    G = U @ U.T
    # a regular icosahedron: every vertex has 5 neighbours at cos = 1/sqrt5,
    # 5 at -1/sqrt5 and one antipode
    for row in G:
        vals = np.sort(row)
        assert abs(vals[-1] - 1) < 1e-15 and abs(vals[0] + 1) < 1e-15
        assert np.sum(np.abs(vals - 1 / 5 ** 0.5) < 1e-12) == 5
        assert np.sum(np.abs(vals + 1 / 5 ** 0.5) < 1e-12) == 5
    # first vertex is (-1, phi, 0) / |.|
    n = math.sqrt(1 + PHI * PHI)
    assert np.allclose(U[0], [-1 / n, PHI / n, 0], atol=1e-15)


@pytest.mark.parametrize("tau", range(0, 5))
def test_icosphere_antipodal_exact(orc, tau):
    U = orc.icosphere(tau)
    keys = {tuple(u) for u in U}
    assert all(tuple(-u) in keys for u in U)


@pytest.mark.parametrize("tau", range(0, 5))
def test_icosphere_prefix(orc, tau):
    # vertices never move, so S_tau is a subset of S_tau+1 (as a prefix)
    a, b = orc.icosphere(tau), orc.icosphere(tau + 1)
    assert np.array_equal(a, b[: a.shape[0]])


@pytest.mark.parametrize("tau", [1, 2, 3])
def test_icosphere_topology(orc, tau):
    """Geodesic subdivision: 12 vertices of degree 5, all others degree 6,
    and every new vertex is the normalised midpoint of two older ones."""
    U = orc.icosphere(tau)
    K = U.shape[0]
    G = U @ U.T
    np.fill_diagonal(G, -2)
    nearest = G.max(axis=1)
    # neighbours: within a factor of the nearest neighbour's angle
    ang = np.arccos(np.clip(G, -1, 1))
    amin = np.arccos(np.clip(nearest, -1, 1))
    deg = np.sum(ang < 1.35 * amin[:, None], axis=1)
    assert np.sum(deg == 5) == 12 and np.sum(deg == 6) == K - 12
    prev = orc.icosphere(tau - 1)
    P = prev.shape[0]
    for k in range(P, K):
        m = prev[:, None, :] + prev[None, :, :]
        nm = np.linalg.norm(m, axis=2, keepdims=True)
        m = m / np.where(nm > 0, nm, 1.0)          # antipodal pairs sum to 0
        d = np.abs(m - U[k]).max(axis=2)
        assert d.min() < 1e-15


# ----------------------------------------------------------------------------
# P build: which candidates survive
# ----------------------------------------------------------------------------

def test_keep_single_sphere_all_in_box_survive(orc):
    U = orc.icosphere(2)
    p = np.array([[0.1, -0.2, 0.05]])
    s = np.array([0.4])
    keep = orc.keep_all(p, s, U)
    assert keep.all()                      # n=1: nothing else can cover
    s_big = np.array([1.5])
    keep = orc.keep_all(np.zeros((1, 3)), s_big, U)
    inbox = np.all(np.abs(1.5 * U) <= 1, axis=1)
    assert np.array_equal(keep[0].astype(bool), inbox)
    keep = orc.keep_all(np.zeros((1, 3)), s_big, U, box_cull=False)
    assert keep.all()


@pytest.mark.parametrize("seed", range(6))
def test_keep_two_spheres_cap_angle(orc, seed):
    """A point r1 u of sphere 1 lies in ball 2 (centre c at distance d in
    direction e) iff u.e > (r1^2 + d^2 - r2^2) / (2 r1 d) (law of cosines)."""
    rng = np.random.default_rng(seed)
    U = orc.icosphere(3)
    r1, r2 = rng.uniform(0.2, 0.4), rng.uniform(0.2, 0.4)
    e = rng.normal(size=3)
    e /= np.linalg.norm(e)
    d = rng.uniform(0.5 * (r1 + r2), 0.95 * (r1 + r2))
    p = np.array([[0.0, 0.0, 0.0], d * e])
    s = np.array([r1, -r2]) * (1 if seed % 2 else -1)     # either sign covers
    keep = orc.keep_all(p, s, U, tol=0.0, box_cull=False)
    cos_cap = (r1 * r1 + d * d - r2 * r2) / (2 * r1 * d)
    ue = U @ e
    far = np.abs(ue - cos_cap) > 1e-9
    assert np.array_equal(keep[0][far].astype(bool), (ue < cos_cap)[far])
    cos_cap2 = (r2 * r2 + d * d - r1 * r1) / (2 * r2 * d)
    ue2 = U @ (-e)
    far2 = np.abs(ue2 - cos_cap2) > 1e-9
    assert np.array_equal(keep[1][far2].astype(bool), (ue2 < cos_cap2)[far2])


def test_keep_concentric_and_touching(orc):
    U = orc.icosphere(2)
    p = np.zeros((2, 3))
    keep = orc.keep_all(p, np.array([0.5, 0.2]), U)
    assert keep[0].all() and not keep[1].any()
    # spheres touching at one point: touching is allowed (open ball), so the
    # contact candidate u = (1,0,0) of sphere 0 survives
    p = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0]])
    s = np.array([0.3, 0.2])
    k = int(np.where(np.all(U == [1.0, 0.0, 0.0], axis=1))[0][0])
    assert orc.keep_one(p, s, U, 0, k)
    # pushed 2 tol closer the contact point is covered
    p2 = np.array([[0.0, 0.0, 0.0], [0.5 - 3e-6, 0.0, 0.0]])
    assert not orc.keep_one(p2, s, U, 0, k)


def test_keep_zero_radius_covers_nothing(orc):
    U = orc.icosphere(1)
    p = np.array([[0.0, 0.0, 0.0], [0.1, 0.0, 0.0]])
    s = np.array([0.0, 0.3])
    keep = orc.keep_all(p, s, U)
    assert not keep[0].any()               # the point sample sits in ball 1
    assert keep[1].all()                   # a zero-radius ball covers nothing


def test_sphere_grid_survivor_count_matches_independent_probe(orc):
    """5,449 of 663,552 candidates survive on the 16^3 sphere grid at tau=2
    with box culling, the count an independent numpy evaluation of the same
    rule gives."""
    w = W.sphere_grid()
    keep = orc.keep_all(w.p, w.s, orc.icosphere(w.tau))
    assert keep.size == 663_552 and int(keep.sum()) == 5449


# ----------------------------------------------------------------------------
# query: the consistent value
# ----------------------------------------------------------------------------

def _solve(orc, p, s, tau, x, **kw):
    keep, surv, res = orc.solve(p, s, tau, x, **kw)
    return res


@pytest.mark.parametrize("seed", range(5))
def test_query_single_sphere_closed_form(orc, seed):
    """n = 1, x inside: survivors are the in-box candidates and
    |x - p - r u|^2 = delta^2 + r^2 - 2 r delta (u . v)."""
    rng = np.random.default_rng(seed)
    U = orc.icosphere(3)
    c = rng.uniform(-0.2, 0.2, 3)
    r = rng.uniform(0.3, 0.6)
    sign = 1 if seed % 2 else -1
    x = c + rng.uniform(-0.15, 0.15, size=(20, 3))
    val, arg, fl, _ = _solve(orc, c[None], np.array([sign * r]), 3, x)
    for t in range(20):
        v = x[t] - c
        delta = np.linalg.norm(v)
        cosang = U @ (v / delta)
        k = int(np.argmax(cosang))
        expect = math.sqrt(delta ** 2 + r ** 2 - 2 * r * delta * cosang[k])
        assert fl[t] & 15 == orc.CODE_SURVIVOR
        assert arg[t] == k                       # g = 0 * (K+1) + k
        assert abs(val[t] - sign * expect) < 1e-12
        # far bound = delta + r is never exceeded; LB = r - delta holds
        assert not (fl[t] & (orc.FLAG_FAR_VIOL | orc.FLAG_LB_VIOL))


def test_query_outside_sample_and_lower(orc):
    p = np.array([[0.0, 0.0, 0.0]])
    val, arg, fl, _ = _solve(orc, p, np.array([-0.3]), 2,
                             np.array([[0.5, 0, 0], [0, 0, 0], [0.1, 0.1, 0]]))
    assert fl[0] & 15 == orc.CODE_OUTSIDE and val[0] == 0          # Prop. 2 proof
    assert fl[1] & 15 == orc.CODE_SAMPLE and val[1] == -0.3        # reproduction
    assert fl[2] & 15 == orc.CODE_SURVIVOR and val[2] < 0
    # every candidate outside the box -> fall back to LB = r - |x - p|,
    # the exact single-sphere value
    x = np.array([[0.2, -0.1, 0.3]])
    val, arg, fl, _ = _solve(orc, np.zeros((1, 3)), np.array([3.0]), 2, x)
    assert fl[0] & 15 == orc.CODE_LOWER and arg[0] == 0
    assert abs(val[0] - (3.0 - np.linalg.norm(x[0]))) < 1e-15


def test_query_plane_column_exact(orc):
    """Samples of s = z above the plane z = 0; a query on a sample column at
    height z_x has exact value z_x (B(x, z_x) lies in the column's ball and
    touches the plane at the column's tangent point, a survivor)."""
    a = np.linspace(-0.5, 0.5, 5)
    z = np.linspace(0.1, 0.9, 5)
    P = np.array(list(itertools.product(a, a, z)))
    S = P[:, 2].copy()
    xs = np.array([[a[1], a[3], 0.05], [a[2], a[2], 0.37], [a[4], a[0], 0.8]])
    val, arg, fl, _ = _solve(orc, P, S, 1, xs)
    assert np.all(fl & 15 == orc.CODE_SURVIVOR)
    assert np.array_equal(val, xs[:, 2])


def test_query_reproduces_inputs_and_is_eikonal(orc):
    w = W.sphere_grid(N=8, up=2)
    x = w.make_queries()
    val, arg, fl, _ = _solve(orc, w.p, w.s, w.tau, x)
    # every input position is in the upsampled grid: values reproduced bitwise
    idx = {tuple(q): i for i, q in enumerate(x)}
    for i in range(w.n):
        t = idx[tuple(w.p[i])]
        assert fl[t] & 15 == orc.CODE_SAMPLE and val[t] == w.s[i]
    # no output ball intersects an opposite-sign input ball (Prop. 1 (i))
    d = np.linalg.norm(x[:, None, :] - w.p[None, :, :], axis=2)
    ok = (fl & 15) <= 1
    opp = np.sign(val)[:, None] * np.sign(w.s)[None, :] < 0
    gap = d - np.abs(w.s)[None, :] - np.abs(val)[:, None]
    assert np.all(gap[ok][opp[ok]] > -1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_query_bracket_against_exact_rmin(orc, seed):
    """LB <= exact r_min <= |s_tau| <= UB_opp on valid tiny inputs (tol = 0,
    no box): the survivors are uncovered contour points, the opposite
    tangent point lies beyond the sigma-contour, and every contour point is
    outside each containing ball."""
    p, s = W.tiny_random(14, seed)
    rng = np.random.default_rng(100 + seed)
    x = rng.uniform(-0.4, 0.4, size=(60, 3))
    val, arg, fl, _ = _solve(orc, p, s, 2, x, tol=0.0, box_cull=False)
    d = np.linalg.norm(x[:, None, :] - p[None], axis=2)
    checked = 0
    for t in range(60):
        code = fl[t] & 15
        if code not in (orc.CODE_SURVIVOR, orc.CODE_OPPOSITE):
            continue
        sig = 1 if val[t] > 0 else -1
        ex = orc.exact_rmin(p, s, x[t], sig, tol=0.0)
        same = np.sign(s) == sig
        opp = np.sign(s) == -sig
        lb = np.max(np.abs(s[same]) - d[t, same])
        assert lb <= ex + 1e-9
        assert ex <= abs(val[t]) + 1e-9
        if opp.any():
            assert abs(val[t]) <= np.min(d[t, opp] - np.abs(s[opp])) + 1e-12
        checked += 1
    assert checked > 10


def test_query_monotone_in_tau_and_converges(orc):
    p, s = W.tiny_random(10, 7)
    x = np.random.default_rng(5).uniform(-0.3, 0.3, size=(12, 3))
    prev = None
    errs = []
    ex = None
    for tau in range(0, 6):
        val, arg, fl, _ = _solve(orc, p, s, tau, x, tol=0.0, box_cull=False)
        ok = (fl & 15) <= 1
        if ex is None:
            ex = np.array([orc.exact_rmin(p, s, x[t], 1 if val[t] > 0 else -1, tol=0.0)
                           if ok[t] else np.nan for t in range(12)])
        if prev is not None:
            assert np.all(np.abs(val[ok]) <= np.abs(prev[ok]) + 1e-15)   # S_tau grows
        prev = val
        errs.append(np.nanmax(np.abs(val[ok]) - ex[ok]))
    assert errs[-1] < errs[0] and errs[-1] < 0.02


def test_query_lazy_equals_brute_force(orc):
    w = W.sphere_grid()
    U = orc.icosphere(w.tau)
    keep = orc.keep_all(w.p, w.s, U)
    surv = orc.collect(w.p, w.s, U, keep)
    x = w.make_queries()
    sel = np.random.default_rng(0).choice(x.shape[0], 60, replace=False)
    a = orc.query(w.p, w.s, surv, x[sel])
    b = orc.query_lazy(w.p, w.s, U, x[sel])
    for u, v in zip(a[:3], b[:3]):                 # value, argmin, flags
        assert np.array_equal(u, v, equal_nan=True) if u.dtype.kind == "f" else np.array_equal(u, v)
    # no opposite clamp: the nearest survivor must be found however far
    a = orc.query(w.p, w.s, surv, x[sel], clamp_opp=False)
    b = orc.query_lazy(w.p, w.s, U, x[sel], clamp_opp=False)
    for u, v in zip(a[:3], b[:3]):
        assert np.array_equal(u, v, equal_nan=True) if u.dtype.kind == "f" else np.array_equal(u, v)


# ----------------------------------------------------------------------------
# exact minimum radius (Sec. 6 algorithm) closed forms
# ----------------------------------------------------------------------------

def test_exact_rmin_single_and_pair(orc):
    p = np.array([[0.1, 0.0, -0.1]])
    x = np.array([0.2, 0.1, 0.0])
    assert abs(orc.exact_rmin(p, np.array([0.5]), x, 1) - (0.5 - np.linalg.norm(x - p[0]))) < 1e-15
    # two equal intersecting spheres, x at the circle centre: r_min = rho
    r, d = 0.4, 0.5
    p = np.array([[-d / 2, 0, 0], [d / 2, 0, 0]])
    got = orc.exact_rmin(p, np.array([r, r]), np.zeros(3), 1)
    assert abs(got - math.sqrt(r * r - d * d / 4)) < 1e-14


# ----------------------------------------------------------------------------
# gradient: analytic formulas against central differences of the value
# ----------------------------------------------------------------------------

def test_grad_matches_finite_differences(orc):
    w = W.sphere_grid(N=8, up=2)
    U = orc.icosphere(2)
    rng = np.random.default_rng(3)
    x = rng.uniform(-0.9, 0.9, size=(40, 3))
    keep = orc.keep_all(w.p, w.s, U)
    surv = orc.collect(w.p, w.s, U, keep)
    val, arg, fl, gap = orc.query(w.p, w.s, surv, x)
    gup = np.ones(x.shape[0])
    gx, gp, gs = orc.grad(w.p, w.s, U, x, val, arg, fl, gup)
    h = 1e-7
    tested = 0
    for t in range(x.shape[0]):
        code = fl[t] & 15
        if code not in (0, 1) or gap[t] < 1e-4:
            continue
        for c in range(3):
            xp, xm = x[t].copy(), x[t].copy()
            xp[c] += h
            xm[c] -= h
            vp = orc.query(w.p, w.s, surv, xp[None])[0][0]
            vm = orc.query(w.p, w.s, surv, xm[None])[0][0]
            assert abs((vp - vm) / (2 * h) - gx[t, c]) < 1e-5
        tested += 1
        # derivative wrt the sample that set the value (survivor moves with it)
        j = arg[t] // (U.shape[0] + 1) if code == 0 else arg[t]
        sp, sm = w.s.copy(), w.s.copy()
        sp[j] += h
        sm[j] -= h
        kp = orc.collect(w.p, sp, U, orc.keep_all(w.p, sp, U))
        km = orc.collect(w.p, sm, U, orc.keep_all(w.p, sm, U))
        vp = orc.query(w.p, sp, kp, x[t][None])[0][0]
        vm = orc.query(w.p, sm, km, x[t][None])[0][0]
        gsingle = orc.grad(w.p, w.s, U, x[t][None], val[t:t + 1], arg[t:t + 1], fl[t:t + 1],
                           np.ones(1))[2][j]
        assert abs((vp - vm) / (2 * h) - gsingle) < 1e-5
        if tested >= 6:
            break
    assert tested >= 4


def _query_one(orc, p, s, U, x):
    """Value, argmin and code at one point after a fresh P build of (p, s)."""
    surv = orc.collect(p, s, U, orc.keep_all(p, s, U))
    v, a, f, _ = orc.query(p, s, surv, x[None])
    return v[0], a[0], f[0] & 15


def _fd_sample(orc, p, s, U, x, j, which, h):
    """Central difference of the value at x in sample j's coordinate `which`
    (0..2: p_j, 3: s_j), rebuilding the survivor set each side; None when the
    argmin or the code changes inside the stencil (a tie is crossed)."""
    pp, pm, sp, sm = p.copy(), p.copy(), s.copy(), s.copy()
    if which < 3:
        pp[j, which] += h
        pm[j, which] -= h
    else:
        sp[j] += h
        sm[j] -= h
    vp, ap, cp = _query_one(orc, pp, sp, U, x)
    vm, am, cm = _query_one(orc, pm, sm, U, x)
    v0, a0, c0 = _query_one(orc, p, s, U, x)
    if not (ap == a0 == am and cp == c0 == cm):
        return None
    return (vp - vm) / (2 * h)


@pytest.mark.parametrize("code", [0, 1])
def test_grad_sample_position_and_value_match_finite_differences(orc, code):
    """d s*/d p_j and d s*/d s_j of SURVIVOR (code 0: the candidate moves with
    its sphere) and OPPOSITE (code 1: the tangent point of sphere j) results
    against central differences of the rebuilt P and the re-run query."""
    w = W.sphere_grid(N=7, up=2)
    U = orc.icosphere(2)
    K = U.shape[0]
    rng = np.random.default_rng(17 + code)
    x = rng.uniform(-0.95, 0.95, size=(400, 3))
    surv = orc.collect(w.p, w.s, U, orc.keep_all(w.p, w.s, U))
    val, arg, fl, gap = orc.query(w.p, w.s, surv, x)
    sel = np.nonzero(((fl & 15) == code) & (gap > 1e-4) & (np.abs(val) > 1e-3))[0]
    h = 1e-7
    tested = 0
    for t in sel[:8]:
        j = arg[t] // (K + 1) if code == 0 else arg[t]
        gx, gp, gs = orc.grad(w.p, w.s, U, x[t][None], val[t:t + 1], arg[t:t + 1], fl[t:t + 1], np.ones(1))
        for which in range(4):
            fd = _fd_sample(orc, w.p, w.s, U, x[t], j, which, h)
            if fd is None:
                continue
            an = gp[j, which] if which < 3 else gs[j]
            assert abs(fd - an) < 1e-5, (t, which, fd, an)
            tested += 1
    assert tested >= 16


def _lower_case(sign):
    # two large spheres of one sign whose candidates all lie outside the box:
    # no survivor and no opposite sphere, so every query inside is LOWER with
    # value sign * max_j (r_j - |x - p_j|)
    p = np.array([[0.1, 0.05, -0.1], [-0.2, 0.1, 0.15]])
    s = sign * np.array([3.0, 2.5])
    return p, s


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_grad_lower_branch_matches_closed_form_and_finite_differences(orc, sign):
    """The LOWER branch (no candidate: value = sign * LB, LB the depth of the
    deepest containing ball): its value is the closed form, and its
    derivatives in x, p_j and s_j match central differences."""
    p, s = _lower_case(sign)
    U = orc.icosphere(1)
    K = U.shape[0]
    rng = np.random.default_rng(23)
    x = rng.uniform(-0.6, 0.6, size=(12, 3))
    surv = orc.collect(p, s, U, orc.keep_all(p, s, U))
    assert surv[0].shape[0] == 0
    val, arg, fl, _ = orc.query(p, s, surv, x)
    assert np.all(fl & 15 == orc.CODE_LOWER)
    depth = np.abs(s)[None, :] - np.linalg.norm(x[:, None, :] - p[None, :, :], axis=2)
    assert np.array_equal(arg, np.argmax(depth, axis=1))
    assert np.allclose(val, sign * depth.max(axis=1), rtol=0, atol=1e-15)
    h = 1e-6
    for t in range(x.shape[0]):
        j = arg[t]
        if abs(depth[t, 0] - depth[t, 1]) < 1e-3:
            continue
        gx, gp, gs = orc.grad(p, s, U, x[t][None], val[t:t + 1], arg[t:t + 1], fl[t:t + 1], np.ones(1))
        for c in range(3):
            e = np.zeros(3)
            e[c] = h
            vp = _query_one(orc, p, s, U, x[t] + e)[0]
            vm = _query_one(orc, p, s, U, x[t] - e)[0]
            assert abs((vp - vm) / (2 * h) - gx[0, c]) < 1e-7
        for which in range(4):
            fd = _fd_sample(orc, p, s, U, x[t], j, which, h)
            assert fd is not None
            an = gp[j, which] if which < 3 else gs[j]
            assert abs(fd - an) < 1e-7, (t, which, fd, an)
        # the other sphere does not set the value: no gradient reaches it
        assert np.all(gp[1 - j] == 0) and gs[1 - j] == 0


# ----------------------------------------------------------------------------
# greedy insertion: the incremental state equals a rebuild from scratch
# ----------------------------------------------------------------------------

def test_insert_state_equals_rebuild(orc):
    w = W.sphere_grid(N=7, up=2)
    U = orc.icosphere(1)
    K = U.shape[0]
    y = np.random.default_rng(11).uniform(-0.8, 0.8, size=(25, 3))
    val, arg, fl, st = orc.insert(w.p, w.s, U, y)
    inserted = np.isin(fl & 15, [0, 1, 5])
    assert st["s"].shape[0] == w.n + inserted.sum()
    assert np.array_equal(st["s"][w.n:], val[inserted])
    # every candidate was tested against every sphere: the final survivor
    # set is the brute-force keep set of the final spheres, plus witnesses
    keep = orc.keep_all(st["p"], st["s"], U)
    g_expect = set()
    for i, k in zip(*np.nonzero(keep)):
        g_expect.add(int(i) * (K + 1) + int(k))
    g_got = set(int(g) for g in st["g"] if g % (K + 1) != K)
    assert g_got == g_expect
    # each inserted value is reproduced when queried afterwards
    surv = (st["g"], st["sph"], st["q"])
    v2, a2, f2, _ = orc.query(st["p"], st["s"], surv, y[inserted])
    assert np.all(f2 & 15 == orc.CODE_SAMPLE) and np.array_equal(v2, val[inserted])


def test_insert_first_value_equals_query(orc):
    w = W.sphere_grid(N=7, up=2)
    U = orc.icosphere(2)
    y = np.array([[0.13, -0.21, 0.05], [0.3, 0.3, 0.3]])
    val, arg, fl, _ = orc.insert(w.p, w.s, U, y[:1])
    q = orc.solve(w.p, w.s, 2, y[:1])[2]
    assert val[0] == q[0][0] and arg[0] == q[1][0] and fl[0] == q[2][0]


# ----------------------------------------------------------------------------
# insertion with known values (Sec. 6 repair of removed samples)
# ----------------------------------------------------------------------------

def test_insert_known_sign_equals_inferred_where_they_agree(orc):
    """Where containment gives the same class as the known value's sign, the
    known-value loop takes the same decisions (only NONCONSERVATIVE may be
    added)."""
    w = W.sphere_grid(N=7, up=2)
    U = orc.icosphere(1)
    y = np.random.default_rng(12).uniform(-0.8, 0.8, size=(30, 3))
    v0, a0, f0, _ = orc.insert(w.p, w.s, U, y)
    ok = np.isin(f0 & 15, [0, 1, 5])
    # the loops only stay in step while every earlier decision agrees
    first_bad = np.argmin(ok) if not ok.all() else y.shape[0]
    yk = y[:first_bad]
    known = np.where(v0[:first_bad] >= 0, 1.0, -1.0) * 1e-9     # sign only, tiny magnitude
    v1, a1, f1, _ = orc.insert(w.p, w.s, U, yk, known=known)
    assert first_bad >= 5
    assert np.array_equal(v1, v0[:first_bad]) and np.array_equal(a1, a0[:first_bad])
    assert np.array_equal(f1 & ~orc.FLAG_NONCONSERVATIVE, f0[:first_bad])
    assert not np.any(f1 & orc.FLAG_NONCONSERVATIVE)   # |value| >= 1e-9 - tol always


def test_insert_known_sign_single_sphere_closed_forms(orc):
    """One positive sphere (p, r), a point y outside its ball: with known sign
    + the value is the distance to the nearest in-box candidate of the sphere
    (brute force over the icosphere); with known sign - the sphere is the
    opposite class and the value is -(|y - p| - r) (its tangent point)."""
    p = np.array([[0.1, -0.05, 0.02]])
    s = np.array([0.3])
    U = orc.icosphere(2)
    y = np.array([[0.62, 0.31, -0.2]])
    v, a, f, _ = orc.insert(p, s, U, y, known=np.array([0.5]))
    q = p[0] + s[0] * U
    q = q[np.all(np.abs(q) <= 1.0, axis=1)]
    d = np.sqrt(((y[0] - q) ** 2).sum(axis=1))
    assert f[0] & 15 == orc.CODE_SURVIVOR and abs(v[0] - d.min()) < 1e-15
    assert f[0] & orc.FLAG_NONCONSERVATIVE        # |v| < 0.5 - tol
    v, a, f, _ = orc.insert(p, s, U, y, known=np.array([-0.01]))
    assert f[0] & 15 == orc.CODE_OPPOSITE and a[0] == 0
    assert abs(v[0] + (np.sqrt(((y[0] - p[0]) ** 2).sum()) - s[0])) < 1e-15
    assert not f[0] & orc.FLAG_NONCONSERVATIVE
    # no survivor and no sphere of either class (one zero sample outside the
    # box, its only candidate box-culled): LOWER, value 0, argmin -1, and the
    # point itself becomes the new sphere's witness
    v, a, f, st = orc.insert(np.array([[1.5, 0.0, 0.0]]), np.array([0.0]), U, y, known=np.array([0.2]))
    assert f[0] & 15 == orc.CODE_LOWER and v[0] == 0.0 and a[0] == -1
    K = U.shape[0]
    assert np.array_equal(st["g"], [1 * (K + 1) + k for k in range(K + 1)])   # zero sphere at y: all survive
    assert np.allclose(st["q"], y[0])


# ----------------------------------------------------------------------------
# same-sign tangent augmentation (the first "next" item: oracle side)
# ----------------------------------------------------------------------------

def test_query_aug_single_sphere_is_the_ball_distance(orc):
    """One sphere, points inside its ball: the near tangent point is
    uncovered, so the augmented value is sign * (r - |x - p|), the distance
    to the sphere, which no icosphere candidate reaches exactly."""
    U = orc.icosphere(2)
    rng = np.random.default_rng(41)
    for sgn in (1.0, -1.0):
        p = np.array([[0.1, -0.05, 0.02]])
        s = np.array([0.3 * sgn])
        surv = orc.collect(p, s, U, orc.keep_all(p, s, U))
        x = p[0] + rng.uniform(-0.15, 0.15, size=(50, 3))
        d = np.linalg.norm(x - p[0], axis=1)
        x, d = x[d < 0.29], d[d < 0.29]
        val, arg, fl = orc.query_aug(p, s, surv, x)
        assert np.all(fl & 15 == orc.CODE_TANGENT) and np.all(arg == 0)
        assert np.all(np.abs(np.abs(val) - (0.3 - d)) < 1e-14) and np.all(np.sign(val) == sgn)
        plain = orc.query(p, s, surv, x)[0]
        assert np.all(np.abs(val) <= np.abs(plain))


@pytest.mark.parametrize("seed", range(4))
def test_query_aug_between_exact_and_plain(orc, seed):
    """exact r_min <= |s_aug| <= |s_tau| on valid tiny inputs (tol = 0, no
    box): the added candidates are uncovered tangent points (members of T in
    Def. 1) and the candidate set only grows; where no tangent point wins the
    result equals the plain query's."""
    p, s = W.tiny_random(14, seed)
    rng = np.random.default_rng(100 + seed)
    x = rng.uniform(-0.4, 0.4, size=(60, 3))
    U = orc.icosphere(2)
    keep = orc.keep_all(p, s, U, tol=0.0, box_cull=False)
    surv = orc.collect(p, s, U, keep)
    v0, a0, f0, _ = orc.query(p, s, surv, x, tol=0.0)
    v1, a1, f1 = orc.query_aug(p, s, surv, x, tol=0.0, box_cull=False)
    won = (f1 & 15) == orc.CODE_TANGENT
    assert np.array_equal(v1[~won], v0[~won], equal_nan=True)
    assert np.array_equal(a1[~won], a0[~won]) and np.array_equal(f1[~won], f0[~won])
    assert won.any()
    checked = 0
    for t in np.nonzero(won)[0]:
        assert abs(v1[t]) < abs(v0[t]) and np.sign(v1[t]) == np.sign(v0[t])
        sig = 1 if v1[t] > 0 else -1
        ex = orc.exact_rmin(p, s, x[t], sig, tol=0.0)
        assert ex <= abs(v1[t]) + 1e-9
        checked += 1
    assert checked >= 3


def _tangent_fd(orc, p, s, U, x, v, a, f, t, h=1e-7):
    """Central differences of the augmented value at point t in x, p_j and
    s_j (j = the winning sphere) next to the analytic gradient; None when a
    step changes the argmin."""
    j = a[t] // 2
    fd = []
    for kind, c in [("x", 0), ("x", 1), ("x", 2), ("p", 0), ("p", 1), ("p", 2), ("s", 0)]:
        vals = []
        for sgn in (1, -1):
            xx, pp, ss = x[t:t + 1].copy(), p.copy(), s.copy()
            if kind == "x":
                xx[0, c] += sgn * h
            elif kind == "p":
                pp[j, c] += sgn * h
            else:
                ss[j] += sgn * h
            sv = orc.collect(pp, ss, U, orc.keep_all(pp, ss, U, tol=0.0, box_cull=False))
            vv, aa, ff = orc.query_aug(pp, ss, sv, xx, tol=0.0, box_cull=False)
            if aa[0] != a[t] or (ff[0] & 15) != orc.CODE_TANGENT:
                return None
            vals.append(vv[0])
        fd.append((vals[0] - vals[1]) / (2 * h))
    one = np.zeros(x.shape[0])
    one[t] = 1.0
    gx, gp, gs = orc.grad(p, s, U, x, v, a, f, one)
    return np.array(fd), np.concatenate([gx[t], gp[j], [gs[j]]])


# (n, seed, points): seeded tiny inputs, uniform points in [-0.6, 0.6]^3, and
# points whose winner is a near tangent point seen from outside its ball or a
# far tangent point (rare: most winners are near points seen from inside)
TANGENT_FD_CASES = [(30, 1, [67]), (14, 2, [103]), (30, 2, [13, 20])]


@pytest.mark.parametrize("n,seed,pts", TANGENT_FD_CASES)
def test_grad_tangent_rare_sides_match_finite_differences(orc, n, seed, pts):
    p, s = W.tiny_random(n, seed)
    x = np.random.default_rng(seed).uniform(-0.6, 0.6, size=(400, 3))
    U = orc.icosphere(1)
    surv = orc.collect(p, s, U, orc.keep_all(p, s, U, tol=0.0, box_cull=False))
    v, a, f = orc.query_aug(p, s, surv, x, tol=0.0, box_cull=False)
    for t in pts:
        assert (f[t] & 15) == orc.CODE_TANGENT
        j = a[t] // 2
        inside = np.linalg.norm(x[t] - p[j]) < abs(s[j])
        assert (a[t] % 2 == 1) or not inside    # a far point, or a near one seen from outside
        r = _tangent_fd(orc, p, s, U, x, v, a, f, t)
        assert r is not None
        fd, an = r
        assert np.allclose(fd, an, atol=1e-6), (fd, an)


def test_grad_tangent_matches_finite_differences(orc):
    """The TANGENT branch of the analytic gradient against central
    differences of the augmented query itself (in x, in p_j and in s_j),
    at points where a tangent point wins with the same argmin on both sides
    of the step: the derivative of the distance to the moving tangent point."""
    p, s = W.tiny_random(14, 1)
    rng = np.random.default_rng(7)
    x = rng.uniform(-0.4, 0.4, size=(80, 3))
    U = orc.icosphere(1)
    surv = orc.collect(p, s, U, orc.keep_all(p, s, U, tol=0.0, box_cull=False))
    v, a, f = orc.query_aug(p, s, surv, x, tol=0.0, box_cull=False)
    won = np.nonzero((f & 15) == orc.CODE_TANGENT)[0]
    assert won.size >= 5
    checked = 0
    for t in won[:12]:
        r = _tangent_fd(orc, p, s, U, x, v, a, f, t)
        if r is None:
            continue
        fd, an = r
        assert np.allclose(fd, an, atol=1e-6), (fd, an)
        checked += 1
    assert checked >= 3


# ----------------------------------------------------------------------------
# refinement order (Sec. 4.2): covered counts and the flood-fill order
# ----------------------------------------------------------------------------

# sub = 8: a sub-point sits at h/16 * (k1, k2, k3) from the cell centre with
# odd k in {+-1, +-3, +-5, +-7}; the points with k1^2 + k2^2 + k3^2 < R^2 are
# 8 for 3 < R^2 <= 11 ((1,1,1)), 32 up to 19 (+ (1,1,3) x 24), 56 up to 27
# (+ (1,3,3) x 24), 88 up to 35 (+ (3,3,3) x 8 and (1,1,5) x 24), all 512
# above 3 * 49 = 147.
@pytest.mark.parametrize("R2,count", [(2.0, 0), (7.0, 8), (15.0, 32), (23.0, 56), (31.0, 88), (150.0, 512)])
def test_cell_coverage_lattice_shells(orc, R2, count):
    h = 0.05
    origin = np.array([-1.0, -1.0, -1.0])
    cell = np.array([[2, -1, 3]])
    centre = origin + h * (cell[0] + 0.5)
    for sign in (1.0, -1.0):
        p = centre[None, :].copy()
        s = np.array([sign * h / 16 * np.sqrt(R2)])
        assert orc.cell_coverage(p, s, cell, origin, h, 8, tol=0.0)[0] == count


def test_cell_coverage_union_zero_and_far(orc):
    """Coverage is by any ball of either sign; zero samples and far balls
    cover nothing; a point counts once however many balls hold it."""
    h = 0.1
    origin = np.zeros(3)
    cells = np.array([[0, 0, 0], [5, 0, 0], [0, 7, 0]])
    c0 = origin + h * 0.5
    p = np.array([c0, c0, c0 + [0.5, 0, 0], c0 + [0, 0.7, 0]])
    s = np.array([0.2, -0.3, 0.0, -1e-3])
    got = orc.cell_coverage(p, s, cells, origin, h, 8, tol=0.0)
    assert list(got) == [512, 0, 0]
    # the tolerance shrinks the balls: with tol = 1e-6 a ball reaching 0.5e-6
    # past the corner sub-points (7 sqrt(3) h/16 away) misses the 8 corners,
    # one reaching 2e-6 past them holds all 512 points
    r_all = h / 16 * np.sqrt(147.0)
    assert orc.cell_coverage(c0[None], np.array([r_all + 0.5e-6]), cells[:1], origin, h, 8, tol=1e-6)[0] == 504
    assert orc.cell_coverage(c0[None], np.array([r_all + 2e-6]), cells[:1], origin, h, 8, tol=1e-6)[0] == 512


# Hand-worked orders (26-neighbourhood, lowest count first, ties to the
# lower index):
FLOOD_CASES = [
    # chain along x, counts 5 1 3 2: start at 1, queue {0, 2}; pop 2, queue
    # 3; pop 3 (2 < 5); then 0
    ([(0, 0, 0), (1, 0, 0), (2, 0, 0), (3, 0, 0)], [5, 1, 3, 2], [1, 2, 3, 0]),
    # two components: start at the global minimum (2), finish its
    # component, then the least covered rest
    ([(0, 0, 0), (1, 0, 0), (5, 5, 5), (6, 5, 5)], [4, 9, 2, 7], [2, 3, 0, 1]),
    # (0,0,0) and (1,1,1) touch at a corner, so 1 follows 0 before the
    # less covered but unconnected cell 2
    ([(0, 0, 0), (1, 1, 1), (5, 0, 0)], [1, 9, 5], [0, 1, 2]),
    # equal counts in a 2 x 2 square: lowest index first
    ([(0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 0)], [3, 3, 3, 3], [0, 1, 2, 3]),
    ([(0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 0)], [3, 3, 3, 1], [3, 0, 1, 2]),
    # the flood follows connectivity, not the global order: the other
    # count-0 cell (4) comes last
    ([(0, 0, 0), (1, 0, 0), (2, 0, 0), (3, 0, 0), (4, 0, 0)], [0, 9, 1, 9, 0], [0, 1, 2, 3, 4]),
    # cells two apart are not neighbours
    ([(0, 0, 0), (2, 0, 0), (1, 5, 0)], [1, 0, 2], [1, 0, 2]),
]


@pytest.mark.parametrize("cells,counts,order", FLOOD_CASES)
def test_flood_order_hand_worked(orc, cells, counts, order):
    assert orc.flood_order(np.array(cells), np.array(counts)) == order


def test_flood_order_components_contiguous(orc):
    """On a random sparse set of cells: a permutation; every connected
    component (26-neighbourhood) is emitted as one contiguous run that starts
    at its least covered cell, and the runs start in increasing order of
    that cell's (count, index)."""
    rng = np.random.default_rng(4)
    all_cells = np.array([(i, j, k) for i in range(9) for j in range(9) for k in range(3)])
    cells = all_cells[rng.random(all_cells.shape[0]) < 0.3]
    counts = rng.integers(0, 20, cells.shape[0])
    order = orc.flood_order(cells, counts)
    assert sorted(order) == list(range(cells.shape[0]))
    # components by union-find over the 26-neighbourhood
    where = {tuple(c): i for i, c in enumerate(cells)}
    parent = list(range(len(cells)))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a
    for i, c in enumerate(cells):
        for d in orc.NEIGHBOURS:
            j = where.get((c[0] + d[0], c[1] + d[1], c[2] + d[2]))
            if j is not None:
                parent[find(i)] = find(j)
    comp = [find(i) for i in order]
    runs = [comp[0]] + [comp[t] for t in range(1, len(comp)) if comp[t] != comp[t - 1]]
    assert len(runs) == len(set(runs)) and len(runs) > 3
    firsts = [order[0]] + [order[t] for t in range(1, len(order)) if comp[t] != comp[t - 1]]
    for f in firsts:
        members = [i for i in range(len(cells)) if find(i) == find(f)]
        assert f == min(members, key=lambda i: (counts[i], i))
    keys = [(counts[f], f) for f in firsts]
    assert keys == sorted(keys)


@pytest.mark.parametrize("n,seed", [(1, 0), (7, 2), (37, 3), (257, 5)])
def test_query_aug_lazy_equals_brute_force(orc, n, seed):
    """The lazy augmented query (plain part from query_lazy, tangent points
    tested only where they can change the result) equals the brute-force
    augmented query bit for bit, option combinations included."""
    p, s = W.tiny_random(n, seed, valid=(seed % 3 != 0), spread=0.9)
    rng = np.random.default_rng(1000 + seed)
    x = np.concatenate([rng.uniform(-1, 1, size=(200, 3)), p[: min(n, 10)], rng.uniform(-1.5, 1.5, size=(10, 3))])
    for tau in (0, 2):
        U = orc.icosphere(tau)
        for box_cull, clamp in [(True, True), (False, True), (True, False)]:
            surv = orc.collect(p, s, U, orc.keep_all(p, s, U, box_cull=box_cull))
            a = orc.query_aug(p, s, surv, x, clamp_opp=clamp, box_cull=box_cull)
            b = orc.query_aug_lazy(p, s, U, x, box_cull=box_cull, clamp_opp=clamp)
            assert np.array_equal(a[0], b[0], equal_nan=True)
            assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_query_aug_lazy_equals_brute_force_grids(orc):
    for w in (W.sphere_grid(N=10, up=2, tau=2), W.union_grid(N=12, up=4)):
        x = w.make_queries()
        x = x[np.random.default_rng(6).choice(x.shape[0], 300, replace=False)]
        U = orc.icosphere(w.tau)
        surv = orc.collect(w.p, w.s, U, orc.keep_all(w.p, w.s, U))
        a = orc.query_aug(w.p, w.s, surv, x)
        b = orc.query_aug_lazy(w.p, w.s, U, x)
        assert np.sum((a[2] & 15) == orc.CODE_TANGENT) > 10
        assert np.array_equal(a[0], b[0], equal_nan=True)
        assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


# ----------------------------------------------------------------------------
# exact uncovered test per sphere (Prop. 1 (ii))
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("rho,covered", [(0.93, True), (0.91, False), (0.9194, False), (0.9195, True)])
def test_sphere_uncovered_octahedral_caps(orc, rho, covered):
    """The unit sphere with six balls of radius rho centred at +-e_x, +-e_y,
    +-e_z (tol = 0): a ball covers the cap of half-angle t with
    2 - 2 cos t = rho^2; the caps cover the sphere exactly when t reaches the
    corner directions (1,1,1)/sqrt 3, cos t = 1/sqrt 3, i.e.
    rho > sqrt(2 - 2/sqrt 3) = 0.919401..."""
    e = np.eye(3)
    p = np.concatenate([np.zeros((1, 3)), e, -e])
    s = np.array([1.0] + [rho] * 6)
    assert orc.sphere_uncovered(p, s, tol=0.0)[0] == (0 if covered else 1)


# ----------------------------------------------------------------------------
# uncovered intersection circles and points (Def. 1 U, D; Sec. 4.1)
# ----------------------------------------------------------------------------

def test_uncovered_intersections_three_spheres(orc):
    """Three unit spheres centred on an equilateral triangle of side a = 1:
    three circles, and two points shared by all three at the centroid
    +- sqrt(1 - a^2/3) along the normal; a fourth ball around the upper point
    covers it and leaves the lower one."""
    h = np.sqrt(3) / 2
    p = np.array([[0.0, 0, 0], [1.0, 0, 0], [0.5, h, 0]])
    s = np.ones(3)
    circ, quads, pts = orc.uncovered_intersections(p, s, tol=0.0)
    assert circ.tolist() == [[0, 1], [0, 2], [1, 2]]
    assert quads.tolist() == [[0, 1, 2, 0], [0, 1, 2, 1]]
    z = np.sqrt(1 - 1 / 3)
    centroid = np.array([0.5, h / 3, 0.0])
    got = sorted(pts.tolist(), key=lambda q: q[2])
    assert np.allclose(got, [centroid - [0, 0, z], centroid + [0, 0, z]], atol=1e-15)
    p4 = np.concatenate([p, [[0.5, h / 3, 1.3]]])
    s4 = np.array([1.0, 1.0, 1.0, 0.6])
    circ, quads, pts = orc.uncovered_intersections(p4, s4, tol=1e-6)
    assert [0, 1] in circ.tolist() and [0, 2] in circ.tolist() and [1, 2] in circ.tolist()
    own = [k for k, q in enumerate(quads.tolist()) if q[:3] == [0, 1, 2]]
    assert len(own) == 1 and pts[own[0], 2] < 0 and abs(pts[own[0], 2] + z) < 1e-15


@pytest.mark.parametrize("rho,covered", [(0.93, True), (0.91, False), (0.9194, False), (0.9195, True)])
def test_uncovered_intersections_octahedral(orc, rho, covered):
    """The unit sphere (index 0) with six balls of radius rho at +-e_x,
    +-e_y, +-e_z (tol 0).  The circle with ball e_a is at cos t = c =
    1 - rho^2/2 from the axis; the points it shares with an adjacent ball e_b
    are c e_a + c e_b +- w e_c, w = sqrt(1 - 2c^2), and the third ball e_c
    covers the one on its side exactly when w > c, i.e. rho >
    sqrt(2 - 2/sqrt 3), the threshold at which the caps cover the sphere.
    Below it: all six circles of sphere 0 and the 24 points (12 adjacent
    pairs, two each) are uncovered; above it: none."""
    e = np.eye(3)
    p = np.concatenate([np.zeros((1, 3)), e, -e])
    s = np.array([1.0] + [rho] * 6)
    circ, quads, pts = orc.uncovered_intersections(p, s, tol=0.0)
    mine_c = [c for c in circ.tolist() if c[0] == 0]
    mine_q = [k for k, q in enumerate(quads.tolist()) if q[0] == 0]
    if covered:
        assert mine_c == [] and mine_q == []
        return
    assert mine_c == [[0, k] for k in range(1, 7)]
    assert len(mine_q) == 24
    c = 1 - rho ** 2 / 2
    w = np.sqrt(1 - 2 * c * c)
    for k in mine_q:
        a = np.sort(np.abs(pts[k]))
        assert np.allclose(a, [w, c, c], atol=1e-14)
        assert abs(np.linalg.norm(pts[k]) - 1) < 1e-14


@pytest.mark.parametrize("seed", range(4))
def test_uncovered_intersections_properties(orc, seed):
    """Random inputs (tol 0): every reported point lies on its three spheres
    and in no other ball; no circle or point involves a sphere that the
    other balls cover entirely (Prop. 1 (ii) test); a circle on which one of
    720 sampled points lies clear of every other ball is reported."""
    rng = np.random.default_rng(40 + seed)
    n = 24
    p = rng.uniform(-0.5, 0.5, size=(n, 3))
    s = rng.uniform(0.15, 0.45, size=n) * rng.choice([-1, 1], size=n)
    circ, quads, pts = orc.uncovered_intersections(p, s, tol=0.0)
    r = np.abs(s)
    for (i, j, m, _), q in zip(quads, pts):
        for k in (i, j, m):
            assert abs(np.linalg.norm(q - p[k]) - r[k]) < 1e-12
        d = np.linalg.norm(p - q, axis=1)
        inside = d < r
        inside[[i, j, m]] = False
        assert not inside.any()
    unc = orc.sphere_uncovered(p, s, tol=0.0)
    involved = set(circ.ravel().tolist()) | set(quads[:, :3].ravel().tolist())
    assert all(unc[k] == 1 for k in involved)
    reported = set(map(tuple, circ.tolist()))
    phi = np.linspace(0, 2 * np.pi, 720, endpoint=False)
    for i in range(n):
        for j in range(i + 1, n):
            dv = p[j] - p[i]
            d = np.linalg.norm(dv)
            if not (abs(r[i] - r[j]) < d < r[i] + r[j]):
                continue
            mu = dv / d
            a = (d * d + r[i] ** 2 - r[j] ** 2) / (2 * d)
            rad = np.sqrt(r[i] ** 2 - a * a)
            u = np.cross(mu, [1.0, 0, 0] if abs(mu[0]) < 0.9 else [0, 1.0, 0])
            u /= np.linalg.norm(u)
            v = np.cross(mu, u)
            q = p[i] + a * mu + rad * (np.outer(np.cos(phi), u) + np.outer(np.sin(phi), v))
            dd = np.linalg.norm(q[:, None, :] - p[None, :, :], axis=2)
            cov = dd < r[None, :]
            cov[:, [i, j]] = False
            free = ~cov.any(axis=1)
            # a sampled point clear of every ball by a margin decides
            margin = (dd - r[None, :]).min(axis=1, initial=np.inf, where=~np.isin(np.arange(n), [i, j])[None, :])
            if np.any(free & (margin > 1e-9)):
                assert (i, j) in reported, (i, j)


def test_sphere_uncovered_simple_cases(orc):
    # alone; inside a larger ball (either sign); two overlapping equal balls
    assert list(orc.sphere_uncovered(np.zeros((1, 3)), np.array([0.3]))) == [1]
    p = np.array([[0.0, 0, 0], [0.05, 0, 0]])
    for big in (0.5, -0.5):
        assert list(orc.sphere_uncovered(p, np.array([big, 0.2]))) == [1, 0]
    p = np.array([[0.0, 0, 0], [0.3, 0, 0]])
    assert list(orc.sphere_uncovered(p, np.array([0.25, 0.25]))) == [1, 1]
    # zero samples: uncovered exactly when the point is outside the others
    p = np.array([[0.0, 0, 0], [0.1, 0, 0], [0.9, 0, 0]])
    assert list(orc.sphere_uncovered(p, np.array([0.5, 0.0, 0.0]))) == [1, 0, 1]


@pytest.mark.parametrize("case", ["inflated_grid", "invalid0", "invalid2"])
def test_sphere_uncovered_bounds_the_discrete_survivors(orc, case):
    """A sphere with a surviving icosphere candidate has an uncovered point,
    and the candidate sets are nested in tau, so the spheres with survivors
    grow with tau and stay inside the exact set (no box culling).  Inputs
    with covered spheres: the 8^3 sphere grid with every value scaled by 1.2
    (211 of 512 spheres keep an uncovered point; 9, 14, 50, 128, 163 of them
    have survivors at tau = 0..4), and invalid tiny random inputs."""
    if case == "inflated_grid":
        w = W.sphere_grid(N=8, up=2, tau=2)
        p, s = w.p, 1.2 * w.s
    else:
        p, s = W.tiny_random(40, int(case[-1]), valid=False, spread=0.35)
    exact = orc.sphere_uncovered(p, s).astype(bool)
    if case == "inflated_grid":
        assert exact.sum() == 211      # regression value of this oracle, not a pin
    prev = None
    for tau in range(0, 5):
        U = orc.icosphere(tau)
        keep = orc.keep_all(p, s, U, box_cull=False).reshape(len(s), -1)
        has = keep.any(axis=1)
        assert np.all(exact[has])
        if prev is not None:
            assert np.all(has[prev])
        prev = has
    assert exact.sum() >= prev.sum()


# ----------------------------------------------------------------------------
# the point q* that sets each value
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(4))
def test_argmin_points_set_the_values(orc, seed):
    """q* from the argmin and code: its distance to x is the value (bitwise
    where the value is the distance to a candidate or a tangent point, to
    rounding where it is d - r or r - d), it lies on its sphere, OUTSIDE
    gives x itself and SAMPLE / INVALID give NaN."""
    p, s = W.tiny_random(30, seed, valid=(seed % 2 == 0), spread=0.6)
    rng = np.random.default_rng(50 + seed)
    x = np.concatenate([rng.uniform(-1.2, 1.2, size=(300, 3)), p[:5]])
    U = orc.icosphere(2)
    K = U.shape[0]
    surv = orc.collect(p, s, U, orc.keep_all(p, s, U))
    for val, arg, fl in (orc.query(p, s, surv, x)[:3], orc.query_aug(p, s, surv, x)):
        q = orc.argmin_points(p, s, U, x, arg, fl)
        code = fl & 15
        seen = set()
        for t in range(x.shape[0]):
            c = int(code[t])
            seen.add(c)
            dx, dy, dz = x[t, 0] - q[t, 0], x[t, 1] - q[t, 1], x[t, 2] - q[t, 2]
            d = np.sqrt(dx * dx + dy * dy + dz * dz)
            if c in (orc.CODE_SURVIVOR, orc.CODE_TANGENT):
                assert d == abs(val[t])
                j = arg[t] // (K + 1) if c == orc.CODE_SURVIVOR else arg[t] // 2
                assert abs(np.linalg.norm(q[t] - p[j]) - abs(s[j])) < 1e-12
            elif c in (orc.CODE_OPPOSITE, orc.CODE_LOWER) and arg[t] >= 0:
                assert abs(d - abs(val[t])) < 1e-12 or (val[t] == 0 and c == orc.CODE_LOWER)
                assert abs(np.linalg.norm(q[t] - p[arg[t]]) - abs(s[arg[t]])) < 1e-12
            elif c == orc.CODE_OUTSIDE:
                assert np.array_equal(q[t], x[t])
            else:
                assert np.all(np.isnan(q[t]))
        assert {orc.CODE_OUTSIDE, orc.CODE_SAMPLE} <= seen and seen & {orc.CODE_SURVIVOR, orc.CODE_OPPOSITE, orc.CODE_TANGENT}


# ----------------------------------------------------------------------------
# scored value (Sec. 3.3): closed forms, hand-worked cases, validity after
# insertion
# ----------------------------------------------------------------------------

def _scored(orc, p, s, x, tau=2):
    U = orc.icosphere(tau)
    surv = orc.collect(p, s, U, orc.keep_all(p, s, U))
    return orc.query_scored(p, s, surv, np.atleast_2d(x)), surv, U


@pytest.mark.parametrize("sign", [1.0, -1.0])
@pytest.mark.parametrize("xpt", [(0.1, 0.0, 0.0), (0.8, 0.0, 0.0), (0.05, -0.3, 0.2), (-0.6, 0.4, 0.1)])
def test_scored_single_sphere_is_the_lipschitz_maximum(orc, sign, xpt):
    """One sample: every value within the Lipschitz bound of it is consistent,
    and the score prefers tangency points whose normals agree, then the
    largest radius: the far tangent point, value sign(s) (|x - p| + |s|)."""
    p = np.array([[0.02, -0.01, 0.03]])
    s = np.array([sign * 0.5])
    (v, a, f), _, _ = _scored(orc, p, s, xpt)
    d = np.linalg.norm(np.asarray(xpt) - p[0])
    assert f[0] & 15 == orc.CODE_TANGENT and a[0] == 1            # sphere 0, far side
    assert abs(v[0] - sign * (d + 0.5)) < 1e-15


def test_scored_two_spheres_hand_worked(orc):
    """Two positive spheres A (r 0.2 at 0) and B (r 0.05 at (0.5,0,0)), x at
    (0.3,0,0) outside both: A's far tangent point (radius 0.5) would strictly
    enclose B (far bound 0.25); B's far tangent point (radius 0.25) agrees
    and is valid; the negative radii are capped at 0.1 by the positive
    spheres (A's near tangent, score 2 * 0.1 < 0.25)."""
    p = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0]])
    s = np.array([0.2, 0.05])
    (v, a, f), _, _ = _scored(orc, p, s, (0.3, 0.0, 0.0))
    assert f[0] & 15 == orc.CODE_TANGENT and a[0] == 2 * 1 + 1
    assert abs(v[0] - 0.25) < 1e-15


def test_scored_prefers_negative_radii(orc):
    """x halfway between a positive and a negative sphere (both r 0.1 at
    distance 0.3): the near tangent points of both agree for one sign each
    at radius 0.2; the negative one scores 2 * 0.2 and wins."""
    p = np.array([[-0.3, 0.0, 0.0], [0.3, 0.0, 0.0]])
    s = np.array([0.1, -0.1])
    (v, a, f), _, _ = _scored(orc, p, s, (0.0, 0.0, 0.0))
    assert f[0] & 15 == orc.CODE_TANGENT and a[0] == 0
    assert abs(v[0] + 0.2) < 1e-15


def test_scored_fallback_without_candidates(orc):
    """A ball larger than the box: its candidates and tangent points all lie
    outside the box, so no grow-to point exists; the plain query's value (the
    lower bound) is kept and flagged."""
    p = np.array([[0.1, 0.05, -0.1]])
    s = np.array([-3.0])
    x = np.array([[0.2, 0.1, 0.0]])
    (v, a, f), surv, _ = _scored(orc, p, s, x, tau=1)
    v0, a0, f0, _ = orc.query(p, s, surv, x)
    assert f[0] == f0[0] | orc.FLAG_SCORE_FALLBACK and v[0] == v0[0] and a[0] == a0[0]


def test_scored_values_keep_the_samples_valid(orc):
    """On random valid inputs, each scored sample added to the inputs (and
    the P build redone from scratch) keeps every other sphere's surviving
    candidates (some survive), intersects no opposite ball, and its grow-to
    point lies on its sphere outside every input ball."""
    rng = np.random.default_rng(41)
    w = W.sphere_grid(N=6, up=2)
    U = orc.icosphere(1)
    K = U.shape[0]
    keep = orc.keep_all(w.p, w.s, U)
    surv = orc.collect(w.p, w.s, U, keep)
    had = keep.sum(axis=1) > 0
    x = rng.uniform(-0.9, 0.9, size=(25, 3))
    v, a, f = orc.query_scored(w.p, w.s, surv, x)
    tested = 0
    for t in range(x.shape[0]):
        code = f[t] & 15
        if code not in (orc.CODE_SURVIVOR, orc.CODE_TANGENT):
            continue
        i = a[t] // (K + 1) if code == orc.CODE_SURVIVOR else a[t] // 2
        p2 = np.vstack([w.p, x[t]])
        s2 = np.append(w.s, v[t])
        keep2 = orc.keep_all(p2, s2, U)
        others = had.copy()
        others[i] = False
        assert np.all(keep2[:-1][others].sum(axis=1) > 0), t
        opp = np.sign(w.s) == -np.sign(v[t])
        dist = np.linalg.norm(w.p - x[t], axis=1)
        assert np.all(dist[opp] >= abs(v[t]) + np.abs(w.s[opp]) - 1e-6 - 1e-12)
        tested += 1
    assert tested >= 15


def test_scored_far_bound_excludes_enclosing_a_covered_sphere(orc):
    """A small positive sphere C inside the ball of a larger one A has no
    survivor; x outside both.  A's far tangent point (radius 0.8) would
    strictly enclose C (far bound 0.55) and is invalid although no survivor
    is lost; the best valid candidate is A's near tangent point with the
    negative radius 0.2 (its normals agree; score 2 * 0.2)."""
    p = np.array([[0.0, 0.0, 0.0], [0.05, 0.0, 0.0]])
    s = np.array([0.3, 0.1])
    (v, a, f), surv, _ = _scored(orc, p, s, (0.5, 0.0, 0.0))
    assert not np.any(surv[1] == 1)                     # C keeps no survivor
    assert f[0] & 15 == orc.CODE_TANGENT and a[0] == 0
    assert abs(v[0] + 0.2) < 1e-15
