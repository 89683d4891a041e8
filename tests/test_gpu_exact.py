"""Exact uncovered test per sphere (gfs_sphere_uncovered, Prop. 1 (ii)) on
the GPU against the oracle's brute force, sphere by sphere; the witnesses
of uncovered spheres; at 64^3 the properties that hold at any size: a
sphere with an icosphere survivor is uncovered, every witness lies on its
sphere outside every other shrunk ball, and every point of a fine
icosphere on a covered sphere lies in another shrunk ball."""
import numpy as np
import pytest
import torch

from paper_2605_01919_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.widening, pytest.mark.timeout(900)]


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2605_01919_gb300 import gfs
    gfs.load()
    return gfs


def gpu_uncovered(G, p, s, tau=1, tol=1e-6, witness=False):
    ctx = G.Context(tau=tau, tol=tol)
    ctx.build(torch.from_numpy(np.ascontiguousarray(p)).cuda(), torch.from_numpy(np.ascontiguousarray(s)).cuda())
    out, wit = ctx.sphere_uncovered(witness=True)
    out, wit = out.cpu().numpy(), wit.cpu().numpy()
    surv = ctx.survivors().cpu().numpy()
    ctx.close()
    return (out, surv, wit) if witness else (out, surv)


def check_witness(p, s, tol, i, t):
    """t lies on sphere i and in no other shrunk ball beyond rounding (it is
    built on up to two other spheres, which the test leaves out)."""
    assert abs(np.linalg.norm(t - p[i]) - abs(s[i])) <= 1e-9 * (1 + abs(s[i])), i
    d = np.linalg.norm(p - t, axis=1)
    rho = np.abs(s) - tol
    inside = (d < rho - 1e-9) & (rho > 0)
    inside[i] = False
    assert not inside.any(), (i, np.nonzero(inside)[0][:4])


def test_exact_uncovered_parity(G, orc):
    e = np.eye(3)
    cases = [(np.concatenate([np.zeros((1, 3)), e, -e]), np.array([1.0] + [rho] * 6))
             for rho in (0.91, 0.9194, 0.9195, 0.93)]
    w = W.sphere_grid(N=8, up=2, tau=2)
    cases += [(w.p, 1.2 * w.s)]
    exact_sdf = (w.p, w.s)
    cases += [W.tiny_random(40, seed, valid=(seed % 2 == 0), spread=0.35) for seed in range(4)]
    cases.append((np.array([[0.0, 0, 0], [0.3, 0, 0]]), np.array([0.25, 0.25])))
    cases.append((np.array([[0.0, 0, 0], [0.1, 0, 0], [0.9, 0, 0], [0.0, 0, 0]]), np.array([0.5, 0.0, 0.0, 0.5])))
    # grids of SDF samples touch exactly: with tol = 0 some spheres keep only
    # tangency points, where rounding decides (the certificate and the full
    # enumeration may then differ); they are compared at the method's tol
    exact_touch = []
    for N in (6, 8, 10):
        w = W.csg_pseudo_grid(N=N, tau=1)
        exact_touch.append((w.p, w.s))
    exact_touch.append(exact_sdf)
    for (p, s), tols in [(c, (0.0, 1e-6)) for c in cases] + [(c, (1e-6,)) for c in exact_touch]:
        for tol in tols:
            got, _, wit = gpu_uncovered(G, p, s, tol=tol, witness=True)
            want = orc.sphere_uncovered(p, s, tol=tol)
            assert np.array_equal(got, want), np.nonzero(got != want)[0][:8]
            for i in np.nonzero(got == 1)[0]:
                check_witness(p, s, tol, i, wit[i])
            assert np.all(np.isnan(wit[got != 1]))


def test_exact_uncovered_contains_survivor_spheres(G):
    """8^3 sphere grid inflated by 1.2 (at most 235 balls meet a sphere;
    tau 3, no box culling): every sphere with a surviving candidate is
    uncovered, and there are more uncovered spheres than spheres with
    survivors."""
    w = W.sphere_grid(N=8, up=2, tau=2)
    s = 1.2 * w.s
    ctx = G.Context(tau=3, box_cull=False)
    ctx.build(torch.from_numpy(w.p).cuda(), torch.from_numpy(s).cuda())
    out = ctx.sphere_uncovered().cpu().numpy()
    surv = ctx.survivors().cpu().numpy()
    ctx.close()
    assert np.all(out != 2)
    has = np.zeros(w.n, dtype=bool)
    has[surv // (ctx.K + 1)] = True
    assert np.all(out[has] == 1)
    assert (out == 1).sum() > has.sum() and (out == 0).any()


def test_exact_uncovered_exact_sdf_samples(G):
    """Samples of an exact SDF form a valid input, so by Prop. 1 (ii) every
    sphere keeps an uncovered point: 12^3 sphere grid (up to 476 balls meet
    a sphere), all 1,728 spheres are uncovered; at tau 2 only some of them
    have icosphere survivors."""
    w = W.sphere_grid(N=12, up=2, tau=2)
    out, surv = gpu_uncovered(G, w.p, w.s, tau=2)
    assert np.all(out == 1)
    assert np.unique(surv // (10 * 4 ** 2 + 3)).size < w.n


def test_exact_uncovered_csg64_properties(G, orc):
    """The 64^3 CSG pseudo-SDF grid (262,144 spheres, thousands of balls meet
    a deep sphere): every sphere decided; spheres with icosphere survivors at
    tau 2 are uncovered; 300 sampled witnesses checked against all balls; on
    40 sampled covered spheres every vertex of a tau 4 icosphere lies in
    another shrunk ball."""
    w = W.csg_pseudo_grid(N=64, tau=2)
    tol = 1e-6
    out, surv, wit = gpu_uncovered(G, w.p, w.s, tau=2, tol=tol, witness=True)
    assert np.all(out != 2)
    has = np.zeros(w.n, dtype=bool)
    has[surv // (10 * 4 ** 2 + 3)] = True
    assert np.all(out[has] == 1)
    assert (out == 0).sum() > w.n // 2
    rng = np.random.default_rng(11)
    for i in rng.choice(np.nonzero(out == 1)[0], 300, replace=False):
        check_witness(w.p, w.s, tol, i, wit[i])
    U = orc.icosphere(4)
    rho = np.abs(w.s) - tol
    for i in rng.choice(np.nonzero(out == 0)[0], 40, replace=False):
        r = abs(w.s[i])
        d = np.linalg.norm(w.p - w.p[i], axis=1)
        near = np.nonzero((np.abs(d - r) < rho) & (rho > 0))[0]
        near = near[near != i]
        near = near[np.argsort(-rho[near], kind="stable")]     # large balls first: most points fall early
        pts = w.p[i] + r * U
        held = np.zeros(len(pts), dtype=bool)
        for c in range(0, len(near), 1024):
            blk = near[c:c + 1024]
            open_ = np.nonzero(~held)[0]
            dd = np.linalg.norm(pts[open_][:, None, :] - w.p[blk][None, :, :], axis=2)
            held[open_] |= (dd < rho[blk][None, :]).any(axis=1)
            if held.all():
                break
        assert held.all(), (i, int((~held).sum()))


def gpu_intersections(G, p, s, tol=1e-6):
    ctx = G.Context(tau=1, tol=tol)
    ctx.build(torch.from_numpy(np.ascontiguousarray(p)).cuda(), torch.from_numpy(np.ascontiguousarray(s)).cuda())
    circ, quads, pts, status = ctx.uncovered_intersections()
    uncov = ctx.sphere_uncovered().cpu().numpy()
    ctx.close()
    return circ.cpu().numpy(), quads.cpu().numpy(), pts.cpu().numpy(), status, uncov


def test_uncovered_intersections_parity(G, orc):
    """Uncovered circles and points (Sec. 4.1 U and D) against the oracle's
    full enumeration: the same sorted lists and the points bit for bit, on
    the triangle and octahedral cases, the inflated sphere grid and valid and
    invalid tiny random inputs for tol 0 and 1e-6, and on grids of exactly
    touching SDF samples (sphere, CSG) for tol 1e-6."""
    h = np.sqrt(3) / 2
    cases = [(np.array([[0.0, 0, 0], [1.0, 0, 0], [0.5, h, 0], [0.5, h / 3, 1.3]]), np.array([1.0, 1, 1, 0.6]))]
    e = np.eye(3)
    for rho in (0.91, 0.93):
        cases.append((np.concatenate([np.zeros((1, 3)), e, -e]), np.array([1.0] + [rho] * 6)))
    w = W.sphere_grid(N=6, up=2, tau=2)
    cases += [(w.p, 1.2 * w.s)]
    cases += [W.tiny_random(40, seed, valid=(seed % 2 == 0), spread=0.35) for seed in range(4)]
    # exactly touching SDF samples: at the method's tol only (see above)
    exact_touch = [(w.p, w.s)]
    for N in (6, 8):
        w = W.csg_pseudo_grid(N=N, tau=1)
        exact_touch.append((w.p, w.s))
    for (p, s), tols in [(c, (0.0, 1e-6)) for c in cases] + [(c, (1e-6,)) for c in exact_touch]:
        for tol in tols:
            wc, wq, wp = orc.uncovered_intersections(p, s, tol=tol)
            gc, gq, gp, status, _ = gpu_intersections(G, p, s, tol=tol)
            assert status == 0
            assert np.array_equal(gc, wc), (len(gc), len(wc))
            assert np.array_equal(gq, wq), (len(gq), len(wq))
            assert np.array_equal(gp, wp)


def test_uncovered_intersections_csg32_properties(G):
    """The 32^3 CSG pseudo-SDF grid (32,768 spheres): every circle and point
    lies on uncovered spheres; 2,000 sampled points lie on their three
    spheres and in no other shrunk ball; on 300 sampled cutting pairs of
    uncovered spheres that are not reported, every one of 360 points of the
    circle lies in another shrunk ball."""
    w = W.csg_pseudo_grid(N=32, tau=1)
    tol = 1e-6
    circ, quads, pts, status, uncov = gpu_intersections(G, w.p, w.s, tol=tol)
    assert status == 0 and len(circ) > 1000 and len(quads) > 1000
    assert np.all(uncov[circ.ravel()] != 0) and np.all(uncov[quads[:, :3].ravel()] != 0)
    assert np.all(circ[:, 0] < circ[:, 1]) and np.all((quads[:, 0] < quads[:, 1]) & (quads[:, 1] < quads[:, 2]))
    r = np.abs(w.s)
    rho = r - tol
    rng = np.random.default_rng(5)
    for k in rng.choice(len(quads), 2000, replace=False):
        i, j, m, _ = quads[k]
        q = pts[k]
        for a in (i, j, m):
            assert abs(np.linalg.norm(q - w.p[a]) - r[a]) < 1e-12
        d = np.linalg.norm(w.p - q, axis=1)
        inside = (d < rho - 1e-9) & (rho > 0)
        inside[[i, j, m]] = False
        assert not inside.any()
    reported = set(map(tuple, circ.tolist()))
    idx = np.nonzero(uncov != 0)[0]
    phi = np.linspace(0, 2 * np.pi, 360, endpoint=False)
    checked = 0
    for i in rng.permutation(idx):
        if checked >= 300:
            break
        d = np.linalg.norm(w.p - w.p[i], axis=1)
        cand = np.nonzero((d < r[i] + r) & (d > np.abs(r[i] - r)) & (np.arange(w.n) > i) & (uncov != 0))[0]
        cand = [j for j in cand if (i, j) not in reported]
        if not cand:
            continue
        j = int(rng.choice(cand))
        dv = w.p[j] - w.p[i]
        dd = np.linalg.norm(dv)
        mu = dv / dd
        al = (dd * dd + r[i] ** 2 - r[j] ** 2) / (2 * dd)
        rad = np.sqrt(r[i] ** 2 - al * al)
        u = np.cross(mu, [1.0, 0, 0] if abs(mu[0]) < 0.9 else [0, 1.0, 0])
        u /= np.linalg.norm(u)
        v = np.cross(mu, u)
        q = w.p[i] + al * mu + rad * (np.outer(np.cos(phi), u) + np.outer(np.sin(phi), v))
        near = np.nonzero(np.linalg.norm(w.p - (w.p[i] + al * mu), axis=1) < rho + rad)[0]
        near = near[(near != i) & (near != j) & (rho[near] > 0)]
        dq = np.linalg.norm(q[:, None, :] - w.p[near][None, :, :], axis=2)
        assert (dq < rho[near][None, :]).any(axis=1).all(), (i, j)
        checked += 1
    assert checked == 300


def test_exact_rmin_parity(G, orc):
    """Exact minimum valid radius over T, U, D (Sec. 6) on the GPU: equal to
    the oracle's brute force bit for bit, for both signs and no sign, with
    and without the box, on random and hand-made inputs (tol 0 and 1e-6)
    and on the 6^3 sphere grid (tol 1e-6)."""
    cases = [(W.tiny_random(n, seed, valid=(seed % 2 == 0), spread=0.35), (0.0, 1e-6))
             for n, seed in ((12, 0), (25, 1), (40, 2))]
    h = np.sqrt(3) / 2
    cases.append(((np.array([[0.0, 0, 0], [1.0, 0, 0], [0.5, h, 0], [0.5, h / 3, 1.3]]) * 0.5,
                   np.array([0.5, 0.5, 0.5, -0.3])), (0.0, 1e-6)))
    w = W.sphere_grid(N=6, up=2, tau=2)
    cases.append(((w.p, w.s), (1e-6,)))
    rng = np.random.default_rng(31)
    for (p, s), tols in cases:
        x = rng.uniform(-0.8, 0.8, size=(10, 3))
        for tol in tols:
            for box in (False, True):
                ctx = G.Context(tau=1, tol=tol, box_cull=box)
                ctx.build(torch.from_numpy(np.ascontiguousarray(p)).cuda(),
                          torch.from_numpy(np.ascontiguousarray(s)).cuda())
                for sg in (1, -1, 0):
                    got = ctx.exact_rmin(torch.from_numpy(x).cuda(),
                                         torch.full((x.shape[0],), sg, dtype=torch.int8, device="cuda")).cpu().numpy()
                    want = np.array([orc.exact_rmin(p, s, x[t], sg, tol=tol, box_cull=box) for t in range(len(x))])
                    assert np.array_equal(got, want), (tol, box, sg, got[got != want], want[got != want])
                ctx.close()


def test_exact_rmin_brackets_the_discrete_value(G):
    """The bracket LB <= exact r_min <= |s_tau| of the oracle's pins (valid
    input, no box: the survivors and the opposite tangent point are contour
    points, every contour point lies outside each containing ball) on
    random valid inputs of 300 samples (exact SDF of two spheres' union at
    random points), at every one of 400 random points where the plain query
    finds a survivor or an opposite tangent point, at the method's tol.
    (On grids of SDF samples, nested spheres touching at one surface point
    meet in "circles" a few ulps wide, whose decision rounding takes; the
    bracket is a statement about inputs in general position.)"""
    checked = 0
    for seed in range(3):
        p, s = W.tiny_random(300, 500 + seed, valid=True, spread=0.5)
        xs = np.random.default_rng(600 + seed).uniform(-0.5, 0.5, size=(400, 3))
        ctx = G.Context(tau=2, tol=1e-6, box_cull=False)
        ctx.build(torch.from_numpy(np.ascontiguousarray(p)).cuda(), torch.from_numpy(np.ascontiguousarray(s)).cuda())
        x = torch.from_numpy(xs).cuda()
        out = ctx.query(x)
        fl = out["flags"].cpu().numpy().astype(np.int32) & 0xFFFF
        v = out["s64"].cpu().numpy()
        ok = np.isin(fl & 15, [0, 1])
        sig = torch.from_numpy(np.sign(v).astype(np.int8)).cuda()
        rmin = ctx.exact_rmin(x, sig).cpu().numpy()
        ctx.close()
        assert np.all(np.isfinite(rmin[ok]))
        assert np.all(rmin[ok] <= np.abs(v[ok]) + 1e-9)
        for t in np.nonzero(ok)[0]:
            same = np.sign(s) == np.sign(v[t])
            lb = np.max(np.abs(s[same]) - np.linalg.norm(p[same] - xs[t], axis=1))
            assert lb <= rmin[t] + 1e-9
        assert np.mean(np.abs(v[ok]) - rmin[ok]) > 0
        checked += int(ok.sum())
    assert checked > 1000
