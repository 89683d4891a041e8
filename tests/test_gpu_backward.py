"""Adjoint of the consistent value (a hand-written backward kernel behind
torch.autograd.Function) against the oracle's analytic gradient at the
oracle's argmin, and against central finite differences of the GPU forward
pass away from argmin switches."""
import numpy as np
import pytest
import torch

from paper_2605_01919_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2605_01919_gb300 import gfs
    gfs.load()
    return gfs


def _setup(G, orc, p, s, tau, x):
    U = orc.icosphere(tau)
    keep = orc.keep_all(p, s, U)
    surv = orc.collect(p, s, U, keep)
    val, arg, fl, gap = orc.query(p, s, surv, x)
    ctx = G.Context(tau=tau)
    pt = torch.from_numpy(p).cuda().requires_grad_(True)
    st = torch.from_numpy(s).cuda().requires_grad_(True)
    ctx.build(pt.detach(), st.detach())
    return U, surv, (val, arg, fl, gap), ctx, pt, st


@pytest.mark.parametrize("which", ["sphere", "torus"])
def test_backward_matches_oracle_gradient(G, orc, which):
    if which == "sphere":
        w = W.sphere_grid()
        x = w.make_queries()
    else:
        w = W.torus_grid(N=20, m=5000)
        x = w.make_queries().astype(np.float64)
    U, surv, (val, arg, fl, gap), ctx, pt, st = _setup(G, orc, w.p, w.s, w.tau, x)
    rng = np.random.default_rng(5)
    gup = rng.normal(size=x.shape[0])
    gx_o, gp_o, gs_o = orc.grad(w.p, w.s, U, x, val, arg, fl, gup)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    sv = G.ConsistentSDF.apply(xt, pt, st, ctx)
    sv.backward(torch.from_numpy(gup).float().cuda())
    gx = xt.grad.cpu().numpy()
    gp = pt.grad.cpu().numpy()
    gs = st.grad.cpu().numpy()
    # per-query gradient: FP32 output of an FP64 evaluation
    assert np.max(np.abs(gx - gx_o)) < 1e-5 * max(1.0, np.abs(gup).max())
    # per-sample sums: 64-bit fixed point (2^-40) over many queries
    scale = np.abs(gup).sum()
    assert np.max(np.abs(gp - gp_o)) < 1e-6 * scale + 1e-5
    assert np.max(np.abs(gs - gs_o)) < 1e-6 * scale + 1e-5
    ctx.close()


def test_backward_deterministic(G):
    w = W.sphere_grid()
    x = torch.from_numpy(w.make_queries()).cuda()
    ctx = G.Context(tau=w.tau)
    ctx.build(torch.from_numpy(w.p).cuda(), torch.from_numpy(w.s).cuda())
    out = ctx.query(x)
    g = torch.linspace(-1, 1, x.shape[0], device="cuda")
    r1 = ctx.backward(x, out["s"], out["argmin"], out["flags"], g)
    r2 = ctx.backward(x, out["s"], out["argmin"], out["flags"], g)
    for a, b in zip(r1, r2):
        assert torch.equal(a, b)
    ctx.close()


H_FD = 1e-4        # central-difference step (the differentiable workload's stated h)
TIE = 1e-5         # points whose two nearest candidates lie within this are skipped


def _fd_tol(v):
    """Bound on |central difference - derivative| for a distance-like value
    v: the truncation error of a central difference is at most h^2/6 times
    the third derivative, which is at most 3/d^2 for a distance d >= |v| to a
    point or a sphere centre; twice that, plus the FP32 rounding of the
    kernel's output."""
    return 1e-6 + H_FD * H_FD / np.maximum(np.abs(v), 1e-3) ** 2


def _gpu_value(G, tau, p, s, x):
    ctx = G.Context(tau=tau)
    ctx.build(torch.from_numpy(p).cuda(), torch.from_numpy(s).cuda())
    out = ctx.query(torch.from_numpy(x).cuda())
    res = (out["s64"].cpu().numpy(), out["argmin"].cpu().numpy(),
           out["flags"].cpu().numpy().astype(np.int32) & 15)
    ctx.close()
    return res


def test_backward_central_differences(G, orc):
    """d s*/dx, d s*/dp_j and d s*/ds_j of the GPU adjoint against central
    differences (h = 1e-4) of the GPU forward pass (rebuilt for p and s).

    Skipped, and only these: points whose two nearest candidates lie within
    1e-5 (oracle gap), and points whose argmin or result code changes between
    the two sides of the stencil (a tie crossed inside it: the difference then
    mixes two branches and is no derivative).  Every other point must agree
    within the truncation bound of _fd_tol."""
    w = W.torus_grid(N=20, m=3000)
    x = w.make_queries().astype(np.float64)
    U, surv, (val, arg, fl, gap), ctx, pt, st = _setup(G, orc, w.p, w.s, w.tau, x)
    ok = np.isin(fl & 15, [0, 1]) & (gap > TIE)
    xs = x[ok][:600]
    xt = torch.from_numpy(xs).cuda()
    out = ctx.query(xt)
    v0 = out["s64"].cpu().numpy()
    a0 = out["argmin"].cpu().numpy()
    c0 = out["flags"].cpu().numpy().astype(np.int32) & 15
    gx, _, _ = ctx.backward(xt, out["s"], out["argmin"], out["flags"], torch.ones(xs.shape[0], device="cuda"),
                            want_p=False, want_s=False)
    g = gx.cpu().numpy()
    h = H_FD
    checked = 0
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        op = ctx.query(torch.from_numpy(xs + e).cuda())
        om = ctx.query(torch.from_numpy(xs - e).cuda())
        same = ((op["argmin"].cpu().numpy() == a0) & (om["argmin"].cpu().numpy() == a0)
                & ((op["flags"].cpu().numpy().astype(np.int32) & 15) == c0)
                & ((om["flags"].cpu().numpy().astype(np.int32) & 15) == c0))
        fd = (op["s64"].cpu().numpy() - om["s64"].cpu().numpy()) / (2 * h)
        err = np.abs(fd - g[:, c])
        bad = same & (err > _fd_tol(v0))
        assert not bad.any(), (np.nonzero(bad)[0][:5], err[bad][:5])
        checked += int(same.sum())
    assert checked >= 0.75 * 3 * xs.shape[0], checked

    # sample derivatives: one backward over points that all set their value
    # from different samples, so each sample's gradient is one point's
    K = U.shape[0]
    sphere = np.where(c0 == 0, a0 // (K + 1), a0)
    _, first = np.unique(sphere, return_index=True)
    pick = np.sort(first)[:24]
    gup = np.zeros(xs.shape[0])
    gup[pick] = 1.0
    _, gp, gs = ctx.backward(xt, out["s"], out["argmin"], out["flags"], torch.from_numpy(gup).float().cuda(),
                             want_x=False)
    gp = gp.cpu().numpy()
    gs = gs.cpu().numpy()
    ctx.close()
    tested = 0
    for t in pick:
        j = sphere[t]
        for which in range(4):
            pp, pm, sp, sm = w.p.copy(), w.p.copy(), w.s.copy(), w.s.copy()
            if which < 3:
                pp[j, which] += h
                pm[j, which] -= h
            else:
                sp[j] += h
                sm[j] -= h
            vp, ap, cp = _gpu_value(G, w.tau, pp, sp, xs[t][None])
            vm, am, cm = _gpu_value(G, w.tau, pm, sm, xs[t][None])
            if not (ap[0] == a0[t] == am[0] and cp[0] == c0[t] == cm[0]):
                continue
            fd = (vp[0] - vm[0]) / (2 * h)
            an = gp[j, which] if which < 3 else gs[j]
            assert abs(fd - an) <= _fd_tol(v0[t]), (t, j, which, fd, an)
            tested += 1
    assert tested >= 0.6 * 4 * pick.shape[0], tested


def test_backward_lower_branch(G, orc):
    """LOWER results (no candidate: value = sign * the depth of the deepest
    containing ball) differentiate like the oracle's branch, and like central
    differences of the GPU forward pass."""
    for sign in (1.0, -1.0):
        p = np.array([[0.1, 0.05, -0.1], [-0.2, 0.1, 0.15]])
        s = sign * np.array([3.0, 2.5])
        x = np.random.default_rng(29).uniform(-0.6, 0.6, size=(64, 3))
        U, surv, (val, arg, fl, gap), ctx, pt, st = _setup(G, orc, p, s, 1, x)
        assert np.all(fl & 15 == orc.CODE_LOWER)
        gup = np.random.default_rng(31).normal(size=x.shape[0])
        gx_o, gp_o, gs_o = orc.grad(p, s, U, x, val, arg, fl, gup)
        xt = torch.from_numpy(x).cuda()
        out = ctx.query(xt)
        assert np.array_equal(out["s64"].cpu().numpy(), val)
        gx, gp, gs = ctx.backward(xt, out["s"], out["argmin"], out["flags"], torch.from_numpy(gup).float().cuda())
        assert np.max(np.abs(gx.cpu().numpy() - gx_o)) < 1e-5 * np.abs(gup).max()
        scale = np.abs(gup).sum()
        assert np.max(np.abs(gp.cpu().numpy() - gp_o)) < 1e-6 * scale + 1e-5
        assert np.max(np.abs(gs.cpu().numpy() - gs_o)) < 1e-6 * scale + 1e-5
        g1, _, _ = ctx.backward(xt, out["s"], out["argmin"], out["flags"], torch.ones(x.shape[0], device="cuda"),
                                want_p=False, want_s=False)
        g1 = g1.cpu().numpy()
        for c in range(3):
            e = np.zeros(3)
            e[c] = H_FD
            vp = ctx.query(torch.from_numpy(x + e).cuda())["s64"].cpu().numpy()
            vm = ctx.query(torch.from_numpy(x - e).cuda())["s64"].cpu().numpy()
            assert np.all(np.abs((vp - vm) / (2 * H_FD) - g1[:, c]) <= _fd_tol(val))
        ctx.close()


def test_consistent_sdf_rejects_other_or_changed_samples(G):
    """ConsistentSDF differentiates the state the context holds: sample
    tensors other than the built ones, or changed in place since the build,
    are refused instead of giving values of one state and gradients for
    another."""
    w = W.sphere_grid(N=8, up=2)
    p = torch.from_numpy(w.p).cuda().requires_grad_(True)
    s = torch.from_numpy(w.s).cuda().requires_grad_(True)
    ctx = G.Context(tau=w.tau)
    ctx.build(p.detach(), s.detach())
    x = torch.from_numpy(w.make_queries()[:100]).cuda()
    G.ConsistentSDF.apply(x, p, s, ctx)                     # the built tensors: accepted
    with pytest.raises(G.GfsError):
        G.ConsistentSDF.apply(x, p, s.detach().clone(), ctx)
    with torch.no_grad():
        s.mul_(1.0)                                        # in-place change bumps the version
    with pytest.raises(G.GfsError):
        G.ConsistentSDF.apply(x, p, s, ctx)
    ctx.close()
