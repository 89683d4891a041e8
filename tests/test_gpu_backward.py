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


def test_backward_central_differences(G, orc):
    """d s*/dx by central differences (h = 1e-4) of the GPU forward pass, at
    points whose two nearest candidates are more than 1e-3 apart (the
    gradient is piecewise smooth between argmin switches)."""
    w = W.torus_grid(N=20, m=3000)
    x = w.make_queries().astype(np.float64)
    U, surv, (val, arg, fl, gap), ctx, pt, st = _setup(G, orc, w.p, w.s, w.tau, x)
    ok = ((fl & 15) <= 1) & (gap > 1e-3)
    xs = x[ok][:400]
    xt = torch.from_numpy(xs).cuda()
    out = ctx.query(xt)
    gx, _, _ = ctx.backward(xt, out["s"], out["argmin"], out["flags"], torch.ones(xs.shape[0], device="cuda"),
                            want_p=False, want_s=False)
    h = 1e-4
    fd = np.zeros_like(xs)
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        vp = ctx.query(torch.from_numpy(xs + e).cuda())["s64"].cpu().numpy()
        vm = ctx.query(torch.from_numpy(xs - e).cuda())["s64"].cpu().numpy()
        fd[:, c] = (vp - vm) / (2 * h)
    g = gx.cpu().numpy()
    same = np.all(np.abs(fd - g) < 1e-3, axis=1)
    # a few points may still straddle an argmin switch within h
    assert same.mean() > 0.97, same.mean()
    ctx.close()
