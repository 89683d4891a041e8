"""The point q* that sets each value (gfs_query_points) on the GPU against
the oracle, bit for bit, for the plain and the tangent-augmented query."""
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


@pytest.mark.parametrize("tangent", [False, True])
def test_argmin_points_parity(G, orc, tangent):
    w = W.sphere_grid(N=10, up=2, tau=2)
    x = w.make_queries()
    U = orc.icosphere(w.tau)
    surv = orc.collect(w.p, w.s, U, orc.keep_all(w.p, w.s, U))
    if tangent:
        val, arg, fl = orc.query_aug(w.p, w.s, surv, x)
    else:
        val, arg, fl, _ = orc.query(w.p, w.s, surv, x)
    want = orc.argmin_points(w.p, w.s, U, x, arg, fl)
    ctx = G.Context(tau=w.tau, tangent=tangent)
    ctx.build(torch.from_numpy(w.p).cuda(), torch.from_numpy(w.s).cuda())
    xt = torch.from_numpy(x).cuda()
    out = ctx.query(xt)
    assert np.array_equal(out["argmin"].cpu().numpy(), arg)
    got = ctx.query_points(xt, out["argmin"], out["flags"]).cpu().numpy()
    ctx.close()
    assert np.array_equal(got, want, equal_nan=True)
    # |x - q*| is the value where the value is a distance to a point
    code = fl & 15
    sel = (code == G.CODE_SURVIVOR) | (code == G.CODE_TANGENT)
    d = np.sqrt(((x[sel] - got[sel]) ** 2).sum(axis=1))
    assert np.allclose(d, np.abs(val[sel]), rtol=1e-14, atol=1e-15)
