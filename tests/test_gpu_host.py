"""The host-buffer entry point (gfs_solve_host): the upload of the query
points runs on a second stream and overlaps the build.  Its results must
equal those of the device-buffer calls bit for bit, and a sample of them the
oracle's.
"""
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


@pytest.mark.parametrize("x32", [False, True])
def test_solve_host_equals_device_path(G, orc, x32):
    w = W.sphere_grid(N=24, tau=2)
    m = (1 << 22) + 12345
    x = np.random.default_rng(7).uniform(-1.1, 1.1, size=(m, 3))
    x = x.astype(np.float32) if x32 else x
    ctx = G.Context(tau=w.tau)
    ctx.build(torch.from_numpy(w.p).cuda(), torch.from_numpy(w.s).cuda())
    dev = ctx.query(torch.from_numpy(x).cuda())
    ref = {k: v.cpu().numpy() for k, v in dev.items() if v is not None}
    ctx.close()
    ph = torch.from_numpy(w.p).pin_memory()
    sh = torch.from_numpy(w.s).pin_memory()
    xh = torch.from_numpy(x).pin_memory()
    so = torch.empty(m, dtype=torch.float32).pin_memory()
    ao = torch.empty(m, dtype=torch.int64).pin_memory()
    fo = torch.empty(m, dtype=torch.int16).pin_memory()
    hctx = G.Context(tau=w.tau)
    for _ in range(2):   # the second call reuses the context's buffers and stream
        so.fill_(-7.0)
        ao.fill_(-7)
        fo.fill_(-7)
        hctx.solve_host(ph, sh, xh, so, ao, fo)
        assert np.array_equal(so.numpy(), ref["s"], equal_nan=True)
        assert np.array_equal(ao.numpy(), ref["argmin"])
        assert np.array_equal(fo.numpy(), ref["flags"])
    hctx.close()
    # a sample against the oracle
    U = orc.icosphere(w.tau)
    keep = orc.keep_all(w.p, w.s, U)
    surv = orc.collect(w.p, w.s, U, keep)
    sel = np.unique(np.concatenate([np.random.default_rng(8).choice(m, 200, replace=False), [0, m - 1]]))
    val, arg, fl, _ = orc.query(w.p, w.s, surv, x[sel].astype(np.float64))
    assert np.array_equal(ao.numpy()[sel], arg)
    assert np.array_equal(fo.numpy()[sel].astype(np.int32) & 0xFFFF, fl)
    assert np.array_equal(so.numpy()[sel], val.astype(np.float32), equal_nan=True)
