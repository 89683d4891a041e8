"""The backward entry point that allocates no device memory.

Some callers cannot allocate: code running while a CUDA graph is being
captured, and runtimes that reserve device memory once at start-up.  For them
gfs_query_backward_noalloc keeps its scratch (per-sample fixed-point sums) in
a static device array instead of a context-owned buffer.  This test calls it
through the C ABI twice in a row (the second call must not see the first
call's sums) and checks both calls against gfs_query_backward; it also checks
the size limit.  It sits in a file of its own that pytest collects last.
"""
import ctypes

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
    L = gfs.load()
    P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.gfs_query_backward_noalloc.argtypes = [P, P, i32, i64, P, P, P, P, P, P, P]
    L.gfs_query_backward_noalloc.restype = i32
    return gfs


def _noalloc(G, ctx, x, out, g):
    m, n = x.shape[0], ctx.n
    gx = torch.empty((m, 3), dtype=torch.float32, device="cuda")
    gp = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    gs = torch.empty(n, dtype=torch.float32, device="cuda")
    ctx._sync_stream()
    st = G.load().gfs_query_backward_noalloc(ctx._h, x.data_ptr(), 0, m, out["s"].data_ptr(),
                                             out["argmin"].data_ptr(), out["flags"].data_ptr(), g.data_ptr(),
                                             gx.data_ptr(), gp.data_ptr(), gs.data_ptr())
    assert st == 0, G.load().gfs_strerror(st)
    return gx, gp, gs


def test_noalloc_backward_matches_allocating_entry_point(G):
    w = W.sphere_grid()
    x = torch.from_numpy(w.make_queries()).cuda()
    ctx = G.Context(tau=w.tau)
    ctx.build(torch.from_numpy(w.p).cuda(), torch.from_numpy(w.s).cuda())
    out = ctx.query(x)
    rng = np.random.default_rng(8)
    for call in range(2):   # two calls in a row: the static sums start from zero each time
        g = torch.from_numpy(rng.normal(size=x.shape[0])).float().cuda()
        ref = ctx.backward(x, out["s"], out["argmin"], out["flags"], g)
        got = _noalloc(G, ctx, x, out, g)
        torch.cuda.synchronize()
        scale = float(g.abs().sum())
        assert float((got[0] - ref[0]).abs().max()) < 1e-5 * max(1.0, float(g.abs().max()))
        assert float((got[1] - ref[1]).abs().max()) < 1e-6 * scale + 1e-5
        assert float((got[2] - ref[2]).abs().max()) < 1e-6 * scale + 1e-5
    ctx.close()


def test_noalloc_backward_rejects_too_many_spheres(G):
    n = 262144 + 1                           # GFS_NOALLOC_MAX_SPHERES + 1
    rng = np.random.default_rng(9)
    p = torch.from_numpy(rng.uniform(-1, 1, size=(n, 3))).cuda()
    s = torch.from_numpy(rng.uniform(0.001, 0.01, size=n)).cuda()
    ctx = G.Context(tau=0)
    ctx.build(p, s)
    x = p[:16].contiguous()
    out = ctx.query(x)
    g = torch.ones(16, device="cuda")
    dummy = torch.empty(4 * n, device="cuda")
    ctx._sync_stream()
    st = G.load().gfs_query_backward_noalloc(ctx._h, x.data_ptr(), 0, 16, out["s"].data_ptr(),
                                             out["argmin"].data_ptr(), out["flags"].data_ptr(), g.data_ptr(),
                                             dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr())
    assert st == 6                           # GFS_ERR_TOO_LARGE
    ctx.close()
