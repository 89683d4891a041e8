"""The backward entry point that allocates no device memory.

Some callers cannot allocate: code running while a CUDA graph is being
captured, and runtimes that reserve device memory once at start-up.  For them
gfs_query_backward_noalloc keeps its scratch (per-sample fixed-point sums) in
a static device array instead of a context-owned buffer.  This test calls it
through the C ABI on fresh contexts of two sizes (the second call must not
see the first call's sums) and inside a captured CUDA graph, and checks every
call bit for bit against gfs_query_backward; it also checks the size limit.
It sits in a file of its own that pytest collects last.
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


def _context(G, w):
    ctx = G.Context(tau=w.tau)
    ctx.build(torch.from_numpy(w.p).cuda(), torch.from_numpy(w.s).cuda())
    return ctx


def test_noalloc_backward_matches_allocating_entry_point(G):
    """Fresh contexts, the no-alloc call first (before any allocating
    backward could grow the context's buffer): no device memory is taken,
    and the results are bit-identical to gfs_query_backward (the same
    kernels and deterministic fixed-point sums).  The second context is
    smaller than the first, so its call must clear what the first left in
    the static array."""
    rng = np.random.default_rng(8)
    for w in (W.sphere_grid(), W.sphere_grid(N=8, up=2, tau=2)):
        x = torch.from_numpy(w.make_queries()).cuda()
        ctx = _context(G, w)
        out = ctx.query(x)
        g = torch.from_numpy(rng.normal(size=x.shape[0])).float().cuda()
        m, n = x.shape[0], ctx.n
        got = (torch.empty((m, 3), dtype=torch.float32, device="cuda"),
               torch.empty((n, 3), dtype=torch.float32, device="cuda"),
               torch.empty(n, dtype=torch.float32, device="cuda"))
        L = G.load()

        def call():
            ctx._sync_stream()
            return L.gfs_query_backward_noalloc(ctx._h, x.data_ptr(), 0, m, out["s"].data_ptr(),
                                                out["argmin"].data_ptr(), out["flags"].data_ptr(), g.data_ptr(),
                                                got[0].data_ptr(), got[1].data_ptr(), got[2].data_ptr())
        assert call() == 0                          # the first call on a device looks up the array's address
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        assert call() == 0
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0       # nothing allocated by the call
        ref = ctx.backward(x, out["s"], out["argmin"], out["flags"], g)
        torch.cuda.synchronize()
        for a, b in zip(got, ref):
            assert torch.equal(a, b)
        ctx.close()


def test_noalloc_backward_in_cuda_graph(G):
    """Captured in a CUDA graph on the context's stream and replayed with two
    different upstream gradients: each replay equals gfs_query_backward bit
    for bit."""
    w = W.sphere_grid()
    x = torch.from_numpy(w.make_queries()).cuda()
    ctx = _context(G, w)
    out = ctx.query(x)
    m, n = x.shape[0], ctx.n
    g = torch.zeros(m, dtype=torch.float32, device="cuda")
    gx = torch.empty((m, 3), dtype=torch.float32, device="cuda")
    gp = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    gs = torch.empty(n, dtype=torch.float32, device="cuda")
    L = G.load()

    def call():
        ctx._sync_stream()
        return L.gfs_query_backward_noalloc(ctx._h, x.data_ptr(), 0, m, out["s"].data_ptr(),
                                            out["argmin"].data_ptr(), out["flags"].data_ptr(), g.data_ptr(),
                                            gx.data_ptr(), gp.data_ptr(), gs.data_ptr())
    assert call() == 0                              # outside capture: the device address lookup
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        st = call()
    assert st == 0
    rng = np.random.default_rng(10)
    for _ in range(2):
        g.copy_(torch.from_numpy(rng.normal(size=m)).float())
        graph.replay()
        torch.cuda.synchronize()
        ref = ctx.backward(x, out["s"], out["argmin"], out["flags"], g)
        torch.cuda.synchronize()
        for a, b in zip((gx, gp, gs), ref):
            assert torch.equal(a, b)
    ctx._sync_stream()
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
