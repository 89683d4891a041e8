"""Batched shapes in one persistent launch: every shape's outputs equal the
single-shape path (bitwise) and, on small shapes, the oracle; the batched
query replays correctly from a captured CUDA graph."""
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


def _shapes(count, scale, tau):
    shapes = []
    for i in range(count):
        w = W.batch_shape(i, tau=tau, scale=scale)
        x = w.make_queries()
        if x.shape[0] > 40000:
            x = x[np.random.default_rng(i).choice(x.shape[0], 40000, replace=False)]
        shapes.append((w, x))
    return shapes


def test_batch_matches_single_shape_and_oracle(G, orc):
    tau = 1
    shapes = _shapes(10, 0.12, tau)
    ctx = G.Context(tau=tau)
    outs = ctx.batch_build([{"p": torch.from_numpy(w.p).cuda(), "s": torch.from_numpy(w.s).cuda(),
                             "x": torch.from_numpy(x).cuda()} for w, x in shapes])
    ctx.batch_query()
    torch.cuda.synchronize()
    for k, (w, x) in enumerate(shapes):
        single = G.Context(tau=tau)
        single.build(torch.from_numpy(w.p).cuda(), torch.from_numpy(w.s).cuda())
        ref = single.query(torch.from_numpy(x).cuda())
        for key in ("flags", "argmin"):
            assert torch.equal(outs[k][key], ref[key]), (k, key)
        assert torch.equal(outs[k]["s64"].view(torch.int64), ref["s64"].view(torch.int64)), k
        assert torch.equal(ctx.batch_survivors(k), single.survivors()), k
        single.close()
        if w.n <= 3000:
            U = orc.icosphere(tau)
            keep = orc.keep_all(w.p, w.s, U)
            surv = orc.collect(w.p, w.s, U, keep)
            sel = np.arange(0, x.shape[0], max(1, x.shape[0] // 500))
            val, arg, fl, _ = orc.query(w.p, w.s, surv, x[sel])
            assert np.array_equal(outs[k]["argmin"].cpu().numpy()[sel], arg)
            assert np.array_equal(outs[k]["flags"].cpu().numpy()[sel].astype(np.int32) & 0xFFFF, fl)
            assert np.array_equal(ctx.batch_survivors(k).cpu().numpy(), surv[0])
    ctx.close()


def test_batch_query_cuda_graph_replay(G):
    tau = 2
    shapes = _shapes(6, 0.1, tau)
    ctx = G.Context(tau=tau)
    outs = ctx.batch_build([{"p": torch.from_numpy(w.p).cuda(), "s": torch.from_numpy(w.s).cuda(),
                             "x": torch.from_numpy(x).cuda()} for w, x in shapes])
    ctx.batch_query()
    torch.cuda.synchronize()
    first = [{k: o[k].clone() for k in ("s64", "argmin", "flags")} for o in outs]
    for o in outs:
        o["s64"].fill_(7.0)
        o["argmin"].fill_(-7)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            ctx.batch_query()
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    for o, f in zip(outs, first):
        assert torch.equal(o["argmin"], f["argmin"])
        assert torch.equal(o["flags"], f["flags"])
        assert torch.equal(o["s64"].view(torch.int64), f["s64"].view(torch.int64))
    ctx.close()


def test_batch_build_and_query_cuda_graph_replay(G):
    """The whole batched path -- rebuild from the samples and query -- captured
    in one CUDA graph and replayed with new sample values and query points
    written into the same buffers: every replay equals a fresh single-shape
    build and query of that data, bitwise."""
    tau = 2
    shapes = _shapes(6, 0.1, tau)
    tensors = [{"p": torch.from_numpy(w.p).cuda(), "s": torch.from_numpy(w.s).cuda(),
                "x": torch.from_numpy(x).cuda()} for w, x in shapes]
    ctx = G.Context(tau=tau)
    outs = ctx.batch_build(tensors)
    ctx.batch_query()
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            ctx.batch_rebuild()
            ctx.batch_query()
    torch.cuda.synchronize()
    rng = np.random.default_rng(17)
    single = G.Context(tau=tau)
    for variant in range(3):
        # new data in place: values scaled (survivor counts change), points moved
        for t, (w, x) in zip(tensors, shapes):
            f = 1.0 + 0.02 * variant
            t["s"].copy_(torch.from_numpy(w.s * f))
            t["x"].copy_(torch.from_numpy(np.clip(x + rng.normal(0, 0.01, x.shape), -1, 1)))
        for o in outs:
            o["s64"].fill_(7.0)
            o["argmin"].fill_(-7)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert ctx.batch_status() == 0
        for o, t in zip(outs, tensors):
            single.build(t["p"], t["s"])
            ref = single.query(t["x"])
            assert torch.equal(o["argmin"], ref["argmin"])
            assert torch.equal(o["flags"], ref["flags"])
            assert torch.equal(o["s64"].view(torch.int64), ref["s64"].view(torch.int64))
        for k, t in enumerate(tensors):
            single.build(t["p"], t["s"])
            assert torch.equal(ctx.batch_survivors(k), single.survivors())
    single.close()
    ctx.close()


def test_batch_rebuild_reports_capacity_overflow(G):
    """A rebuild whose survivors exceed the first build's capacity sets the
    status bits instead of writing past the lists; a new gfs_batch_build then
    sizes for the counts and matches the single-shape path."""
    rng = np.random.default_rng(9)
    p = rng.uniform(-0.9, 0.9, size=(6000, 3))
    s_big = np.full(6000, -0.5)                  # overlapping balls: few survivors
    s_small = np.full(6000, -1e-3)               # tiny disjoint balls: nearly all survive
    x = rng.uniform(-1, 1, size=(2000, 3))
    t = {"p": torch.from_numpy(p).cuda(), "s": torch.from_numpy(s_big).cuda(), "x": torch.from_numpy(x).cuda()}
    ctx = G.Context(tau=0)
    ctx.batch_build([t])
    assert ctx.batch_status() == 0
    t["s"].copy_(torch.from_numpy(s_small))
    ctx.batch_rebuild()
    assert ctx.batch_status() & 2                 # negative class overflowed
    outs = ctx.batch_build([t])
    ctx.batch_query()
    assert ctx.batch_status() == 0
    single = G.Context(tau=0)
    single.build(t["p"], t["s"])
    ref = single.query(t["x"])
    assert torch.equal(outs[0]["argmin"], ref["argmin"])
    assert torch.equal(outs[0]["flags"], ref["flags"])
    single.close()
    ctx.close()


def _lazy_worker(args):
    from oracle import oracle as O
    p, s, tau, x = args
    return O.query_lazy(p, s, O.icosphere(tau), x)


def test_batch_all_256_shapes_tau3_sampled(G, orc):
    """All 256 shapes of the batch workload (tau 3, half-size grids and
    sample counts: 10.2M samples, 80M queries) in one batched build and
    query: 8 shapes spread over the batch equal the single-shape path
    bitwise, and a few of their outputs and candidates equal the oracle's."""
    import multiprocessing as mp
    tau = 3
    ws = [W.batch_shape(i, tau=tau, scale=0.5) for i in range(256)]
    xs = [torch.from_numpy(w.make_queries()).cuda() for w in ws]
    ctx = G.Context(tau=tau)
    outs = ctx.batch_build([{"p": torch.from_numpy(w.p).cuda(), "s": torch.from_numpy(w.s).cuda(), "x": x}
                            for w, x in zip(ws, xs)])
    ctx.batch_query()
    torch.cuda.synchronize()
    picks = [0, 1, 37, 100, 129, 200, 254, 255]
    rng = np.random.default_rng(5)
    jobs, checks = [], []
    for k in picks:
        w = ws[k]
        single = G.Context(tau=tau)
        single.build(torch.from_numpy(w.p).cuda(), torch.from_numpy(w.s).cuda())
        ref = single.query(xs[k])
        for key in ("flags", "argmin"):
            assert torch.equal(outs[k][key], ref[key]), (k, key)
        assert torch.equal(outs[k]["s64"].view(torch.int64), ref["s64"].view(torch.int64)), k
        surv = ctx.batch_survivors(k)
        assert torch.equal(surv, single.survivors()), k
        single.close()
        # candidate keep decisions and two queries per shape against the oracle
        U = orc.icosphere(tau)
        K = U.shape[0]
        survset = set(int(g) for g in surv.cpu().numpy())
        for i, kk in zip(rng.integers(0, w.n, 40), rng.integers(0, K, 40)):
            assert orc.keep_one(w.p, w.s, U, int(i), int(kk)) == ((int(i) * (K + 1) + int(kk)) in survset)
        sel = rng.choice(xs[k].shape[0], 2, replace=False)
        jobs.append((w.p, w.s, tau, xs[k].cpu().numpy()[sel].astype(np.float64)))
        checks.append((k, sel))
    with mp.get_context("spawn").Pool(min(16, mp.cpu_count())) as pool:
        res = pool.map(_lazy_worker, jobs, chunksize=1)
    for (k, sel), (val, arg, fl, _) in zip(checks, res):
        assert np.array_equal(outs[k]["argmin"].cpu().numpy()[sel], arg), k
        assert np.array_equal(outs[k]["flags"].cpu().numpy()[sel].astype(np.int32) & 0xFFFF, fl), k
        assert np.array_equal(outs[k]["s64"].cpu().numpy()[sel], val, equal_nan=True), k
    ctx.close()
