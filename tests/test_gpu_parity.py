"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Decisions are compared bit for bit: the surviving candidate set, the result
code and violation bits, and the argmin (candidate id or sphere index).  The
FP64 value is compared bitwise too (the library re-evaluates the winner with
the same FP64 expression).  The FP32 value must lie within
1e-5 * max(|s|, 0.1 h) of the oracle's value (h: sample spacing), the stated
tolerance; it is in fact the correctly rounded oracle value.
"""
import multiprocessing as mp

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


def run_gpu(G, p, s, tau, x, precision=0, box_cull=True, clamp_opp=True, x32=False):
    ctx = G.Context(tau=tau, box_cull=box_cull, clamp_opp=clamp_opp, precision=precision)
    ctx.build(torch.from_numpy(np.ascontiguousarray(p)).cuda(), torch.from_numpy(np.ascontiguousarray(s)).cuda())
    xt = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32 if x32 else np.float64)).cuda()
    out = ctx.query(xt)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items() if v is not None}
    res["flags"] = res["flags"].astype(np.int32) & 0xFFFF
    res["surv"] = ctx.survivors().cpu().numpy()
    res["stats"] = ctx.stats()
    ctx.close()
    return res


def oracle_all(orc, p, s, tau, x, box_cull=True, clamp_opp=True):
    U = orc.icosphere(tau)
    keep = orc.keep_all(p, s, U, box_cull=box_cull)
    surv = orc.collect(p, s, U, keep)
    val, arg, fl, gap = orc.query(p, s, surv, x, clamp_opp=clamp_opp)
    return surv[0], val, arg, fl


def assert_parity(res, surv_g, val, arg, fl, h):
    assert np.array_equal(res["surv"], surv_g), "surviving candidate sets differ"
    assert np.array_equal(res["flags"], fl), f"flags differ at {np.nonzero(res['flags'] != fl)[0][:10]}"
    assert np.array_equal(res["argmin"], arg), f"argmin differs at {np.nonzero(res['argmin'] != arg)[0][:10]}"
    assert np.array_equal(res["s64"], val, equal_nan=True)
    ok = ~np.isnan(val)
    tol = 1e-5 * np.maximum(np.abs(val[ok]), 0.1 * h)
    assert np.all(np.abs(res["s"][ok].astype(np.float64) - val[ok]) <= tol)
    assert np.array_equal(res["s"], val.astype(np.float32), equal_nan=True)


@pytest.mark.parametrize("precision", [0, 1])
def test_sphere_grid_full_parity(G, orc, precision):
    """16^3 sphere grid, tau = 2, all 31^3 queries (several tiles and a ragged
    tail: 663,552 candidates, 29,791 queries)."""
    w = W.sphere_grid()
    x = w.make_queries()
    surv, val, arg, fl = oracle_all(orc, w.p, w.s, w.tau, x)
    res = run_gpu(G, w.p, w.s, w.tau, x, precision=precision)
    assert surv.shape[0] == 5449
    assert_parity(res, surv, val, arg, fl, w.h)


CASES = [(n, seed) for n, seed in [(1, 0), (2, 1), (7, 2), (37, 3), (100, 4), (257, 5), (600, 6)]]


@pytest.mark.parametrize("n,seed", CASES)
@pytest.mark.parametrize("tau", [0, 1, 3])
def test_tiny_random_parity(G, orc, n, seed, tau):
    p, s = W.tiny_random(n, seed, valid=(seed % 3 != 0), spread=0.9)
    rng = np.random.default_rng(1000 + seed)
    x = np.concatenate([rng.uniform(-1, 1, size=(300, 3)), p[: min(n, 20)],
                        rng.uniform(-1.5, 1.5, size=(20, 3))])
    for box_cull, clamp in [(True, True), (False, True), (True, False)]:
        surv, val, arg, fl = oracle_all(orc, p, s, tau, x, box_cull=box_cull, clamp_opp=clamp)
        for precision in (0, 1):
            res = run_gpu(G, p, s, tau, x, precision=precision, box_cull=box_cull, clamp_opp=clamp)
            assert_parity(res, surv, val, arg, fl, 0.05)


def test_degenerate_inputs(G, orc):
    """Duplicated samples, zero samples, touching spheres, nested spheres,
    both-sign containment (invalid input) and queries at sample points."""
    p = np.array([[0.0, 0, 0], [0.0, 0, 0], [0.5, 0, 0], [0.2, 0.1, 0], [0.2, 0.1, 0.0],
                  [-0.4, 0.3, 0.2], [-0.4, 0.3, 0.2], [0.7, 0.7, 0.7]])
    s = np.array([0.3, 0.3, 0.2, 0.0, 0.05, -0.25, -0.1, 0.5])
    rng = np.random.default_rng(9)
    # the last point lies inside both ball 0 (+) and ball 5 (-), which overlap
    x = np.concatenate([p, rng.uniform(-1, 1, size=(500, 3)), [[0.3, 0.0, 0.0], [0.25, 0.0, 0.0],
                                                               [-0.219, 0.164, 0.109]]])
    for tau in (1, 2):
        surv, val, arg, fl = oracle_all(orc, p, s, tau, x)
        assert np.any((fl & 15) == 4)                     # invalid (both signs) occurs
        for precision in (0, 1):
            res = run_gpu(G, p, s, tau, x, precision=precision)
            assert_parity(res, surv, val, arg, fl, 0.05)


def test_union_grid_small_parity(G, orc):
    """Union of spheres and boxes on a 20^3 grid, tau = 3, 4x upsampled
    queries (exact ties at box faces exercise the FP64 re-decision)."""
    w = W.union_grid(N=20, up=4)
    x = w.make_queries()
    sel = np.random.default_rng(2).choice(x.shape[0], 20000, replace=False)
    xs = np.concatenate([x[sel], w.p[::7]])
    surv, val, arg, fl = oracle_all(orc, w.p, w.s, w.tau, xs)
    for precision in (0, 1):
        res = run_gpu(G, w.p, w.s, w.tau, xs, precision=precision)
        assert_parity(res, surv, val, arg, fl, w.h)


def test_fp32_queries_torus_parity(G, orc):
    """FP32 query coordinates (torus grid, uniform random points)."""
    w = W.torus_grid(N=24, m=6000)
    x = w.make_queries()
    surv, val, arg, fl = oracle_all(orc, w.p, w.s, w.tau, x.astype(np.float64))
    res = run_gpu(G, w.p, w.s, w.tau, x, x32=True)
    assert_parity(res, surv, val, arg, fl, w.h)


# ---------------------------------------------------------------------------
# full-size union grid (64^3, tau = 3, 253^3 queries): sampled outputs
# ---------------------------------------------------------------------------

def _lazy_worker(args):
    from oracle import oracle as O
    p, s, tau, x = args
    return O.query_lazy(p, s, O.icosphere(tau), x)


def test_union_grid_full_size_sampled(G, orc):
    w = W.union_grid()
    x = w.make_queries()
    ctx = G.Context(tau=w.tau)
    ctx.build(torch.from_numpy(w.p).cuda(), torch.from_numpy(w.s).cuda())
    xt = torch.from_numpy(x).cuda()
    out = ctx.query(xt)
    surv = ctx.survivors().cpu().numpy()
    st = ctx.stats()
    s32, s64 = out["s"].cpu().numpy(), out["s64"].cpu().numpy()
    arg, fl = out["argmin"].cpu().numpy(), out["flags"].cpu().numpy().astype(np.int32) & 0xFFFF
    ctx.close()
    rng = np.random.default_rng(77)
    # keep decisions of sampled candidates (brute force per candidate)
    U = orc.icosphere(w.tau)
    K = U.shape[0]
    survset = set(int(g) for g in surv)
    ii = rng.integers(0, w.n, 1500)
    kk = rng.integers(0, K, 1500)
    for i, k in zip(ii, kk):
        assert orc.keep_one(w.p, w.s, U, int(i), int(k)) == ((int(i) * (K + 1) + int(k)) in survset)
    # every reported survivor that we sample is kept by the oracle
    for g in rng.choice(surv, 300, replace=False):
        assert orc.keep_one(w.p, w.s, U, int(g) // (K + 1), int(g) % (K + 1))
    # sampled queries against the lazy oracle, in parallel host processes
    sel = rng.choice(x.shape[0], 64, replace=False)
    chunks = np.array_split(sel, 16)
    ctxm = mp.get_context("spawn")
    with ctxm.Pool(min(16, mp.cpu_count())) as pool:
        outs = pool.map(_lazy_worker, [(w.p, w.s, w.tau, x[c]) for c in chunks])
    val = np.concatenate([o[0] for o in outs])
    oarg = np.concatenate([o[1] for o in outs])
    ofl = np.concatenate([o[2] for o in outs])
    assert np.array_equal(fl[sel], ofl)
    assert np.array_equal(arg[sel], oarg)
    assert np.array_equal(s64[sel], val, equal_nan=True)
    assert np.array_equal(s32[sel], val.astype(np.float32), equal_nan=True)
    print("stats", st)


def test_union_grid_full_size_fp32_equals_fp64_path(G, orc):
    """At full size, the FP32-filtered path and the FP64 path agree on every
    output (all 16.2M queries); any disagreement is settled by the oracle."""
    w = W.union_grid()
    xh = w.make_queries()
    xt = torch.from_numpy(xh).cuda()
    res = []
    for precision in (0, 1):
        ctx = G.Context(tau=w.tau, precision=precision)
        ctx.build(torch.from_numpy(w.p).cuda(), torch.from_numpy(w.s).cuda())
        out = ctx.query(xt)
        res.append({k: v.cpu() for k, v in out.items()})
        res[-1]["surv"] = ctx.survivors().cpu()
        ctx.close()
    a, b = res
    assert torch.equal(a["surv"], b["surv"])
    bad = ((a["flags"] != b["flags"]) | (a["argmin"] != b["argmin"]) |
           (a["s64"].view(torch.int64) != b["s64"].view(torch.int64))).nonzero().flatten().numpy()
    if bad.size:
        sel = bad[:12]
        v, arg, fl, _ = orc.query_lazy(w.p, w.s, orc.icosphere(w.tau), xh[sel])
        fp32_ok = np.array_equal(a["argmin"].numpy()[sel], arg)
        fp64_ok = np.array_equal(b["argmin"].numpy()[sel], arg)
        pytest.fail(f"{bad.size} queries differ; FP32 path matches oracle: {fp32_ok}, FP64 path: {fp64_ok}")


# ---------------------------------------------------------------------------
# full-size 128^3 workloads: sampled outputs against the lazy oracle
# ---------------------------------------------------------------------------

def _near_surface(w, x, n, seed, band):
    """n indices of points of x whose nearest grid sample has |s| < band * h.
    The lazy oracle's cost grows with the distance to the nearest surviving
    candidate (its search shell), so the full-size 128^3 checks sample near
    the surface; far points are checked at full size on the 64^3 workload and
    exhaustively on the small ones."""
    N = round(w.n ** (1 / 3))
    idx = np.clip(np.rint((x.astype(np.float64) + 1.0) / w.h).astype(np.int64), 0, N - 1)
    sn = w.s[(idx[:, 0] * N + idx[:, 1]) * N + idx[:, 2]]
    near = np.nonzero(np.abs(sn) < band * w.h)[0]
    return np.random.default_rng(seed).choice(near, n, replace=False)


def _sampled_check(G, orc, w, x, sel, n_keep=400, seed=91):
    ctx = G.Context(tau=w.tau)
    ctx.build(torch.from_numpy(w.p).cuda(), torch.from_numpy(w.s).cuda())
    out = ctx.query(torch.from_numpy(np.ascontiguousarray(x)).cuda())
    surv = ctx.survivors().cpu().numpy()
    s64 = out["s64"].cpu().numpy()
    arg = out["argmin"].cpu().numpy()
    fl = out["flags"].cpu().numpy().astype(np.int32) & 0xFFFF
    ctx.close()
    rng = np.random.default_rng(seed)
    U = orc.icosphere(w.tau)
    K = U.shape[0]
    survset = set(int(g) for g in surv)
    for i, k in zip(rng.integers(0, w.n, n_keep), rng.integers(0, K, n_keep)):
        assert orc.keep_one(w.p, w.s, U, int(i), int(k)) == ((int(i) * (K + 1) + int(k)) in survset)
    for g in rng.choice(surv, min(100, surv.size), replace=False):
        assert orc.keep_one(w.p, w.s, U, int(g) // (K + 1), int(g) % (K + 1))
    xs = x[sel].astype(np.float64)
    ctxm = mp.get_context("spawn")
    with ctxm.Pool(min(16, mp.cpu_count())) as pool:
        outs = pool.map(_lazy_worker, [(w.p, w.s, w.tau, xs[i:i + 1]) for i in range(xs.shape[0])], chunksize=1)
    val = np.concatenate([o[0] for o in outs])
    oarg = np.concatenate([o[1] for o in outs])
    ofl = np.concatenate([o[2] for o in outs])
    assert np.array_equal(fl[sel], ofl)
    assert np.array_equal(arg[sel], oarg)
    assert np.array_equal(s64[sel], val, equal_nan=True)
    return fl


def test_csg_pseudo_grid_full_size_sampled(G, orc):
    """128^3 CSG pseudo-SDF with 5% noisy samples (balls of both signs may
    overlap: INVALID points occur); 32 points within 2h of the surface."""
    w = W.csg_pseudo_grid()
    rng = np.random.default_rng(12)
    x = rng.uniform(-1, 1, size=(1 << 20, 3))
    fl = _sampled_check(G, orc, w, x, _near_surface(w, x, 32, 13, 2.0))
    assert np.any((fl & 15) <= 1)


def test_torus_grid_full_size_sampled(G, orc):
    """128^3 torus grid, 2^22 uniform FP32 points (the differentiable-query
    workload); 32 points within 8h of the surface."""
    w = W.torus_grid()
    x = w.make_queries()
    _sampled_check(G, orc, w, x, _near_surface(w, x, 32, 14, 8.0))
