"""Same-sign tangent augmentation (gfs_query_tangent) against the oracle's
augmented query, through the C ABI.

The pass refines a plain query's outputs in place: for points of code
SURVIVOR / OPPOSITE / LOWER the near and far tangent points of the spheres of
the point's own sign (Def. 1 T) join the candidates.  Decisions (code and
violation bits, argmin 2j + side for tangent winners) and the FP64 value are
compared bit for bit; the FP32 value is the rounded FP64 value, within
1e-5 * max(|s|, 0.1 h) of the oracle's.  The backward pass is compared with
the oracle's analytic gradient, whose TANGENT branch is pinned by finite
differences in the oracle tests.
"""
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


def run_gpu(G, p, s, tau, x, precision=0, box_cull=True, clamp_opp=True, x32=False):
    ctx = G.Context(tau=tau, box_cull=box_cull, clamp_opp=clamp_opp, precision=precision, tangent=True)
    ctx.build(torch.from_numpy(np.ascontiguousarray(p)).cuda(), torch.from_numpy(np.ascontiguousarray(s)).cuda())
    xt = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32 if x32 else np.float64)).cuda()
    out = ctx.query(xt)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items() if v is not None}
    res["flags"] = res["flags"].astype(np.int32) & 0xFFFF
    ctx.close()
    return res


def oracle_aug(orc, p, s, tau, x, box_cull=True, clamp_opp=True):
    U = orc.icosphere(tau)
    surv = orc.collect(p, s, U, orc.keep_all(p, s, U, box_cull=box_cull))
    return orc.query_aug(p, s, surv, x, clamp_opp=clamp_opp, box_cull=box_cull)


def assert_parity(res, val, arg, fl, h):
    assert np.array_equal(res["flags"], fl), f"flags differ at {np.nonzero(res['flags'] != fl)[0][:10]}"
    assert np.array_equal(res["argmin"], arg), f"argmin differs at {np.nonzero(res['argmin'] != arg)[0][:10]}"
    assert np.array_equal(res["s64"], val, equal_nan=True)
    ok = ~np.isnan(val)
    tol = 1e-5 * np.maximum(np.abs(val[ok]), 0.1 * h)
    assert np.all(np.abs(res["s"][ok].astype(np.float64) - val[ok]) <= tol)
    assert np.array_equal(res["s"], val.astype(np.float32), equal_nan=True)


@pytest.fixture(scope="module")
def sphere_case(orc):
    """16^3 sphere grid, tau = 2: 1200 of the 31^3 points plus sample points,
    with the oracle's augmented results."""
    w = W.sphere_grid()
    x = w.make_queries()
    sel = np.random.default_rng(3).choice(x.shape[0], 1200, replace=False)
    xs = np.concatenate([x[sel], w.p[::97]])
    return w, xs, oracle_aug(orc, w.p, w.s, w.tau, xs)


@pytest.mark.parametrize("precision", [0, 1])
def test_tangent_sphere_grid_parity(G, sphere_case, precision):
    w, xs, (val, arg, fl) = sphere_case
    assert np.sum((fl & 15) == G.CODE_TANGENT) > 50
    res = run_gpu(G, w.p, w.s, w.tau, xs, precision=precision)
    assert_parity(res, val, arg, fl, w.h)


CASES = [(1, 0), (2, 1), (7, 2), (37, 3), (100, 4), (257, 5), (600, 6)]


@pytest.mark.parametrize("n,seed", CASES)
@pytest.mark.parametrize("tau", [0, 3])
def test_tangent_tiny_random_parity(G, orc, n, seed, tau):
    """Seeded tiny inputs (valid and invalid), points inside and outside the
    box, every option combination of the box cull and the opposite clamp."""
    p, s = W.tiny_random(n, seed, valid=(seed % 3 != 0), spread=0.9)
    rng = np.random.default_rng(1000 + seed)
    x = np.concatenate([rng.uniform(-1, 1, size=(300, 3)), p[: min(n, 20)],
                        rng.uniform(-1.5, 1.5, size=(20, 3))])
    for box_cull, clamp in [(True, True), (False, True), (True, False)]:
        val, arg, fl = oracle_aug(orc, p, s, tau, x, box_cull=box_cull, clamp_opp=clamp)
        for precision in (0, 1):
            res = run_gpu(G, p, s, tau, x, precision=precision, box_cull=box_cull, clamp_opp=clamp)
            assert_parity(res, val, arg, fl, 0.05)


def test_tangent_degenerate_inputs(G, orc):
    """Duplicated, zero, touching and nested samples, and both-sign points."""
    p = np.array([[0.0, 0, 0], [0.0, 0, 0], [0.5, 0, 0], [0.2, 0.1, 0], [0.2, 0.1, 0.0],
                  [-0.4, 0.3, 0.2], [-0.4, 0.3, 0.2], [0.7, 0.7, 0.7]])
    s = np.array([0.3, 0.3, 0.2, 0.0, 0.05, -0.25, -0.1, 0.5])
    rng = np.random.default_rng(9)
    x = np.concatenate([p, rng.uniform(-1, 1, size=(500, 3)), [[0.3, 0.0, 0.0], [0.25, 0.0, 0.0],
                                                               [-0.219, 0.164, 0.109]]])
    for tau in (1, 2):
        val, arg, fl = oracle_aug(orc, p, s, tau, x)
        assert np.any((fl & 15) == G.CODE_TANGENT)
        res = run_gpu(G, p, s, tau, x)
        assert_parity(res, val, arg, fl, 0.05)


def test_tangent_union_grid_small_parity(G, orc):
    """Union of spheres and boxes on a 12^3 grid, tau = 3, sampled 4x
    upsampled points and sample points."""
    w = W.union_grid(N=12, up=4)
    x = w.make_queries()
    sel = np.random.default_rng(2).choice(x.shape[0], 1500, replace=False)
    xs = np.concatenate([x[sel], w.p[::11]])
    val, arg, fl = oracle_aug(orc, w.p, w.s, w.tau, xs)
    res = run_gpu(G, w.p, w.s, w.tau, xs)
    assert_parity(res, val, arg, fl, w.h)


def test_tangent_fp32_points_torus_parity(G, orc):
    """FP32 point coordinates (14^3 torus grid, uniform points)."""
    w = W.torus_grid(N=14, m=800)
    x = w.make_queries()
    val, arg, fl = oracle_aug(orc, w.p, w.s, w.tau, x.astype(np.float64))
    res = run_gpu(G, w.p, w.s, w.tau, x, x32=True)
    assert_parity(res, val, arg, fl, w.h)


def test_tangent_backward_matches_oracle_gradient(G, orc):
    """ConsistentSDF on a tangent-augmented context: d/dx, d/dp_j and d/ds_j
    of every result, TANGENT ones included, against the oracle's gradient at
    the oracle's augmented argmin."""
    w = W.sphere_grid(N=10, up=2, tau=2)
    x = w.make_queries()
    U = orc.icosphere(w.tau)
    surv = orc.collect(w.p, w.s, U, orc.keep_all(w.p, w.s, U))
    val, arg, fl = orc.query_aug(w.p, w.s, surv, x)
    assert np.sum((fl & 15) == G.CODE_TANGENT) > 100
    gup = np.random.default_rng(5).normal(size=x.shape[0])
    gx_o, gp_o, gs_o = orc.grad(w.p, w.s, U, x, val, arg, fl, gup)
    ctx = G.Context(tau=w.tau, tangent=True)
    pt = torch.from_numpy(w.p).cuda().requires_grad_(True)
    st = torch.from_numpy(w.s).cuda().requires_grad_(True)
    ctx.build(pt.detach(), st.detach())
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    sv = G.ConsistentSDF.apply(xt, pt, st, ctx)
    sv.backward(torch.from_numpy(gup).float().cuda())
    assert np.array_equal(sv.detach().cpu().numpy(), val.astype(np.float32))
    assert np.max(np.abs(xt.grad.cpu().numpy() - gx_o)) < 1e-5 * max(1.0, np.abs(gup).max())
    scale = np.abs(gup).sum()
    assert np.max(np.abs(pt.grad.cpu().numpy() - gp_o)) < 1e-6 * scale + 1e-5
    assert np.max(np.abs(st.grad.cpu().numpy() - gs_o)) < 1e-6 * scale + 1e-5
    ctx.close()


def test_tangent_full_size_properties(G):
    """64^3 union grid (262,144 samples, tau = 3) with 2^16 of its 253^3
    points: the pass only lowers values, keeps the sign, leaves every point
    it does not refine bit-identical, and its TANGENT values are distances to
    points on the winning sphere."""
    w = W.union_grid()
    x = w.make_queries()
    sel = np.random.default_rng(8).choice(x.shape[0], 1 << 16, replace=False)
    xt = torch.from_numpy(x[sel]).cuda()
    ctx = G.Context(tau=w.tau)
    ctx.build(torch.from_numpy(w.p).cuda(), torch.from_numpy(w.s).cuda())
    plain = ctx.query(xt)
    aug = {k: v.clone() for k, v in plain.items()}
    ctx.tangent_into(xt, aug["s"], aug["s64"], aug["argmin"], aug["flags"])
    torch.cuda.synchronize()
    ctx.close()
    f0 = plain["flags"].cpu().numpy().astype(np.int32) & 0xFFFF
    f1 = aug["flags"].cpu().numpy().astype(np.int32) & 0xFFFF
    v0, v1 = plain["s64"].cpu().numpy(), aug["s64"].cpu().numpy()
    a0, a1 = plain["argmin"].cpu().numpy(), aug["argmin"].cpu().numpy()
    won = (f1 & 15) == G.CODE_TANGENT
    assert won.any() and not ((f0 & 15) == G.CODE_TANGENT).any()
    same = ~won
    assert np.array_equal(f0[same], f1[same]) and np.array_equal(a0[same], a1[same])
    assert np.array_equal(v0[same], v1[same], equal_nan=True)
    assert np.all(np.isin(f0[won] & 15, [G.CODE_SURVIVOR, G.CODE_OPPOSITE, G.CODE_LOWER]))
    assert np.all(np.abs(v1[won]) <= np.abs(v0[won])) and np.array_equal(np.signbit(v1[won]), np.signbit(v0[won]))
    # |value| = | |x - p_j| - e r_j | for the winner (j, side), to rounding
    j, side = a1[won] // 2, a1[won] % 2
    d = np.linalg.norm(x[sel][won] - w.p[j], axis=1)
    r = np.abs(w.s[j])
    expect = np.where(side == 0, np.abs(d - r), d + r)
    assert np.allclose(np.abs(v1[won]), expect, rtol=1e-12, atol=1e-14)
    assert np.array_equal(w.s[j] < 0, np.signbit(v1[won]))
    print(f"tangent wins: {won.sum()} of {won.size}")


def _aug_worker(args):
    from oracle import oracle as O
    p, s, tau, x = args
    return O.query_aug_lazy(p, s, O.icosphere(tau), x)


def test_tangent_full_size_sampled(G, orc):
    """64^3 union grid (262,144 samples, tau = 3): 48 points within 2h of the
    surface, augmented on the GPU, against the lazy augmented oracle (spawned
    host processes) bit for bit."""
    import multiprocessing as mp
    from tests.test_gpu_parity import _near_surface
    w = W.union_grid()
    x = w.make_queries()
    sel = _near_surface(w, x, 48, 17, 2.0)
    xs = np.ascontiguousarray(x[sel])
    res = run_gpu(G, w.p, w.s, w.tau, xs)
    with mp.get_context("spawn").Pool(min(16, mp.cpu_count())) as pool:
        outs = pool.map(_aug_worker, [(w.p, w.s, w.tau, xs[i:i + 1]) for i in range(xs.shape[0])], chunksize=1)
    val = np.concatenate([o[0] for o in outs])
    arg = np.concatenate([o[1] for o in outs])
    fl = np.concatenate([o[2] for o in outs])
    assert np.sum((fl & 15) == G.CODE_TANGENT) > 5
    assert_parity(res, val, arg, fl, w.h)


def test_tangent_batched_equals_single_shape_and_oracle(G, orc):
    """gfs_batch_query_tangent on 8 small batch shapes (grids and scattered
    samples, tau 1): every shape's refined outputs equal the single-shape
    pass bit for bit (the batched hierarchies differ, the decisions may not),
    and the small shapes equal the oracle's augmented query."""
    tau = 1
    shapes = []
    for i in range(8):
        w = W.batch_shape(i, tau=tau, scale=0.12)
        x = w.make_queries()
        if x.shape[0] > 20000:
            x = x[np.random.default_rng(i).choice(x.shape[0], 20000, replace=False)]
        shapes.append((w, x))
    ctx = G.Context(tau=tau, tangent=True)
    outs = ctx.batch_build([{"p": torch.from_numpy(w.p).cuda(), "s": torch.from_numpy(w.s).cuda(),
                             "x": torch.from_numpy(x).cuda()} for w, x in shapes])
    ctx.batch_query()
    torch.cuda.synchronize()
    won = 0
    for k, (w, x) in enumerate(shapes):
        ref = run_gpu(G, w.p, w.s, tau, x)
        got = {key: outs[k][key].cpu().numpy() for key in ("s", "s64", "argmin", "flags")}
        got["flags"] = got["flags"].astype(np.int32) & 0xFFFF
        for key in ("flags", "argmin"):
            assert np.array_equal(got[key], ref[key]), (k, key)
        assert np.array_equal(got["s64"].view(np.int64), ref["s64"].view(np.int64)), k
        won += int(np.sum((got["flags"] & 15) == G.CODE_TANGENT))
        if w.n <= 2000:
            sel = np.arange(0, x.shape[0], max(1, x.shape[0] // 150))
            val, arg, fl = oracle_aug(orc, w.p, w.s, tau, x[sel])
            assert np.array_equal(got["argmin"][sel], arg) and np.array_equal(got["flags"][sel], fl)
            assert np.array_equal(got["s64"][sel], val, equal_nan=True)
    assert won > 0
    ctx.close()
