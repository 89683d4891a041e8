"""Scored value (Sec. 3.3) on the GPU against the oracle's brute force, bit
for bit: the FP64 value, the argmin (survivor id or tangent id 2j + side)
and the result word (including SCORE_FALLBACK and LB_VIOL)."""
import time

import numpy as np
import pytest
import torch

from paper_2605_01919_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.widening]


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2605_01919_gb300 import gfs
    gfs.load()
    return gfs


def _compare(G, orc, p, s, tau, x, box_cull=True, x32=False):
    U = orc.icosphere(tau)
    surv = orc.collect(p, s, U, orc.keep_all(p, s, U, box_cull=box_cull))
    xo = x.astype(np.float32).astype(np.float64) if x32 else x
    val, arg, fl = orc.query_scored(p, s, surv, xo, box_cull=box_cull)
    ctx = G.Context(tau=tau, box_cull=box_cull)
    ctx.build(torch.from_numpy(np.ascontiguousarray(p)).cuda(), torch.from_numpy(np.ascontiguousarray(s)).cuda())
    xt = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32 if x32 else np.float64)).cuda()
    out = ctx.query_scored(xt)
    torch.cuda.synchronize()
    gf = out["flags"].cpu().numpy().astype(np.int32) & 0xFFFF
    ga = out["argmin"].cpu().numpy()
    bad = np.nonzero((gf != fl) | (ga != arg))[0]
    assert bad.size == 0, f"differ at {bad[:8]}: gpu {gf[bad[:4]]} {ga[bad[:4]]} oracle {fl[bad[:4]]} {arg[bad[:4]]}"
    assert np.array_equal(out["s64"].cpu().numpy(), val, equal_nan=True)
    assert np.array_equal(out["s"].cpu().numpy(), val.astype(np.float32), equal_nan=True)
    ctx.close()
    return val, arg, fl


def test_scored_sphere_grid(G, orc):
    w = W.sphere_grid(N=10, up=2, tau=2)
    x = w.make_queries()
    val, arg, fl = _compare(G, orc, w.p, w.s, w.tau, x)
    codes = fl & 15
    assert np.sum(codes == orc.CODE_TANGENT) > 100 and np.sum(codes == orc.CODE_SURVIVOR) > 10
    assert np.sum(codes == orc.CODE_SAMPLE) == w.n


def test_scored_union_grid(G, orc):
    w = W.union_grid(N=12, up=2, tau=1)
    _compare(G, orc, w.p, w.s, w.tau, w.make_queries())


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (9, 2), (60, 3), (250, 4)])
@pytest.mark.parametrize("tau", [0, 2])
def test_scored_tiny_random(G, orc, n, seed, tau):
    p, s = W.tiny_random(n, seed)
    x = np.random.default_rng(100 + seed).uniform(-1.1, 1.1, size=(400, 3))
    for box in (True, False):
        _compare(G, orc, p, s, tau, x, box_cull=box)


def test_scored_hand_worked_and_fallback(G, orc):
    p = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0]])
    s = np.array([0.2, 0.05])
    val, arg, fl = _compare(G, orc, p, s, 2, np.array([[0.3, 0.0, 0.0]]))
    assert abs(val[0] - 0.25) < 1e-15 and arg[0] == 3
    p = np.array([[0.1, 0.05, -0.1]])
    s = np.array([-3.0])
    val, arg, fl = _compare(G, orc, p, s, 1, np.array([[0.2, 0.1, 0.0], [0.0, 0.0, 0.0]]))
    assert np.all(fl & orc.FLAG_SCORE_FALLBACK)


def test_scored_fp32_points_torus(G, orc):
    w = W.torus_grid(N=14, m=3000)
    _compare(G, orc, w.p, w.s, w.tau, w.make_queries().astype(np.float64), x32=True)
