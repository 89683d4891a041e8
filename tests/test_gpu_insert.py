"""Greedy sequential insertion on the GPU against the oracle's sequential
loop: every step's value (FP64, bitwise), argmin and result word
(including LOST_WITNESS), the final survivor set, and queries against the
final state."""
import functools

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


def _compare(G, orc, p, s, tau, y, xq, known=None, clamp_opp=True, stats=None):
    U = orc.icosphere(tau)
    val, arg, fl, st = orc.insert(p, s, U, y, known=known, clamp_opp=clamp_opp)
    ctx = G.Context(tau=tau, clamp_opp=clamp_opp)
    ctx.build(torch.from_numpy(p).cuda(), torch.from_numpy(s).cuda())
    out = ctx.insert(torch.from_numpy(y).cuda(), known=None if known is None else torch.from_numpy(known).cuda())
    if stats is not None:
        stats.update(ctx.stats())
    torch.cuda.synchronize()
    gv = out["s64"].cpu().numpy()
    ga = out["argmin"].cpu().numpy()
    gf = out["flags"].cpu().numpy().astype(np.int32) & 0xFFFF
    bad = np.nonzero((gf != fl) | (ga != arg))[0]
    assert bad.size == 0, f"steps differ: {bad[:10]} gpu {gf[bad[:5]]} {ga[bad[:5]]} oracle {fl[bad[:5]]} {arg[bad[:5]]}"
    assert np.array_equal(gv, val, equal_nan=True)
    surv = ctx.survivors().cpu().numpy()
    assert np.array_equal(surv, st["g"])
    # queries against the final state use the inserted samples and witnesses
    res = ctx.query(torch.from_numpy(xq).cuda())
    ov, oa, of, _ = orc.query(st["p"], st["s"], (st["g"], st["sph"], st["q"]), xq, clamp_opp=clamp_opp)
    assert np.array_equal(res["flags"].cpu().numpy().astype(np.int32) & 0xFFFF, of)
    assert np.array_equal(res["argmin"].cpu().numpy(), oa)
    assert np.array_equal(res["s64"].cpu().numpy(), ov, equal_nan=True)
    ctx.close()
    return fl


def test_insert_refinement_sphere_grid(G, orc):
    """Refinement: new points in random order inside the 10^3 sphere grid."""
    w = W.sphere_grid(N=10, up=2, tau=2)
    rng = np.random.default_rng(21)
    y = rng.uniform(-0.9, 0.9, size=(300, 3))
    xq = rng.uniform(-1, 1, size=(500, 3))
    fl = _compare(G, orc, w.p, w.s, w.tau, y, xq)
    assert np.any((fl & 15) == 0)


def test_insert_with_rebuilds_and_repeats(G, orc):
    """More steps than the rebuild interval (256), repeated points (SAMPLE
    steps) and points outside every ball (OUTSIDE steps)."""
    w = W.union_grid(N=10, up=2, tau=1)
    rng = np.random.default_rng(22)
    y = rng.uniform(-1, 1, size=(600, 3))
    y[100:110] = y[0:10]                          # re-inserting a point: SAMPLE
    xq = rng.uniform(-1, 1, size=(300, 3))
    fl = _compare(G, orc, w.p, w.s, w.tau, y, xq)
    inserted_first = np.isin(fl[:10] & 15, [0, 1, 5])
    assert np.all((fl[100:110][inserted_first] & 15) == 2)   # re-insertions reproduce the value


def test_insert_pseudo_sdf_repair(G, orc):
    """Repair: samples fully covered at tau are removed and re-inserted in
    index order with the greedy loop (noisy pseudo-SDF, small grid)."""
    w = W.csg_pseudo_grid(N=10, tau=1)
    U = orc.icosphere(w.tau)
    keep = orc.keep_all(w.p, w.s, U)
    covered = keep.sum(axis=1) == 0
    p2, s2 = w.p[~covered], w.s[~covered]
    y = w.p[covered][:200]
    xq = np.random.default_rng(3).uniform(-1, 1, size=(300, 3))
    _compare(G, orc, p2, s2, w.tau, y, xq)


def test_insert_known_values_repair(G, orc):
    """Repair with known values (Sec. 6): samples fully covered at tau are
    removed and re-inserted in index order with their own values known (their
    signs fix the classes; NONCONSERVATIVE marks values below them)."""
    w = W.csg_pseudo_grid(N=10, tau=1)
    U = orc.icosphere(w.tau)
    keep = orc.keep_all(w.p, w.s, U)
    covered = keep.sum(axis=1) == 0
    p2, s2 = w.p[~covered], w.s[~covered]
    y, known = w.p[covered][:300], w.s[covered][:300]
    val, arg, fl, st = orc.insert(p2, s2, U, y, known=known)
    ctx = G.Context(tau=w.tau)
    ctx.build(torch.from_numpy(p2).cuda(), torch.from_numpy(s2).cuda())
    out = ctx.insert(torch.from_numpy(y).cuda(), known=torch.from_numpy(known).cuda())
    torch.cuda.synchronize()
    gf = out["flags"].cpu().numpy().astype(np.int32) & 0xFFFF
    ga = out["argmin"].cpu().numpy()
    bad = np.nonzero((gf != fl) | (ga != arg))[0]
    assert bad.size == 0, f"steps differ: {bad[:10]} gpu {gf[bad[:5]]} {ga[bad[:5]]} oracle {fl[bad[:5]]} {arg[bad[:5]]}"
    assert np.array_equal(out["s64"].cpu().numpy(), val, equal_nan=True)
    assert np.array_equal(ctx.survivors().cpu().numpy(), st["g"])
    assert np.any(fl & orc.FLAG_NONCONSERVATIVE) and not np.any(np.isin(fl & 15, [3, 4]))
    ctx.close()


@functools.lru_cache(maxsize=1)
def _csg24_repair(orc):
    """The 24^3 CSG pseudo-SDF at tau 2: the samples with no surviving
    candidate are removed, the rest kept."""
    w = W.csg_pseudo_grid(N=24, tau=2)
    U = orc.icosphere(w.tau)
    covered = orc.keep_all(w.p, w.s, U).sum(axis=1) == 0
    return w, covered


def test_insert_csg24_repair_2000_steps(G, orc):
    """Config-3 style repair on a 24^3 CSG pseudo-SDF grid: 2,000 removed
    samples re-inserted with known values in index order (neighbours, mostly
    within each other's reach), step by step against the sequential oracle."""
    w, covered = _csg24_repair(orc)
    idx = np.nonzero(covered)[0][:2000]
    assert idx.size == 2000
    xq = np.random.default_rng(4).uniform(-1, 1, size=(400, 3))
    _compare(G, orc, w.p[~covered], w.s[~covered], w.tau, w.p[idx], xq, known=w.s[idx])


def test_insert_csg24_repair_scattered_order(G, orc):
    """The same repair in a seeded random order: points far apart commit
    together (fewer rounds than steps, out-of-order commits with provisional
    sphere numbering), with the sequential loop's results step by step."""
    w, covered = _csg24_repair(orc)
    idx = np.random.default_rng(8).permutation(np.nonzero(covered)[0])[:2400]
    xq = np.random.default_rng(6).uniform(-1, 1, size=(400, 3))
    st = {}
    _compare(G, orc, w.p[~covered], w.s[~covered], w.tau, w.p[idx], xq, known=w.s[idx], stats=st)
    assert st["insert_steps"] == idx.size
    assert st["insert_rounds"] < idx.size // 4, st["insert_rounds"]


def test_insert_refinement_parallel_rounds(G, orc):
    """Refinement with inferred signs at scattered points of a 16^3 union
    grid, enough steps for rebuilds between rounds; values, argmins (renumbered
    spheres) and result words against the sequential oracle."""
    w = W.union_grid(N=16, up=2, tau=1)
    rng = np.random.default_rng(41)
    y = rng.uniform(-1, 1, size=(3000, 3))
    y[2000:2020] = y[1500:1520]                    # repeats: SAMPLE of a renumbered sphere
    xq = rng.uniform(-1, 1, size=(400, 3))
    st = {}
    fl = _compare(G, orc, w.p, w.s, w.tau, y, xq, stats=st)
    assert st["insert_rounds"] < 1000, st["insert_rounds"]
    assert np.any((fl[2000:2020] & 15) == 2)


def test_insert_lost_witness_without_clamp(G, orc):
    """Without the opposite clamp a new ball can swallow the last survivors of
    an opposite sphere: LOST_WITNESS on the step that removes the last one
    (no value bound, so one step per round)."""
    w = W.union_grid(N=10, up=2, tau=0)
    y = np.random.default_rng(5).uniform(-1, 1, size=(800, 3))
    xq = np.random.default_rng(7).uniform(-1, 1, size=(300, 3))
    fl = _compare(G, orc, w.p, w.s, w.tau, y, xq, clamp_opp=False)
    assert np.sum((fl & 0x80) != 0) >= 5


def test_insert_exact_removal_repair(G, orc):
    """Sec. 6 repair with the exact removal set: on the 10^3 CSG pseudo-SDF
    the spheres that the other balls cover exactly (the oracle's Prop. 1
    (ii) test: 117 of 1,000) are removed and re-inserted with their values
    known, in index order and in a seeded permutation, step by step against
    the sequential oracle."""
    w = W.csg_pseudo_grid(N=10, tau=1)
    covered = orc.sphere_uncovered(w.p, w.s) == 0
    assert covered.sum() == 117
    idx = np.nonzero(covered)[0]
    xq = np.random.default_rng(12).uniform(-1, 1, size=(300, 3))
    for sel in (idx, np.random.default_rng(13).permutation(idx)):
        _compare(G, orc, w.p[~covered], w.s[~covered], w.tau, w.p[sel], xq, known=w.s[sel])
