"""Refinement order (Sec. 4.2) on the GPU: covered sub-point counts of grid
cells (gfs_cell_coverage) against the oracle's brute force, bit for bit, and
a greedy refinement run in flood-fill order against the oracle's sequential
loop in the same order."""
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


def surface_cells(w):
    """Cells of the node-aligned grid with a corner sample within half a cell
    diagonal of the surface (the cells that may contain it)."""
    N = round(w.n ** (1 / 3))
    S = w.s.reshape(N, N, N)
    near = np.abs(S) < 0.5 * np.sqrt(3) * w.h
    cell = np.zeros((N - 1,) * 3, dtype=bool)
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                cell |= near[a:N - 1 + a, b:N - 1 + b, c:N - 1 + c]
    return np.argwhere(cell).astype(np.int32)


def gpu_counts(G, w, cells, sub, tau=None):
    ctx = G.Context(tau=w.tau if tau is None else tau)
    ctx.build(torch.from_numpy(w.p).cuda(), torch.from_numpy(w.s).cuda())
    out = ctx.cell_coverage(torch.from_numpy(cells).cuda(), [-1.0, -1.0, -1.0], w.h, sub)
    torch.cuda.synchronize()
    ctx.close()
    return out.cpu().numpy().astype(np.uint32)


@pytest.mark.parametrize("sub", [1, 3, 8])
def test_cell_coverage_parity(G, orc, sub):
    """Surface cells of a 12^3 union grid plus random cells (some outside
    the grid)."""
    w = W.union_grid(N=12, up=4)
    cells = surface_cells(w)
    rng = np.random.default_rng(sub)
    cells = np.concatenate([cells, rng.integers(-2, 13, size=(60, 3)).astype(np.int32)])
    want = orc.cell_coverage(w.p, w.s, cells, [-1.0, -1.0, -1.0], w.h, sub)
    assert 0 < want.sum() < cells.shape[0] * sub ** 3
    assert np.array_equal(gpu_counts(G, w, cells, sub), want)


def test_cell_coverage_full_size_sampled(G, orc):
    """Every surface cell of the 64^3 union grid (262,144 samples) on the
    GPU; 40 sampled cells against the oracle."""
    w = W.union_grid()
    cells = surface_cells(w)
    got = gpu_counts(G, w, cells, 8)
    sel = np.random.default_rng(3).choice(cells.shape[0], 40, replace=False)
    want = orc.cell_coverage(w.p, w.s, cells[sel], [-1.0, -1.0, -1.0], w.h, 8)
    assert np.array_equal(got[sel], want)
    assert got.min() < got.max()


def test_flood_order_refinement_parity(G, orc):
    """Refinement of a 10^3 union grid at its surface cell centres in
    flood-fill order (counts from the GPU, order from the library's host
    code): the order equals the oracle's, and every insertion step equals
    the oracle's sequential loop in that order."""
    w = W.union_grid(N=10, up=2, tau=2)
    cells = surface_cells(w)
    counts = gpu_counts(G, w, cells, 8)
    assert np.array_equal(counts, orc.cell_coverage(w.p, w.s, cells, [-1.0, -1.0, -1.0], w.h, 8))
    order = G.flood_order(cells, counts)
    assert list(order) == orc.flood_order(cells, counts)
    y = -1.0 + w.h * (cells[order].astype(np.float64) + 0.5)
    U = orc.icosphere(w.tau)
    val, arg, fl, _ = orc.insert(w.p, w.s, U, y)
    ctx = G.Context(tau=w.tau)
    ctx.build(torch.from_numpy(w.p).cuda(), torch.from_numpy(w.s).cuda())
    out = ctx.insert(torch.from_numpy(np.ascontiguousarray(y)).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(out["flags"].cpu().numpy().astype(np.int32) & 0xFFFF, fl)
    assert np.array_equal(out["argmin"].cpu().numpy(), arg)
    assert np.array_equal(out["s64"].cpu().numpy(), val, equal_nan=True)
    ctx.close()
