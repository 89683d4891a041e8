"""Host-side checks of the C-ABI library (no device needed): it builds for
sm_103a, loads, exports every entry point include/gfs.h declares, and its
host logic (icosphere table, option checks, error names) behaves."""
import ctypes
import os
import re

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gfs():
    from paper_2605_01919_gb300 import gfs as G
    G.load()
    return G


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "gfs.h")).read()
    return sorted(set(re.findall(r"\b(gfs_[a-z0-9_]+)\s*\(", hdr)))


def test_exports_every_declared_symbol(gfs):
    L = gfs.load()
    names = declared_symbols()
    assert len(names) >= 11
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(gfs.EXPORTED)   # the binding lists every entry point, and no other


def test_icosphere_table_matches_oracle_bitwise(gfs, orc):
    # two independent implementations of the documented construction
    for tau in range(0, 6):
        a, b = gfs.icosphere(tau), orc.icosphere(tau)
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64))


def test_icosphere_bad_args(gfs):
    L = gfs.load()
    buf = np.zeros((12, 3))
    assert L.gfs_icosphere(-1, buf.ctypes.data_as(ctypes.c_void_p), 12) == -1
    assert L.gfs_icosphere(1, buf.ctypes.data_as(ctypes.c_void_p), 12) == -1   # needs 42 rows


def test_option_validation_and_errors(gfs):
    L = gfs.load()
    opt = gfs.Options()
    L.gfs_default_options(ctypes.byref(opt))
    assert (opt.tau, opt.tol, opt.box_cull, opt.clamp_opp, opt.precision) == (3, 1e-6, 1, 1, 0)
    h = ctypes.c_void_p()
    bad = gfs.Options()
    L.gfs_default_options(ctypes.byref(bad))
    bad.tau = 9
    assert L.gfs_create(ctypes.byref(h), ctypes.byref(bad), None) == 1       # GFS_ERR_ARG
    bad.tau = 2
    bad.reserved[0] = 5
    assert L.gfs_create(ctypes.byref(h), ctypes.byref(bad), None) == 1
    assert L.gfs_strerror(0) == b"ok"
    assert b"argument" in L.gfs_strerror(1)
    # null handles are rejected before touching a device
    assert L.gfs_build(None, None, None, 5) == 1
    assert L.gfs_query(None, None, 0, 1, None, None, None, None) == 1


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-device path")
def test_no_device_fails_loudly(gfs):
    L = gfs.load()
    h = ctypes.c_void_p()
    assert L.gfs_create(ctypes.byref(h), None, None) == 3                      # GFS_ERR_CUDA
    with pytest.raises(gfs.GfsError):
        gfs.Context()


def test_flood_order_matches_oracle(gfs, orc):
    """The library's flood-fill order (host code) equals the oracle's on the
    hand-worked cases and on random sparse cell sets, ties included."""
    from tests.test_oracle import FLOOD_CASES
    for cells, counts, order in FLOOD_CASES:
        assert list(gfs.flood_order(np.array(cells), np.array(counts))) == order
    rng = np.random.default_rng(11)
    for trial in range(20):
        side = int(rng.integers(2, 12))
        all_cells = np.array([(i, j, k) for i in range(side) for j in range(side) for k in range(side)]) - side // 2
        cells = all_cells[rng.random(all_cells.shape[0]) < rng.uniform(0.05, 0.6)]
        if cells.shape[0] == 0:
            continue
        cells = cells[rng.permutation(cells.shape[0])]
        counts = rng.integers(0, 6, cells.shape[0])        # many ties
        assert list(gfs.flood_order(cells, counts)) == orc.flood_order(cells, counts)


def test_flood_order_errors(gfs):
    L = gfs.load()
    P = ctypes.c_void_p
    cells = np.array([[0, 0, 0], [1, 0, 0], [0, 0, 0]], dtype=np.int32)
    counts = np.zeros(3, dtype=np.uint32)
    out = np.zeros(3, dtype=np.int64)
    args = [cells.ctypes.data_as(P), counts.ctypes.data_as(P)]
    assert L.gfs_flood_order(*args, 3, out.ctypes.data_as(P)) == 1          # a cell listed twice
    assert L.gfs_flood_order(*args, 2, out.ctypes.data_as(P)) == 0
    assert list(out[:2]) == [0, 1]
    assert L.gfs_flood_order(*args, 0, out.ctypes.data_as(P)) == 0          # empty
    assert L.gfs_flood_order(None, None, 2, None) == 1
    far = np.array([[1 << 21, 0, 0]], dtype=np.int32)
    assert L.gfs_flood_order(far.ctypes.data_as(P), counts.ctypes.data_as(P), 1, out.ctypes.data_as(P)) == 6


def test_every_context_call_rejects_a_null_context(gfs):
    """Each entry point that takes a context returns GFS_ERR_ARG for a null
    one, before touching a device."""
    L = gfs.load()
    origin = np.zeros(3)
    calls = [
        lambda: L.gfs_set_stream(None, None),
        lambda: L.gfs_query_tangent(None, None, 0, 1, None, None, None, None),
        lambda: L.gfs_query_points(None, None, 0, 1, None, None, None),
        lambda: L.gfs_query_backward(None, None, 0, 1, None, None, None, None, None, None, None),
        lambda: L.gfs_insert(None, None, 1, None, None, None),
        lambda: L.gfs_insert_known(None, None, None, 1, None, None, None),
        lambda: L.gfs_survivors(None, None, 0, ctypes.byref(ctypes.c_int64())),
        lambda: L.gfs_sphere_uncovered(None, None, None),
        lambda: L.gfs_uncovered_intersections(None, 0, None, 0, None, None, None),
        lambda: L.gfs_exact_rmin(None, None, None, 1, None),
        lambda: L.gfs_cell_coverage(None, None, 1, origin.ctypes.data_as(ctypes.c_void_p), 0.1, 8, None),
        lambda: L.gfs_batch_build(None, None, 1),
        lambda: L.gfs_batch_query(None),
        lambda: L.gfs_batch_query_tangent(None),
        lambda: L.gfs_batch_survivors(None, 0, None, 0, ctypes.byref(ctypes.c_int64())),
    ]
    for call in calls:
        assert call() == 1
