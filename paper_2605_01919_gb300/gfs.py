"""Thin ctypes binding of the C ABI in include/gfs.h.

Only argument marshalling happens here: torch tensors provide device memory
and the current CUDA stream; every step of the computation runs in the
library's kernels.  There is no CPU fallback: if the shared library or a CUDA
device is missing, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

CODE_SURVIVOR, CODE_OPPOSITE, CODE_SAMPLE, CODE_OUTSIDE, CODE_INVALID, CODE_LOWER, CODE_TANGENT = range(7)
FLAG_LB_VIOL, FLAG_FAR_VIOL, FLAG_OPP_VIOL, FLAG_LOST_WITNESS = 0x10, 0x20, 0x40, 0x80
FLAG_SCORE_FALLBACK = 0x200

EXPORTED = ["gfs_default_options", "gfs_create", "gfs_set_stream", "gfs_build", "gfs_query", "gfs_query_tangent",
            "gfs_query_scored", "gfs_query_points", "gfs_query_backward", "gfs_query_backward_noalloc", "gfs_insert",
            "gfs_insert_known", "gfs_survivors", "gfs_batch_build", "gfs_batch_rebuild", "gfs_batch_status",
            "gfs_batch_query", "gfs_batch_query_tangent", "gfs_batch_survivors", "gfs_stats", "gfs_solve_host",
            "gfs_icosphere", "gfs_strerror", "gfs_destroy", "gfs_cell_coverage", "gfs_flood_order",
            "gfs_sphere_uncovered", "gfs_uncovered_intersections", "gfs_exact_rmin", "gfs_fma_probe"]


class Options(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_int), ("tol", ctypes.c_double), ("box_cull", ctypes.c_int),
                ("clamp_opp", ctypes.c_int), ("precision", ctypes.c_int), ("timing", ctypes.c_int),
                ("reserved", ctypes.c_int * 6)]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "n_spheres", "n_candidates", "n_survivors", "n_survivors_pos", "n_survivors_neg",
        "cull_fp64_rechecks", "query_fp64_rechecks", "query_deferred", "tree_levels",
        "query_sphere_node_tests", "query_sphere_items", "query_surv_node_tests", "query_band_passes",
        "query_surv_items")] + [(n, ctypes.c_double) for n in (
        "ms_build_total", "ms_build_cull", "ms_query_fast", "ms_query_exact")] + [
        (n, ctypes.c_int64) for n in ("kernel_launches", "sort_calls", "cull_node_tests", "cull_items")] + [
        ("ms_query_spheres", ctypes.c_double)] + [
        (n, ctypes.c_int64) for n in ("insert_rounds", "insert_steps", "insert_rebuilds")] + [
        (n, ctypes.c_double) for n in ("insert_ms_total", "insert_ms_rebuild", "insert_ms_final", "insert_ms_query",
                                       "insert_ms_commit", "insert_ms_update")] + [
        (n, ctypes.c_int64) for n in ("insert_slots", "insert_sph_exact", "insert_sph_tested", "insert_surv_exact",
                                      "insert_surv_tested", "batch_sphere_items", "batch_sphere_node_tests", "batch_surv_items")] + [
        ("batch_cull_tile", ctypes.c_int64 * 3), ("batch_query_grid", ctypes.c_int64)]


class Shape(ctypes.Structure):
    _fields_ = [("p_xyz", ctypes.c_void_p), ("s", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("x", ctypes.c_void_p), ("x_is_fp32", ctypes.c_int), ("m", ctypes.c_int64),
                ("s_out", ctypes.c_void_p), ("s64_out", ctypes.c_void_p), ("argmin_out", ctypes.c_void_p),
                ("flags_out", ctypes.c_void_p)]


class GfsError(RuntimeError):
    pass


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libgfs.so (building it first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise GfsError(f"CUDA library not built: {path}")
        _build.build()
    L = ctypes.CDLL(path)
    P, i64, i32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    L.gfs_default_options.argtypes = [ctypes.POINTER(Options)]
    L.gfs_default_options.restype = None
    L.gfs_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(Options), P]
    L.gfs_create.restype = i32
    L.gfs_set_stream.argtypes = [P, P]
    L.gfs_set_stream.restype = i32
    L.gfs_build.argtypes = [P, P, P, i64]
    L.gfs_build.restype = i32
    L.gfs_query.argtypes = [P, P, i32, i64, P, P, P, P]
    L.gfs_query.restype = i32
    L.gfs_query_tangent.argtypes = [P, P, i32, i64, P, P, P, P]
    L.gfs_query_tangent.restype = i32
    L.gfs_query_scored.argtypes = [P, P, i32, i64, P, P, P, P]
    L.gfs_query_scored.restype = i32
    L.gfs_query_backward.argtypes = [P, P, i32, i64, P, P, P, P, P, P, P]
    L.gfs_query_backward.restype = i32
    L.gfs_insert.argtypes = [P, P, i64, P, P, P]
    L.gfs_insert.restype = i32
    L.gfs_insert_known.argtypes = [P, P, P, i64, P, P, P]
    L.gfs_insert_known.restype = i32
    L.gfs_batch_build.argtypes = [P, P, i32]
    L.gfs_batch_build.restype = i32
    L.gfs_batch_query.argtypes = [P]
    L.gfs_batch_query.restype = i32
    L.gfs_batch_rebuild.argtypes = [P]
    L.gfs_batch_rebuild.restype = i32
    L.gfs_batch_status.argtypes = [P, ctypes.POINTER(ctypes.c_uint)]
    L.gfs_batch_status.restype = i32
    L.gfs_batch_query_tangent.argtypes = [P]
    L.gfs_batch_query_tangent.restype = i32
    L.gfs_batch_survivors.argtypes = [P, i32, P, i64, ctypes.POINTER(i64)]
    L.gfs_batch_survivors.restype = i32
    L.gfs_survivors.argtypes = [P, P, i64, ctypes.POINTER(i64)]
    L.gfs_survivors.restype = i32
    L.gfs_stats.argtypes = [P, ctypes.POINTER(Stats)]
    L.gfs_stats.restype = i32
    L.gfs_solve_host.argtypes = [P, P, P, i64, P, i32, i64, P, P, P]
    L.gfs_solve_host.restype = i32
    L.gfs_query_points.argtypes = [P, P, i32, i64, P, P, P]
    L.gfs_query_points.restype = i32
    L.gfs_sphere_uncovered.argtypes = [P, P, P]
    L.gfs_uncovered_intersections.argtypes = [P, i64, P, i64, P, P, P]
    L.gfs_uncovered_intersections.restype = i32
    L.gfs_exact_rmin.argtypes = [P, P, P, i64, P]
    L.gfs_exact_rmin.restype = i32
    L.gfs_sphere_uncovered.restype = i32
    L.gfs_cell_coverage.argtypes = [P, P, i64, P, f64, i32, P]
    L.gfs_cell_coverage.restype = i32
    L.gfs_flood_order.argtypes = [P, P, i64, P]
    L.gfs_flood_order.restype = i32
    L.gfs_fma_probe.argtypes = [i32, i64, i32, P, i64, P, ctypes.POINTER(f64)]
    L.gfs_fma_probe.restype = i32
    L.gfs_icosphere.argtypes = [i32, P, i64]
    L.gfs_icosphere.restype = i32
    L.gfs_strerror.argtypes = [i32]
    L.gfs_strerror.restype = ctypes.c_char_p
    L.gfs_destroy.argtypes = [P]
    L.gfs_destroy.restype = None
    _lib = L
    return L


def _check(st: int):
    if st != 0:
        raise GfsError(f"gfs error {st}: {load().gfs_strerror(st).decode()}")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def fma_probe(fp64: bool, iters: int, sink: torch.Tensor, blocks_per_sm: int = 4,
              stream: torch.cuda.Stream | None = None) -> float:
    """Launch the FMA peak probe (FP32 or FP64) on `stream` (default: the
    current stream); returns the launch's flop count."""
    st = stream if stream is not None else torch.cuda.current_stream()
    flops = ctypes.c_double(0.0)
    _check(load().gfs_fma_probe(int(fp64), int(iters), int(blocks_per_sm), _ptr(sink),
                                sink.numel() * sink.element_size(), ctypes.c_void_p(st.cuda_stream),
                                ctypes.byref(flops)))
    return flops.value


def icosphere(tau: int):
    """The library's direction table (host computation), numpy (K, 3)."""
    import numpy as np
    K = 10 * 4 ** tau + 2
    out = np.zeros((K, 3), dtype=np.float64)
    k = load().gfs_icosphere(tau, out.ctypes.data_as(ctypes.c_void_p), K)
    if k != K:
        raise GfsError("icosphere construction failed")
    return out


def flood_order(cells, counts):
    """Flood-fill refinement order (Sec. 4.2) of cells ((c, 3) integer
    coordinates) with covered counts (c,): host computation in the library,
    returns the cell indices in order (numpy int64)."""
    import numpy as np
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    counts = np.ascontiguousarray(counts, dtype=np.uint32)
    assert cells.ndim == 2 and cells.shape[1] == 3 and counts.shape == (cells.shape[0],)
    out = np.zeros(cells.shape[0], dtype=np.int64)
    _check(load().gfs_flood_order(cells.ctypes.data_as(ctypes.c_void_p), counts.ctypes.data_as(ctypes.c_void_p),
                                  cells.shape[0], out.ctypes.data_as(ctypes.c_void_p)))
    return out


class Context:
    """A sample set with its candidate/survivor hierarchies on one device."""

    def __init__(self, tau: int = 3, tol: float = 1e-6, box_cull: bool = True, clamp_opp: bool = True,
                 precision: int = 0, stream: torch.cuda.Stream | None = None, timing: bool = False,
                 tangent: bool = False):
        """tangent: every query is followed by the same-sign tangent
        augmentation (gfs_query_tangent), also under ConsistentSDF."""
        if not torch.cuda.is_available():
            raise GfsError("no CUDA device: the consistent-SDF library has no CPU path")
        L = load()
        opt = Options()
        L.gfs_default_options(ctypes.byref(opt))
        opt.tau, opt.tol, opt.box_cull, opt.clamp_opp, opt.precision = tau, tol, int(box_cull), int(clamp_opp), precision
        opt.timing = int(timing)
        self.opt = opt
        self.tau = tau
        self.tangent = tangent
        self.K = 10 * 4 ** tau + 2
        self._stream = stream
        h = ctypes.c_void_p()
        _check(L.gfs_create(ctypes.byref(h), ctypes.byref(opt), self._stream_handle()))
        self._h = h
        self.n = 0
        self.p = None
        self.s = None

    def _stream_handle(self):
        st = self._stream if self._stream is not None else torch.cuda.current_stream()
        return ctypes.c_void_p(st.cuda_stream)

    def _sync_stream(self):
        _check(load().gfs_set_stream(self._h, self._stream_handle()))

    def close(self):
        if getattr(self, "_h", None):
            load().gfs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- P build -------------------------------------------------------------
    def build(self, p: torch.Tensor, s: torch.Tensor):
        assert p.is_cuda and s.is_cuda and p.dtype == torch.float64 and s.dtype == torch.float64
        # what ConsistentSDF checks its sample tensors against: storage,
        # shape and in-place version of the tensors this state was built from
        built_from = (p.data_ptr(), s.data_ptr(), tuple(p.shape), tuple(s.shape), p._version, s._version)
        p = p.contiguous()
        s = s.contiguous()
        self._sync_stream()
        _check(load().gfs_build(self._h, _ptr(p), _ptr(s), p.shape[0]))
        self.n = p.shape[0]
        self.p, self.s = p, s
        self._built_from = built_from
        return self

    def built_from(self, p: torch.Tensor, s: torch.Tensor) -> bool:
        """True when the current state is the build of exactly these sample
        tensors, unmodified since (no insertion, no in-place change)."""
        rec = getattr(self, "_built_from", None)
        return rec is not None and rec == (p.data_ptr(), s.data_ptr(), tuple(p.shape), tuple(s.shape),
                                           p._version, s._version)

    # -- query ---------------------------------------------------------------
    def query(self, x: torch.Tensor, want_f64: bool = True):
        assert x.is_cuda and x.dtype in (torch.float64, torch.float32) and x.shape[-1] == 3
        x = x.contiguous()
        m = x.shape[0]
        dev = x.device
        out = {
            "s": torch.empty(m, dtype=torch.float32, device=dev),
            "s64": torch.empty(m, dtype=torch.float64, device=dev) if want_f64 else None,
            "argmin": torch.empty(m, dtype=torch.int64, device=dev),
            "flags": torch.empty(m, dtype=torch.int16, device=dev),
        }
        self.query_into(x, out["s"], out["s64"], out["argmin"], out["flags"])
        return out

    def query_into(self, x, s_out, s64_out, argmin_out, flags_out):
        self._sync_stream()
        _check(load().gfs_query(self._h, _ptr(x), int(x.dtype == torch.float32), x.shape[0], _ptr(s_out),
                                _ptr(s64_out), _ptr(argmin_out), _ptr(flags_out)))
        if self.tangent:
            self.tangent_into(x, s_out, s64_out, argmin_out, flags_out)

    def query_points(self, x, argmin, flags) -> torch.Tensor:
        """q*: the point that sets each value of a query's result (m, 3)
        FP64, NaN where no point does (SAMPLE, INVALID)."""
        x = x.contiguous()
        out = torch.empty((x.shape[0], 3), dtype=torch.float64, device=x.device)
        self._sync_stream()
        _check(load().gfs_query_points(self._h, _ptr(x), int(x.dtype == torch.float32), x.shape[0],
                                       _ptr(argmin.contiguous()), _ptr(flags.contiguous()), _ptr(out)))
        return out

    def tangent_into(self, x, s_out, s64_out, argmin_out, flags_out):
        """Same-sign tangent augmentation of a query's outputs, in place."""
        self._sync_stream()
        _check(load().gfs_query_tangent(self._h, _ptr(x), int(x.dtype == torch.float32), x.shape[0], _ptr(s_out),
                                        _ptr(s64_out), _ptr(argmin_out), _ptr(flags_out)))

    def scored_into(self, x, s_out, s64_out, argmin_out, flags_out):
        """Sec. 3.3 scored value over a query's outputs, in place."""
        self._sync_stream()
        _check(load().gfs_query_scored(self._h, _ptr(x), int(x.dtype == torch.float32), x.shape[0], _ptr(s_out),
                                       _ptr(s64_out), _ptr(argmin_out), _ptr(flags_out)))

    def query_scored(self, x: torch.Tensor):
        """The scored value at x (a plain query, then the scored pass)."""
        x = x.contiguous()
        out = self.query(x)
        self.scored_into(x, out["s"], out["s64"], out["argmin"], out["flags"])
        return out

    def backward(self, x, s, argmin, flags, grad_s, want_x=True, want_p=True, want_s=True):
        m = x.shape[0]
        dev = x.device
        gx = torch.empty((m, 3), dtype=torch.float32, device=dev) if want_x else None
        gp = torch.empty((self.n, 3), dtype=torch.float32, device=dev) if want_p else None
        gs = torch.empty(self.n, dtype=torch.float32, device=dev) if want_s else None
        self._sync_stream()
        _check(load().gfs_query_backward(self._h, _ptr(x.contiguous()), int(x.dtype == torch.float32), m,
                                         _ptr(s.contiguous()), _ptr(argmin.contiguous()),
                                         _ptr(flags.contiguous()), _ptr(grad_s.contiguous().float()),
                                         _ptr(gx), _ptr(gp), _ptr(gs)))
        return gx, gp, gs

    # -- greedy sequential insertion -------------------------------------------
    def insert(self, y: torch.Tensor, known: torch.Tensor | None = None):
        """Insert the rows of y in order (Sec. 4 greedy loop); returns the
        per-step FP64 value, argmin and result word.  known (optional, T FP64
        values on the device): their signs fix the points' classes and
        NONCONSERVATIVE marks values below them (Sec. 6 repair)."""
        assert y.is_cuda and y.dtype == torch.float64 and y.shape[-1] == 3
        y = y.contiguous()
        T = y.shape[0]
        if known is not None:
            assert known.is_cuda and known.dtype == torch.float64 and known.shape == (T,)
            known = known.contiguous()
        self._built_from = None   # the state now holds more samples than any caller's tensors
        out = {"s64": torch.empty(T, dtype=torch.float64, device=y.device),
               "argmin": torch.empty(T, dtype=torch.int64, device=y.device),
               "flags": torch.empty(T, dtype=torch.int16, device=y.device)}
        self._sync_stream()
        _check(load().gfs_insert_known(self._h, _ptr(y), _ptr(known), T, _ptr(out["s64"]), _ptr(out["argmin"]),
                                       _ptr(out["flags"])))
        self.n = self.stats()["n_spheres"]
        return out

    # -- exact coverage of the sample spheres (Prop. 1 (ii)) ----------------------
    def sphere_uncovered(self, witness: bool = False):
        """Per sphere of the current state (input order): 1 keeps a point
        outside every other shrunk ball, 0 fully covered, 2 undecided (its
        covering certificate outgrew 512 balls).  With witness=True also the
        (n, 3) float64 uncovered points (NaN rows where not uncovered)."""
        n = self.stats()["n_spheres"]
        out = torch.empty(n, dtype=torch.uint8, device="cuda")
        wit = torch.empty((n, 3), dtype=torch.float64, device="cuda") if witness else None
        self._sync_stream()
        _check(load().gfs_sphere_uncovered(self._h, _ptr(out), _ptr(wit) if wit is not None else None))
        return (out, wit) if witness else out

    def uncovered_intersections(self):
        """The U and D precomputation of Sec. 4.1: (circles (c, 2) int64 pairs
        i < j whose intersection circle keeps a point in no other shrunk ball,
        quads (u, 4) int64 (i, j, m, side) of the uncovered points shared by
        three spheres, points (u, 3) float64, status word), all on the device,
        sorted lexicographically."""
        L = load()
        counts = (ctypes.c_int64 * 3)()
        self._sync_stream()
        rc = L.gfs_uncovered_intersections(self._h, 0, None, 0, None, None, counts)
        if rc not in (0, 1):   # 1 = GFS_ERR_ARG: the counts are set
            _check(rc)
        nc, npt = int(counts[0]), int(counts[1])
        circ = torch.empty((nc, 2), dtype=torch.int64, device="cuda")
        quads = torch.empty((npt, 4), dtype=torch.int64, device="cuda")
        pts = torch.empty((npt, 3), dtype=torch.float64, device="cuda")
        _check(L.gfs_uncovered_intersections(self._h, nc, _ptr(circ) if nc else None, npt,
                                             _ptr(quads) if npt else None, _ptr(pts) if npt else None, counts))
        return circ, quads, pts, int(counts[2])

    def exact_rmin(self, x: torch.Tensor, sigma: torch.Tensor) -> torch.Tensor:
        """Exact minimum valid radius for a known sign (Sec. 6) over T, U, D
        at points x ((m, 3) float64 cuda) for signs sigma ((m,) int8 cuda:
        +1, -1, 0); (m,) float64, inf where no candidate exists."""
        x = x.contiguous()
        sigma = sigma.to(torch.int8).contiguous()
        out = torch.empty(x.shape[0], dtype=torch.float64, device="cuda")
        self._sync_stream()
        _check(load().gfs_exact_rmin(self._h, _ptr(x), _ptr(sigma), int(x.shape[0]), _ptr(out)))
        return out

    # -- refinement order (Sec. 4.2) ------------------------------------------------
    def cell_coverage(self, cells: torch.Tensor, origin, h: float, sub: int = 8) -> torch.Tensor:
        """Covered sub-point counts of grid cells (cells: (c, 3) int32 cuda
        integer coordinates; points origin + h * (ijk + (abc + 1/2) / sub))
        against the current samples' balls; returns (c,) int32 counts."""
        import numpy as np
        assert cells.is_cuda and cells.dtype == torch.int32 and cells.shape[-1] == 3
        cells = cells.contiguous()
        o = np.ascontiguousarray(origin, dtype=np.float64)
        out = torch.empty(cells.shape[0], dtype=torch.int32, device=cells.device)
        self._sync_stream()
        _check(load().gfs_cell_coverage(self._h, _ptr(cells), cells.shape[0], o.ctypes.data_as(ctypes.c_void_p),
                                        float(h), int(sub), _ptr(out)))
        return out

    def survivors(self) -> torch.Tensor:
        cnt = ctypes.c_int64(0)
        self._sync_stream()
        # first call sizes the output (status GFS_ERR_ARG when it is too small), second fills it
        st = load().gfs_survivors(self._h, None, 0, ctypes.byref(cnt))
        if st not in (0, 1):
            _check(st)
        out = torch.empty(max(cnt.value, 1), dtype=torch.int64, device="cuda")
        _check(load().gfs_survivors(self._h, _ptr(out), out.numel(), ctypes.byref(cnt)))
        return out[: cnt.value]

    def solve_host(self, p, s, x, s_out, argmin_out, flags_out):
        """Whole path from host (numpy or pinned torch CPU) buffers."""
        def ptr(a):
            if a is None:
                return None
            return ctypes.c_void_p(a.data_ptr() if isinstance(a, torch.Tensor) else a.ctypes.data)
        is32 = int((x.dtype == torch.float32) if isinstance(x, torch.Tensor) else (x.dtype.itemsize == 4))
        self._sync_stream()
        _check(load().gfs_solve_host(self._h, ptr(p), ptr(s), p.shape[0], ptr(x), is32, x.shape[0],
                                     ptr(s_out), ptr(argmin_out), ptr(flags_out)))
        self.n = p.shape[0]

    # -- batched shapes -----------------------------------------------------------
    def batch_build(self, shapes):
        """shapes: list of dicts with CUDA tensors p (n,3) f64, s (n,) f64 and
        x (m,3) f64/f32.  Allocates each shape's outputs (returned as a list of
        dicts) and builds every shape in one pass; keep the returned list alive
        while calling batch_query."""
        arr = (Shape * len(shapes))()
        outs = []
        for k, sh in enumerate(shapes):
            p, sv, x = sh["p"].contiguous(), sh["s"].contiguous(), sh["x"].contiguous()
            m = x.shape[0]
            o = {"p": p, "s_in": sv, "x": x,
                 "s": torch.empty(m, dtype=torch.float32, device=x.device),
                 "s64": torch.empty(m, dtype=torch.float64, device=x.device),
                 "argmin": torch.empty(m, dtype=torch.int64, device=x.device),
                 "flags": torch.empty(m, dtype=torch.int16, device=x.device)}
            arr[k] = Shape(p.data_ptr(), sv.data_ptr(), p.shape[0], x.data_ptr(), int(x.dtype == torch.float32), m,
                           o["s"].data_ptr(), o["s64"].data_ptr(), o["argmin"].data_ptr(), o["flags"].data_ptr())
            outs.append(o)
        self._sync_stream()
        _check(load().gfs_batch_build(self._h, ctypes.cast(arr, ctypes.c_void_p), len(shapes)))
        self._batch = outs
        return outs

    def batch_rebuild(self):
        """Repeat the last batch_build from the shapes' current sample values
        (same tensors, same sizes): no host synchronisation or allocation, so
        it can be captured in a CUDA graph with batch_query."""
        self._sync_stream()
        _check(load().gfs_batch_rebuild(self._h))
        return self._batch

    def batch_status(self) -> int:
        """Status bits of the batched builds since the last call (0: complete;
        1/2: survivor capacity exceeded; 4: node capacity exceeded)."""
        st = ctypes.c_uint(0)
        self._sync_stream()
        _check(load().gfs_batch_status(self._h, ctypes.byref(st)))
        return st.value

    def batch_query(self):
        self._sync_stream()
        _check(load().gfs_batch_query(self._h))
        if self.tangent:
            _check(load().gfs_batch_query_tangent(self._h))
        return self._batch

    def batch_survivors(self, shape: int) -> torch.Tensor:
        cnt = ctypes.c_int64(0)
        self._sync_stream()
        st = load().gfs_batch_survivors(self._h, shape, None, 0, ctypes.byref(cnt))
        if st not in (0, 1):
            _check(st)
        out = torch.empty(max(cnt.value, 1), dtype=torch.int64, device="cuda")
        _check(load().gfs_batch_survivors(self._h, shape, _ptr(out), out.numel(), ctypes.byref(cnt)))
        return out[: cnt.value]

    def stats(self) -> dict:
        st = Stats()
        _check(load().gfs_stats(self._h, ctypes.byref(st)))
        return {n: (list(getattr(st, n)) if n == "batch_cull_tile" else getattr(st, n)) for n, _ in Stats._fields_}


class ConsistentSDF(torch.autograd.Function):
    """s*(x) with a hand-written adjoint: gradients flow to the query points,
    and to the sample positions and values through the argmin.

    Usage: ``s = ConsistentSDF.apply(x, p, s_samples, ctx)`` where ``ctx`` is
    a :class:`Context` built on (p, s_samples)."""

    @staticmethod
    def forward(fctx, x, p, s_samples, gctx: Context):
        if not gctx.built_from(p, s_samples):
            raise GfsError("ConsistentSDF: the context was not built from these sample tensors, or they "
                           "changed since its build (in place, or by an insertion); call ctx.build(p, s) first")
        out = gctx.query(x, want_f64=False)
        fctx.gctx = gctx
        fctx.save_for_backward(x, out["s"], out["argmin"], out["flags"])
        return out["s"]

    @staticmethod
    def backward(fctx, grad_s):
        x, s, argmin, flags = fctx.saved_tensors
        need_x, need_p, need_s = fctx.needs_input_grad[0], fctx.needs_input_grad[1], fctx.needs_input_grad[2]
        gx, gp, gs = fctx.gctx.backward(x, s, argmin, flags, grad_s, need_x, need_p, need_s)
        return (gx.to(x.dtype) if gx is not None else None,
                gp.to(torch.float64) if gp is not None else None,
                gs.to(torch.float64) if gs is not None else None, None)
