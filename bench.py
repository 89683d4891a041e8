"""Benchmark: consistent SDF queries per second, including the P build.

One step = the whole hot path over one synthetic workload: build the sphere
hierarchy, generate and cull all candidates (P build), build the survivor
hierarchies, and evaluate the consistent value at every query point.
Workload: 64^3 node grid over [-1,1]^3 sampling the union of 6 spheres and 4
boxes (seeded), icosphere depth 3 (642 candidates per sample), 4x upsampled
253^3 = 16,194,277 query points.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle instead
(a bounded sample per step, extrapolated to the same workload).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "union64_tau3_q253"
CONFIG = {
    "workload": WORKLOAD,
    "samples": "64^3 node grid on [-1,1]^3, union of 6 spheres + 4 boxes (seed 2000)",
    "tau": 3,
    "candidates": 64 ** 3 * 642,
    "queries": 253 ** 3,
    "query_dtype": "f64",
}
METRIC = "consistent SDF queries/sec (incl. P build)"
UNIT = "queries/s"
FP32_LANES = 128   # FP32 lanes per SM (nominal figure, reported beside the measured peak)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gfs", choices=["gfs", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the sub-benchmarks of the backward, insertion and batched paths")
    ap.add_argument("--only", choices=["backward", "repair", "insert", "batch", "tangent", "refine_order",
                                       "exact_coverage", "sphere16", "scored"],
                    default=None,
                    help="run one sub-benchmark alone and print its JSON (profiling)")
    ap.add_argument("--insert-steps", type=int, default=8192)
    ap.add_argument("--repair-steps", type=int, default=1 << 20)
    ap.add_argument("--batch-shapes", type=int, default=256)
    ap.add_argument("--batch-scale", type=float, default=1.0,
                    help="scale of the batch shapes' grid sides and sample counts (1 = the full workload)")
    ap.add_argument("--tangent-every", type=int, default=256,
                    help="tangent sub-benchmark: use every k-th of the 253^3 points (the pass is FP64, one "
                         "thread per point)")
    ap.add_argument("--exact-csg", type=int, default=64,
                    help="exact-coverage sub-benchmark: side of the CSG grid")
    ap.add_argument("--exact-only-csg", action="store_true",
                    help="exact-coverage sub-benchmark: the CSG grid alone (small cases for profiler captures)")
    ap.add_argument("--scored-every", type=int, default=256,
                    help="scored sub-benchmark: use every k-th of the 253^3 points")
    ap.add_argument("--query-subsample", type=int, default=1,
                    help="use every k-th query point (small cases for profiler captures)")
    return ap.parse_args()


def aggregate(total_ms: float, units_per_rank: int, steps: int, world: int, device=None):
    """Whole-job throughput of `world` replicas: every rank processed
    units_per_rank units per step; the job time is the slowest rank's.
    Returns (value, ms_per_step).  Uses torch.distributed when world > 1."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / steps
    return world * units_per_rank / (ms_per_step / 1e3), ms_per_step


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def gpu_numa_cpus(gpu_index: int):
    """CPUs of the NUMA node the GPU is attached to (from nvidia-smi's PCI bus
    id and sysfs), or None.  Pinned host buffers first touched from those CPUs
    sit next to the GPU's host link."""
    try:
        bus = subprocess.run(["nvidia-smi", f"--id={gpu_index}", "--query-gpu=pci.bus_id",
                              "--format=csv,noheader"], capture_output=True, text=True, timeout=20).stdout.strip()
        dom, rest = bus.split(":", 1)
        bdf = f"{int(dom, 16):04x}:{rest}".lower()
        node = int(open(f"/sys/bus/pci/devices/{bdf}/numa_node").read())
        if node < 0:
            return None
        cpus = set()
        for part in open(f"/sys/devices/system/node/node{node}/cpulist").read().strip().split(","):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        return node, cpus
    except Exception:
        return None


# ----------------------------------------------------------------------------
# measured arithmetic peaks (the denominators of the ALU rooflines)
# ----------------------------------------------------------------------------
def measure_alu_peaks(dev, local, seconds=0.6):
    """FP32 and FP64 fused multiply-add rates of this GPU, from the library's
    probe kernel (independent FMA chains on every SM), timed with CUDA events
    on the launching stream: the best launch (burst) and the median over a
    loop of about `seconds` (sustained), with the SM clock sampled meanwhile."""
    import torch
    from paper_2605_01919_gb300 import gfs
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sink = torch.empty(sms * 8 * 256, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    out = {"sm_count": sms, "probe": "gfs_fma_probe: 4 blocks x 256 threads per SM, 16 independent FMA chains "
                                     "per thread"}
    clocks = ClockSampler(local)
    clocks.start()
    for name, fp64 in (("fp32", False), ("fp64", True)):
        iters = 64
        for _ in range(12):            # size one launch to about 20 ms
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            gfs.fma_probe(fp64, iters, sink, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            if ms > 10.0:
                break
            iters = int(iters * max(2.0, min(64.0, 20.0 / max(ms, 1e-3))))
        ts, flops = [], 0.0
        t_end = time.perf_counter() + seconds
        while time.perf_counter() < t_end or len(ts) < 5:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            flops = gfs.fma_probe(fp64, iters, sink, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        out[f"{name}_tflops"] = flops / (min(ts) / 1e3) / 1e12
        out[f"{name}_tflops_sustained"] = flops / (float(np.median(ts)) / 1e3) / 1e12
        out[f"{name}_launch_ms"] = float(np.median(ts))
    out["clocks"] = clocks.stop()
    out["fp32_tflops_nominal_max_clock"] = sms * FP32_LANES * 2 * 2070.0e6 / 1e12
    return out


def alu_roofline(kernel, units, flops_per_unit, unit_def, ms, peaks, fp64=False, **extra):
    """Roofline block of an ALU-bound kernel: algorithmic flops (units x
    flops per unit) over its measured duration, against the measured FMA
    peak of the pipe that bounds it."""
    key = "fp64_tflops" if fp64 else "fp32_tflops"
    peak = peaks.get(key) if peaks else None
    achieved = flops_per_unit * units / (ms / 1e3) / 1e12 if ms and ms > 0 else None
    r = {"kernel": kernel, "bound": "alu", "pipe": "fp64" if fp64 else "fp32", "achieved": achieved, "peak": peak,
         "unit": "TFLOP/s", "frac": (achieved / peak) if (achieved is not None and peak) else None,
         "traffic": None, "units_per_launch": units, "flops_per_unit": flops_per_unit, "unit_def": unit_def,
         "ms_per_launch": ms, "peak_source": f"measured {key} (FMA probe, burst) in this run"}
    r.update(extra)
    return r


def hbm_roofline(kernel, bytes_, unit_def, ms, **extra):
    peak = measured_peaks().get("hbm_gbs")
    achieved = bytes_ / (ms / 1e3) / 1e9 if ms and ms > 0 else None
    r = {"kernel": kernel, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
         "frac": (achieved / peak) if (achieved is not None and peak) else None, "traffic": None,
         "bytes_per_launch": bytes_, "unit_def": unit_def, "ms_per_launch": ms,
         "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"}
    r.update(extra)
    return r


# ----------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the same workload
# ----------------------------------------------------------------------------
_ORC = {}


def _oracle_init(p, s, tau):
    """Worker start-up: the workload and the icosphere table, loaded once."""
    from oracle import oracle as O
    _ORC.update(O=O, p=p, s=s, U=O.icosphere(tau))


def _oracle_chunk(args):
    """One worker's share of an oracle sample: keep decisions for the given
    (sphere, direction) pairs, then the lazy oracle at the given points."""
    pairs, xq = args
    O, p, s, U = _ORC["O"], _ORC["p"], _ORC["s"], _ORC["U"]
    for i, k in pairs:
        O.keep_one(p, s, U, int(i), int(k))
    if len(xq):
        O.query_lazy(p, s, U, xq)
    return True


def cpu_baseline_line(w, x, steps: int, n_keep: int = 2000, n_query: int = 2, procs: int | None = None):
    """The FP64 oracle on the host cores: `procs` spawned worker processes
    (default: all cores, at most 16) each time keep decisions and lazy
    queries of a seeded random sample; the wall-clock time per unit of each
    phase, over all workers, is extrapolated to the whole workload."""
    import multiprocessing as mp
    procs = procs or max(1, min(16, os.cpu_count() or 1))
    K = 10 * 4 ** w.tau + 2
    tk, tq = [], []
    with mp.get_context("spawn").Pool(procs, initializer=_oracle_init, initargs=(w.p, w.s, w.tau)) as pool:
        pool.map(_oracle_chunk, [([], np.zeros((0, 3)))] * procs)   # start-up, not timed
        for st in range(steps):
            rng = np.random.default_rng(st)
            ii = rng.integers(0, w.n, n_keep * procs)
            kk = rng.integers(0, K, n_keep * procs)
            jobs = [(list(zip(ii[c::procs], kk[c::procs])), np.zeros((0, 3))) for c in range(procs)]
            t0 = time.perf_counter()
            pool.map(_oracle_chunk, jobs, chunksize=1)
            tk.append((time.perf_counter() - t0) / (n_keep * procs))
            sel = rng.integers(0, x.shape[0], n_query * procs)
            jobs = [([], x[sel[c:c + 1]].astype(np.float64)) for c in range(sel.size)]
            t0 = time.perf_counter()
            pool.map(_oracle_chunk, jobs, chunksize=1)
            tq.append((time.perf_counter() - t0) / sel.size)
    t_keep, t_q = float(np.mean(tk)), float(np.mean(tq))
    total = w.n * K * t_keep + x.shape[0] * t_q
    return {
        "value": x.shape[0] / total,
        "unit": UNIT,
        "cores": procs,
        "kind": "oracle",
        "sample": (f"{steps} x ({n_keep * procs} random candidate keep decisions + {n_query * procs} random "
                   f"queries, lazy FP64 oracle, {procs} worker processes); extrapolated to {w.n * K} "
                   f"candidates + {x.shape[0]} queries from the wall-clock time per unit: "
                   f"{t_keep * 1e3:.4f} ms/candidate, {t_q:.3f} s/query"),
    }


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2605_01919_gb300 import workloads as W
    w = W.union_grid()
    x = w.make_queries()
    cb = cpu_baseline_line(w, x, max(1, args.warmup + args.steps), n_keep=1000, n_query=2)
    line = {
        "impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * x.shape[0] / cb["value"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": CONFIG, "cpu_baseline": cb,
        "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(_finite(line)), flush=True)


# ----------------------------------------------------------------------------
# the CUDA path
# ----------------------------------------------------------------------------
KERNEL_TU = ("gfs_kernels.cu", "gfs_internal.cuh", "gfs_kernels.h")


def kernel_hash() -> str:
    """Hash of the sources of the single-shape query and cull kernels (the
    batched kernels in gfs_batch.cuh are separate kernels)."""
    h = hashlib.sha256()
    for f in KERNEL_TU:
        h.update(open(os.path.join(ROOT, "paper_2605_01919_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary of the kernel
    (profiles/<kernel>_union64.md, line "dram_bytes_per_launch: N
    source_hash: H"), if it was taken on the current kernel sources."""
    import re
    try:
        with open(os.path.join(ROOT, "profiles", f"{kernel}_union64.md")) as f:
            m = re.search(r"dram_bytes_per_launch:\s*(\d+)\s+source_hash:\s*([0-9a-f]+)", f.read())
        if m and m.group(2) == kernel_hash():
            return int(m.group(1))
    except OSError:
        pass
    return None



# ----------------------------------------------------------------------------
# sub-benchmarks of the other rows of the hot path (rank 0, one GPU)
# ----------------------------------------------------------------------------
def _ev_time(fn, reps=3, warm=True):
    """Median CUDA-event time (ms) of fn over reps runs, after one untimed
    run unless warm is False (fn has just run)."""
    import torch
    if warm:
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def extra_backward():
    """128^3 torus grid, tau 3, 2^22 uniform FP32 points: forward, and
    forward + hand-written backward (d/dx, d/dp_i, d/ds_i)."""
    import torch
    from paper_2605_01919_gb300 import gfs
    from paper_2605_01919_gb300 import workloads as W
    w = W.torus_grid()
    x = torch.from_numpy(w.make_queries()).cuda()
    p, s = torch.from_numpy(w.p).cuda(), torch.from_numpy(w.s).cuda()
    ctx = gfs.Context(tau=w.tau)
    t_build = _ev_time(lambda: ctx.build(p, s), reps=2)
    out = ctx.query(x, want_f64=False)
    g = torch.ones(x.shape[0], device="cuda")
    t_fwd = _ev_time(lambda: ctx.query(x, want_f64=False))
    t_bwd = _ev_time(lambda: ctx.backward(x, out["s"], out["argmin"], out["flags"], g))
    m = x.shape[0]
    n = w.n
    ctx.close()
    # the adjoint reads each point's coordinates, value, argmin, result word and
    # upstream gradient and writes its d/dx (42 B per point), and writes d/dp
    # and d/ds of every sample (16 B per sample)
    roof = hbm_roofline("k_query_grad", 42 * m + 16 * n, "42 B per query point + 16 B per sample", t_bwd)
    return {"workload": "torus128_tau3_2^22_fp32_points", "roofline": roof, "build_ms": t_build, "forward_ms": t_fwd,
            "backward_ms": t_bwd, "forward_queries_per_s": m / (t_fwd / 1e3),
            "forward_backward_queries_per_s": m / ((t_fwd + t_bwd) / 1e3),
            "queries_per_s_incl_build": m / ((t_build + t_fwd) / 1e3)}


def extra_insert(T=8192, peaks=None):
    """Greedy sequential refinement on the 128^3 CSG pseudo-SDF (tau 3): new
    points at the centres of the cells whose eight corner samples do not all
    exceed half the cell diagonal (the cells that may contain the surface),
    inserted in index order, each against the inputs and every earlier
    insertion."""
    import torch
    from paper_2605_01919_gb300 import gfs
    from paper_2605_01919_gb300 import workloads as W
    w = W.csg_pseudo_grid()
    N = round(w.n ** (1 / 3))
    S = w.s.reshape(N, N, N)
    near = np.abs(S) < 0.5 * np.sqrt(3) * w.h
    cell = near[:-1, :-1, :-1] | near[1:, :-1, :-1] | near[:-1, 1:, :-1] | near[:-1, :-1, 1:] | \
        near[1:, 1:, :-1] | near[1:, :-1, 1:] | near[:-1, 1:, 1:] | near[1:, 1:, 1:]
    g = np.linspace(-1, 1, N)
    c = 0.5 * (g[:-1] + g[1:])
    ix, iy, iz = np.nonzero(cell)
    y = np.stack([c[ix], c[iy], c[iz]], axis=1)[:T]
    p, s = torch.from_numpy(w.p).cuda(), torch.from_numpy(w.s).cuda()
    ctx = gfs.Context(tau=w.tau, timing=True)
    t_build = _ev_time(lambda: ctx.build(p, s), reps=1)
    yt = torch.from_numpy(np.ascontiguousarray(y)).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = ctx.insert(yt)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    st = ctx.stats()
    fl = out["flags"].cpu().numpy().astype(np.int32) & 0xFFFF
    ctx.close()
    return {"workload": "csg128_tau3_refine_surface_cells", "candidate_cells": int(cell.sum()),
            "inserted": int(y.shape[0]), "build_ms": t_build, "insert_s": dt,
            "insertions_per_s": y.shape[0] / dt, "rounds": st["insert_rounds"],
            "roofline": _insert_roofline(st, peaks), "codes": np.bincount(fl & 15, minlength=6).tolist(),
            "lost_witness_steps": int(np.sum((fl & 0x80) != 0)),
            "far_violations": int(np.sum((fl & 0x20) != 0))}


def _insert_roofline(st, peaks):
    """Roofline of the insertion's step queries (k_ins_query): FP32 screens of
    spheres and survivors (8 flops each) over the query kernels' device time
    against the FP32 peak, with the FP64 evaluations (about 20 flops each:
    differences, products, a square root) against the FP64 peak beside it."""
    ms = st["insert_ms_query"]
    screens = st["insert_sph_tested"] + st["insert_surv_tested"]
    exact = st["insert_sph_exact"] + st["insert_surv_exact"]
    r = alu_roofline("k_ins_query", screens, 8, "(step point, sphere or survivor) FP32 screens of the step queries",
                     ms, peaks)
    if peaks and ms > 0:
        a64 = 20.0 * exact / (ms / 1e3) / 1e12
        r["fp64"] = {"units": exact, "flops_per_unit": 20, "achieved": a64, "peak": peaks.get("fp64_tflops"),
                     "frac": a64 / peaks["fp64_tflops"] if peaks.get("fp64_tflops") else None}
    r["launches"] = st["insert_rounds"]
    return r


def _repair_setup():
    """Sec. 6 repair set-up on the 128^3 CSG pseudo-SDF: build on all samples,
    decide each sphere's exact coverage (Prop. 1 (ii)), remove the covered
    ones (undecided spheres stay), rebuild on the rest."""
    import torch
    from paper_2605_01919_gb300 import gfs
    from paper_2605_01919_gb300 import workloads as W
    w = W.csg_pseudo_grid()
    p, s = torch.from_numpy(w.p).cuda(), torch.from_numpy(w.s).cuda()
    ctx = gfs.Context(tau=w.tau, timing=True)
    ctx.build(p, s)
    surv = ctx.survivors().cpu().numpy()
    cnt = np.bincount(surv // (ctx.K + 1), minlength=w.n)
    cov = {}
    cov["ms"] = _ev_time(lambda: cov.__setitem__("out", ctx.sphere_uncovered()), reps=1)
    out = cov["out"].cpu().numpy()
    removed = np.nonzero(out == 0)[0]
    info = {"exact_covered": int(removed.size), "exact_uncovered": int(np.sum(out == 1)),
            "undecided": int(np.sum(out == 2)), "no_survivor_at_tau": int(np.sum(cnt == 0)),
            "covered_with_survivor": int(np.sum((out == 0) & (cnt > 0))), "exact_coverage_ms": cov["ms"]}
    kept = torch.from_numpy(out != 0).cuda()
    return w, ctx, removed, p[kept].contiguous(), s[kept].contiguous(), info


def extra_repair(T=1 << 20, T_index=8192, peaks=None):
    """Repair of the 128^3 CSG pseudo-SDF (tau 3, Sec. 6): build on all
    samples; the samples whose spheres are exactly covered by the other balls
    (gfs_sphere_uncovered) are removed; rebuild on the rest; re-insert T
    removed samples with their own values known (their signs fix the classes,
    NONCONSERVATIVE counts values below them) by the greedy loop.  The paper
    assigns the repaired values in parallel and fixes no order; the
    sequential loop needs one: a seeded permutation of the removed samples
    (consecutive points far apart, so the rounds commit many steps), and for
    comparison the first T_index in index order (neighbours, mostly within
    each other's reach)."""
    import torch
    w, ctx, removed, p2, s2, info = _repair_setup()
    t_build = _ev_time(lambda: ctx.build(p2, s2), reps=1)
    res = {"workload": "csg128_tau3_repair_known_values", "samples": int(w.n), "removed": int(removed.size),
           "removal": info, "rebuild_ms": t_build}
    for name, sel in (("scattered", np.random.default_rng(3001).permutation(removed)[:T]),
                      ("index_order", removed[:T_index])):
        ctx.build(p2, s2)
        yt = torch.from_numpy(np.ascontiguousarray(w.p[sel])).cuda()
        kn = torch.from_numpy(np.ascontiguousarray(w.s[sel])).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = ctx.insert(yt, known=kn)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        st = ctx.stats()
        fl = out["flags"].cpu().numpy().astype(np.int32) & 0xFFFF
        res[name] = {"inserted": int(sel.size), "insert_s": dt, "insertions_per_s": sel.size / dt,
                     "rounds": st["insert_rounds"], "rebuilds": st["insert_rebuilds"],
                     "step_queries": st["insert_slots"], "ms_query": st["insert_ms_query"],
                     "ms_commit": st["insert_ms_commit"], "ms_update": st["insert_ms_update"],
                     "ms_rebuild": st["insert_ms_rebuild"], "roofline": _insert_roofline(st, peaks),
                     "codes": np.bincount(fl & 15, minlength=6).tolist(),
                     "nonconservative": int(np.sum((fl & 0x100) != 0)),
                     "lost_witness_steps": int(np.sum((fl & 0x80) != 0)),
                     "far_violations": int(np.sum((fl & 0x20) != 0)),
                     "survivors_after": st["n_survivors_pos"] + st["n_survivors_neg"]}
        del yt, kn, out
    ctx.close()
    return res


def extra_sphere16(peaks=None, reps=20):
    """The small workload: 16^3 grid of the exact SDF of a sphere (r 0.6), tau
    2 (663,552 candidates), FP64 queries at the 31^3 points of the 2x
    upsampled grid; build + query per step, inputs resident, median of reps."""
    import torch
    from paper_2605_01919_gb300 import gfs
    from paper_2605_01919_gb300 import workloads as W
    w = W.sphere_grid()
    x = torch.from_numpy(w.make_queries()).cuda()
    p, s = torch.from_numpy(w.p).cuda(), torch.from_numpy(w.s).cuda()
    m = int(x.shape[0])
    out = {"s": torch.empty(m, dtype=torch.float32, device="cuda"),
           "argmin": torch.empty(m, dtype=torch.int64, device="cuda"),
           "flags": torch.empty(m, dtype=torch.int16, device="cuda")}
    ctx = gfs.Context(tau=w.tau, timing=True)

    def step():
        ctx.build(p, s)
        ctx.query_into(x, out["s"], None, out["argmin"], out["flags"])
    for _ in range(3):
        step()
    ts, st = [], None
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        step()
        b.record()
        st = ctx.stats()
        ts.append(a.elapsed_time(b))
    ms = float(np.median(ts))
    ctx.close()
    return {"workload": "sphere16_tau2_q31^3_f64", "candidates": int(w.n) * 162, "queries": m, "ms_per_step": ms,
            "queries_per_s_incl_build": m / (ms / 1e3), "survivors": st["n_survivors_pos"] + st["n_survivors_neg"],
            "roofline": alu_roofline("k_query_spheres", st["query_sphere_items"], 8,
                                     "(query point, sphere) distance tests of the sphere pass", st["ms_query_spheres"],
                                     peaks, node_tests_per_launch=st["query_sphere_node_tests"])}


def extra_batch(count=256, scale=1.0, peaks=None):
    """The first `count` shapes of the 256-shape batch (unions of 1-8
    primitives; even index = grid with 2x upsampled queries, odd = scattered
    samples with 8n uniform queries), sizes scaled by `scale`: one batched
    build + persistent query launches vs. the same shapes one by one; the
    batched query is also replayed from a captured CUDA graph."""
    import torch
    from paper_2605_01919_gb300 import gfs
    from paper_2605_01919_gb300 import workloads as W
    shapes = []
    t_gen = time.perf_counter()
    for i in range(count):
        w = W.batch_shape(i, scale=scale)
        shapes.append({"p": torch.from_numpy(w.p).cuda(), "s": torch.from_numpy(w.s).cuda(),
                       "x": torch.from_numpy(w.make_queries()).cuda()})
    t_gen = time.perf_counter() - t_gen
    M = sum(int(sh["x"].shape[0]) for sh in shapes)
    Nn = sum(int(sh["p"].shape[0]) for sh in shapes)
    ctx = gfs.Context(tau=3)
    # the launches of the full batch take seconds each: one warm run, one timed
    ctx.batch_build(shapes)            # first build also autotunes the persistent grids
    t_build = _ev_time(lambda: ctx.batch_build(shapes), reps=1, warm=False)
    t_query = _ev_time(lambda: ctx.batch_query(), reps=1)
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            ctx.batch_query()
    torch.cuda.synchronize()
    t_graph = _ev_time(lambda: g.replay(), reps=1)
    bst = ctx.stats()
    # the whole batched path (rebuild from the samples + query) as one graph
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.stream(st):
        with torch.cuda.graph(g2, stream=st):
            ctx.batch_rebuild()
            ctx.batch_query()
    torch.cuda.synchronize()
    t_graph_full = _ev_time(lambda: g2.replay(), reps=1)
    status = ctx.batch_status()
    single = gfs.Context(tau=3)

    def one_by_one():
        for sh in shapes:
            single.build(sh["p"], sh["s"])
            single.query(sh["x"], want_f64=False)
    t_single = _ev_time(one_by_one, reps=1)
    ctx.close()
    single.close()
    return {"workload": f"batch{count}_scale{scale}_tau3", "shapes": count, "samples": Nn, "queries": M,
            "roofline": alu_roofline("k_batch_query (both phases)", bst["batch_sphere_items"] + bst["batch_surv_items"],
                                     8, "(query point, sphere or survivor) distance tests of the batched query",
                                     t_graph, peaks, node_tests_per_launch=bst["batch_sphere_node_tests"]),
            "batched_build_ms": t_build, "batched_query_ms": t_query, "graph_replay_query_ms": t_graph,
            "graph_replay_build_query_ms": t_graph_full,
            "graph_queries_per_s_incl_build": M / (t_graph_full / 1e3), "graph_status": status,
            "cull_tiles_by_size_class": bst["batch_cull_tile"], "query_grid": bst["batch_query_grid"],
            "batched_queries_per_s_incl_build": M / ((t_build + t_query) / 1e3),
            "one_by_one_ms": t_single, "one_by_one_queries_per_s_incl_build": M / (t_single / 1e3),
            "input_generation_s": t_gen}


def extra_tangent(every=256):
    """Same-sign tangent augmentation (Def. 1 tangent points as candidates,
    gfs_query_tangent) on the 64^3 union grid, tau 3, with its 253^3 points
    (every k-th): the plain query, and the query followed by the tangent pass;
    how many values a tangent point lowers."""
    import torch
    from paper_2605_01919_gb300 import gfs
    from paper_2605_01919_gb300 import workloads as W
    w = W.union_grid()
    x = torch.from_numpy(np.ascontiguousarray(w.make_queries()[::every])).cuda()
    m = int(x.shape[0])
    ctx = gfs.Context(tau=w.tau)
    ctx.build(torch.from_numpy(w.p).cuda(), torch.from_numpy(w.s).cuda())
    out = {"s": torch.empty(m, dtype=torch.float32, device="cuda"),
           "argmin": torch.empty(m, dtype=torch.int64, device="cuda"),
           "flags": torch.empty(m, dtype=torch.int16, device="cuda")}

    def plain():
        ctx.query_into(x, out["s"], None, out["argmin"], out["flags"])

    def both():
        plain()
        ctx.tangent_into(x, out["s"], None, out["argmin"], out["flags"])
    t_plain = _ev_time(plain, reps=2)
    t_both = _ev_time(both, reps=2)
    won = int(((out["flags"].to(torch.int32) & 15) == gfs.CODE_TANGENT).sum().item())
    ctx.close()
    return {"workload": f"union64_tau3_253^3_points_every{every}", "queries": m, "query_ms": t_plain,
            "query_plus_tangent_ms": t_both, "tangent_pass_ms": t_both - t_plain, "tangent_wins": won,
            "queries_per_s_with_tangent": m / (t_both / 1e3)}


def extra_scored(every=256):
    """Scored value (Sec. 3.3, gfs_query_scored) on the 64^3 union grid, tau
    3, at every k-th of its 253^3 points: the plain query, and the query
    followed by the scored pass; how the results split by code, and how many
    fall back to the minimum value."""
    import torch
    from paper_2605_01919_gb300 import gfs
    from paper_2605_01919_gb300 import workloads as W
    w = W.union_grid()
    x = torch.from_numpy(np.ascontiguousarray(w.make_queries()[::every])).cuda()
    m = int(x.shape[0])
    ctx = gfs.Context(tau=w.tau)
    ctx.build(torch.from_numpy(w.p).cuda(), torch.from_numpy(w.s).cuda())
    out = {"s": torch.empty(m, dtype=torch.float32, device="cuda"),
           "s64": torch.empty(m, dtype=torch.float64, device="cuda"),
           "argmin": torch.empty(m, dtype=torch.int64, device="cuda"),
           "flags": torch.empty(m, dtype=torch.int16, device="cuda")}

    def plain():
        ctx.query_into(x, out["s"], out["s64"], out["argmin"], out["flags"])

    def both():
        plain()
        ctx.scored_into(x, out["s"], out["s64"], out["argmin"], out["flags"])
    both()  # the per-sphere survivor lists are sorted on the first call
    t_plain = _ev_time(plain, reps=2)
    t_both = _ev_time(both, reps=2)
    fl = out["flags"].cpu().numpy().astype(np.int32) & 0xFFFF
    ctx.close()
    return {"workload": f"union64_tau3_253^3_points_every{every}", "queries": m, "query_ms": t_plain,
            "query_plus_scored_ms": t_both, "scored_pass_ms": t_both - t_plain,
            "queries_per_s_scored": m / (t_both / 1e3), "codes": np.bincount(fl & 15, minlength=7).tolist(),
            "fallbacks": int(np.sum((fl & 0x200) != 0))}


def extra_refine_order(N=64):
    """Sec. 4.2 refinement order on the N^3 union grid (tau 3; N = 64 is the
    headline workload's sample grid): the centres of
    the cells that may contain the surface are inserted greedily, once in
    flood-fill order (covered counts of 8^3 points per cell from
    gfs_cell_coverage, order from gfs_flood_order) and once in raster order;
    time of the coverage pass, insertions/s, and the mean absolute error of
    the inserted values against the union's field for both orders."""
    import torch
    from paper_2605_01919_gb300 import gfs
    from paper_2605_01919_gb300 import workloads as W
    w = W.union_grid(N=N, up=2)
    field = W.union_field()
    S = w.s.reshape(N, N, N)
    near = np.abs(S) < 0.5 * np.sqrt(3) * w.h
    cell = np.zeros((N - 1,) * 3, dtype=bool)
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                cell |= near[a:N - 1 + a, b:N - 1 + b, c:N - 1 + c]
    cells = np.argwhere(cell).astype(np.int32)
    centres = -1.0 + w.h * (cells.astype(np.float64) + 0.5)
    p, s = torch.from_numpy(w.p).cuda(), torch.from_numpy(w.s).cuda()
    ctx = gfs.Context(tau=w.tau)
    ctx.build(p, s)
    ct = torch.from_numpy(cells).cuda()
    t_cov = _ev_time(lambda: ctx.cell_coverage(ct, [-1.0, -1.0, -1.0], w.h, 8))
    counts = ctx.cell_coverage(ct, [-1.0, -1.0, -1.0], w.h, 8).cpu().numpy()
    t0 = time.perf_counter()
    flood = gfs.flood_order(cells, counts)
    t_order = time.perf_counter() - t0
    res = {"workload": f"union{N}_tau3_surface_cells", "cells": int(cells.shape[0]),
           "coverage_ms": t_cov, "flood_order_ms": 1e3 * t_order}
    for name, idx in (("flood", flood), ("raster", np.arange(cells.shape[0]))):
        y = np.ascontiguousarray(centres[idx])
        ctx.build(p, s)
        yt = torch.from_numpy(y).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = ctx.insert(yt)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        v = out["s64"].cpu().numpy()
        code = out["flags"].cpu().numpy().astype(np.int32) & 15
        ins = (code == gfs.CODE_SURVIVOR) | (code == gfs.CODE_OPPOSITE) | (code == gfs.CODE_LOWER)
        err = np.abs(v[ins] - field(y[ins]))
        res[name] = {"insertions_per_s": y.shape[0] / dt, "inserted": int(ins.sum()),
                     "mean_abs_err": float(err.mean()) if err.size else None,
                     "max_abs_err": float(err.max()) if err.size else None}
    ctx.close()
    return res


def extra_exact_coverage(csg_n=64, only_csg=False):
    """Exact coverage of each sample sphere (gfs_sphere_uncovered, Prop. 1
    (ii)): the 12^3 sphere grid (exact SDF samples: all keep an uncovered
    point), the 10^3 sphere grid with every value scaled by 1.2 (covered
    spheres), and the 64^3 CSG pseudo-SDF (most spheres covered, thousands of
    balls meeting a deep sphere); spheres per second and the split."""
    import torch
    from paper_2605_01919_gb300 import gfs
    from paper_2605_01919_gb300 import workloads as W
    res = {}
    cases = [] if only_csg else [("sphere12_exact_sdf", W.sphere_grid(N=12, up=2, tau=2), 1.0),
                                 ("sphere10_inflated_1.2", W.sphere_grid(N=10, up=2, tau=2), 1.2)]
    cases.append((f"csg{csg_n}_pseudo_sdf", W.csg_pseudo_grid(N=csg_n, tau=2), 1.0))
    for name, w, f in cases:
        s = np.ascontiguousarray(f * w.s)
        ctx = gfs.Context(tau=2)
        ctx.build(torch.from_numpy(w.p).cuda(), torch.from_numpy(s).cuda())
        t = _ev_time(lambda: ctx.sphere_uncovered(), reps=1)
        out = ctx.sphere_uncovered().cpu().numpy()
        surv = ctx.survivors().cpu().numpy()
        ctx.close()
        res[name] = {"spheres": int(w.n), "ms": t, "spheres_per_s": w.n / (t / 1e3),
                     "uncovered": int((out == 1).sum()), "covered": int((out == 0).sum()),
                     "undecided": int((out == 2).sum()),
                     "no_survivor_at_tau2": int(w.n - np.unique(surv // (10 * 4 ** 2 + 3)).size)}
        if name.startswith("csg"):
            # the U and D precomputation of Sec. 4.1 (includes its own
            # per-sphere test, the sort and the copies to the caller)
            ctx = gfs.Context(tau=2)
            ctx.build(torch.from_numpy(w.p).cuda(), torch.from_numpy(s).cuda())
            t0 = time.perf_counter()
            circ, quads, _, status = ctx.uncovered_intersections()
            torch.cuda.synchronize()
            res[name]["intersections"] = {"s": time.perf_counter() - t0, "circles": int(circ.shape[0]),
                                          "points": int(quads.shape[0]), "status": status}
            ctx.close()
    if only_csg:
        return res
    # the exact minimum valid radius over T, U, D (Sec. 6) against the
    # discrete value, on the 16^3 union grid at 1,024 of its upsampled points
    # (a moderate input: every point scans all uncovered points, circles
    # and spheres)
    w = W.union_grid(N=16, up=2, tau=3)
    ctx = gfs.Context(tau=w.tau)
    ctx.build(torch.from_numpy(w.p).cuda(), torch.from_numpy(w.s).cuda())
    xq = w.make_queries()
    x = torch.from_numpy(np.ascontiguousarray(xq[np.random.default_rng(5).choice(len(xq), 1024, replace=False)])).cuda()
    out = ctx.query(x)
    sig = torch.sign(out["s64"]).to(torch.int8)
    t0 = time.perf_counter()
    ctx.exact_rmin(x[:1], sig[:1])  # the state's U and D lists
    torch.cuda.synchronize()
    t_lists = time.perf_counter() - t0
    t = _ev_time(lambda: ctx.exact_rmin(x, sig), reps=1)
    rmin = ctx.exact_rmin(x, sig).cpu().numpy()
    v = np.abs(out["s64"].cpu().numpy())
    fl = out["flags"].cpu().numpy().astype(np.int32) & 15
    ok = np.isin(fl, [0, 1]) & np.isfinite(rmin)
    res["exact_rmin_union16"] = {"spheres": int(w.n), "points": int(x.shape[0]), "lists_s": t_lists, "ms": t,
                                 "points_per_s": x.shape[0] / (t / 1e3),
                                 "mean_discrete_minus_exact": float(np.mean(v[ok] - rmin[ok])),
                                 "max_discrete_minus_exact": float(np.max(v[ok] - rmin[ok]))}
    ctx.close()
    return res


def _finite(v):
    """The JSON line carries no NaN or infinity (strict parsers reject them):
    such values become null."""
    if isinstance(v, float):
        return v if np.isfinite(v) else None
    if isinstance(v, dict):
        return {k: _finite(u) for k, u in v.items()}
    if isinstance(v, (list, tuple)):
        return [_finite(u) for u in v]
    return v


def _isolated(only, extra=(), timeout=600):
    """Run one sub-benchmark in a child process, so that a failure there
    cannot end this process or its CUDA context; returns its JSON object."""
    import subprocess
    cmd = [sys.executable, os.path.abspath(__file__), "--only", only, *extra]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout)
    except subprocess.TimeoutExpired:
        return {"error": f"timed out after {timeout} s"}
    for line in reversed(r.stdout.splitlines()):
        if line.startswith("{"):
            return json.loads(line).get(only, {"error": "no result"})
    return {"error": f"exit {r.returncode}: {r.stderr[-400:]}"}


def run_gfs(args):
    import torch
    import torch.distributed as dist

    from paper_2605_01919_gb300 import gfs
    from paper_2605_01919_gb300 import workloads as W

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = W.union_grid()
    xh = np.ascontiguousarray(w.make_queries()[:: args.query_subsample])
    m, n = xh.shape[0], w.n
    p = torch.from_numpy(w.p).to(dev)
    s = torch.from_numpy(w.s).to(dev)
    x = torch.from_numpy(xh).to(dev)
    s_out = torch.empty(m, dtype=torch.float32, device=dev)
    arg_out = torch.empty(m, dtype=torch.int64, device=dev)
    fl_out = torch.empty(m, dtype=torch.int16, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ctx = gfs.Context(tau=w.tau, timing=True)

    def step():
        ctx.build(p, s)
        ctx.query_into(x, s_out, None, arg_out, fl_out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    phases = []
    launches0 = ctx.stats()
    stream = torch.cuda.current_stream()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)              # L2 flush between steps (outside the timed interval)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
        phases.append(ctx.stats())         # synchronises; phase times from events on the library stream
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop() if rank == 0 else None
    step_ms = [a.elapsed_time(b) for a, b in ev]
    launches1 = phases[-1]
    # own kernels, plus the radix-sort calls (each runs a handful of sort kernels)
    own_launches = launches1["kernel_launches"] - launches0["kernel_launches"]
    sort_calls = launches1["sort_calls"] - launches0["sort_calls"]
    value, ms_per_step = aggregate(float(sum(step_ms)), m, args.steps, world, device=dev)

    # ---- end to end through the host-buffer entry point ----------------------
    e2e = None
    if not args.no_e2e:
        # run the host side on the CPUs next to this GPU, so that the pinned
        # buffers are placed in that node's memory (the previous affinity is
        # restored afterwards)
        numa = gpu_numa_cpus(local)
        old_aff = os.sched_getaffinity(0)
        if numa:
            os.sched_setaffinity(0, numa[1] & old_aff or numa[1])
        ph = torch.from_numpy(w.p).pin_memory()
        sh = torch.from_numpy(w.s).pin_memory()
        xh_t = torch.from_numpy(xh).pin_memory()
        so = torch.empty(m, dtype=torch.float32).pin_memory()
        ao = torch.empty(m, dtype=torch.int64).pin_memory()
        fo = torch.empty(m, dtype=torch.int16).pin_memory()
        ctx_h = gfs.Context(tau=w.tau)
        ctx_h.solve_host(ph, sh, xh_t, so, ao, fo)   # warm-up
        torch.cuda.synchronize()
        e_times = []
        for k in range(max(1, min(args.steps, 3))):
            flush.fill_(k & 0xFF)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx_h.solve_host(ph, sh, xh_t, so, ao, fo)
            e_times.append(time.perf_counter() - t0)
        ctx_h.close()
        e_s = float(np.mean(e_times))
        os.sched_setaffinity(0, old_aff)
        e2e = {"value": world * m / e_s, "unit": UNIT, "h2d_bytes_per_step": n * 24 + n * 8 + m * 24,
               "d2h_bytes_per_step": m * (4 + 8 + 2), "ms_per_step": 1e3 * e_s,
               "host_numa_node": numa[0] if numa else None}

    # ---- roofline of the dominant kernel --------------------------------------
    # k_query_spheres, the first of the query's two FP32 kernels (the pass
    # over the spheres); its duration comes from the library's events around
    # it on the stream it is launched on
    last = phases[-1]
    q_sph = float(np.mean([ph_["ms_query_spheres"] for ph_ in phases]))
    q_fin = float(np.mean([ph_["ms_query_fast"] - ph_["ms_query_spheres"] for ph_ in phases]))
    q_exact = float(np.mean([ph_["ms_query_exact"] for ph_ in phases]))
    cull = float(np.mean([ph_["ms_build_cull"] for ph_ in phases]))
    build = float(np.mean([ph_["ms_build_total"] for ph_ in phases]))
    # the method's work in the sphere pass: one distance test per (query
    # point, sphere) pair it evaluates, 8 flops (3 differences, 3
    # multiply-adds); the hierarchy's child-node bound tests are the
    # implementation's pruning and are reported separately
    peaks = measure_alu_peaks(dev, local)
    items = last["query_sphere_items"]
    nodes = last["query_sphere_node_tests"]
    roofline = alu_roofline("k_query_spheres", items, 8, "(query point, sphere) distance tests of the sphere pass",
                            q_sph, peaks, traffic=recorded_traffic("k_query_spheres"),
                            node_tests_per_launch=nodes)
    roofline["frac_incl_node_tests"] = (8.0 * (items + nodes) / (q_sph / 1e3) / 1e12 / roofline["peak"]
                                        if roofline["peak"] else None)
    roofline["frac_of_nominal_peak"] = (roofline["achieved"] / peaks["fp32_tflops_nominal_max_clock"]
                                        if roofline["achieved"] else None)
    cull_roofline = alu_roofline("k_cull", last["cull_items"], 8,
                                 "(open candidate, sphere) coverage tests after the neighbour pre-test", cull,
                                 peaks, node_tests_per_launch=last["cull_node_tests"])

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": dict(CONFIG, queries=m, parallelism=f"replicas{world}", l2="256 MiB buffer written between steps "
                       "(outside the timed interval); queries (389 MB) exceed L2"),
        "roofline": roofline,
        "rooflines_other": {"cull": cull_roofline},
        "peaks": peaks,
        "phases_ms": {"build_total": build, "cull": cull, "query_spheres": q_sph, "query_finish": q_fin,
                      "query_exact": q_exact},
        "counters": {k: last[k] for k in ("n_survivors_pos", "n_survivors_neg", "cull_fp64_rechecks",
                                          "query_fp64_rechecks", "query_deferred", "query_sphere_node_tests",
                                          "query_sphere_items", "query_surv_node_tests", "query_surv_items",
                                          "query_band_passes", "tree_levels", "cull_node_tests", "cull_items")},
        "step_ms": step_ms,
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": own_launches,
        "gpu_launches_note": f"own kernels in the timed region; plus {sort_calls} radix-sort calls",
    }
    if rank == 0 and world == 1 and not args.no_extras:
        del p, s, x, s_out, arg_out, fl_out, flush
        torch.cuda.empty_cache()
        line["extras"] = {}
        for name, fn in (("sphere16", lambda: extra_sphere16(peaks)), ("backward", extra_backward),
                         ("repair", lambda: extra_repair(args.repair_steps, peaks=peaks)),
                         ("insert", lambda: extra_insert(args.insert_steps, peaks=peaks)),
                         ("batch", lambda: extra_batch(args.batch_shapes, args.batch_scale, peaks=peaks)),
                         ("tangent", lambda: _isolated("tangent", ["--tangent-every", str(args.tangent_every)],
                                                       timeout=150)),
                         ("refine_order", lambda: _isolated("refine_order", timeout=150)),
                         ("scored", lambda: _isolated("scored", ["--scored-every", str(args.scored_every)],
                                                      timeout=150)),
                         ("exact_coverage", lambda: _isolated("exact_coverage", timeout=300))):
            t_x = time.perf_counter()
            try:
                line["extras"][name] = fn()
            except Exception as e:  # a failing sub-benchmark must not hide the headline line
                line["extras"][name] = {"error": f"{type(e).__name__}: {e}"}
            line["extras"][name]["wall_s"] = time.perf_counter() - t_x
            torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_line(w, xh, steps=2, n_keep=2000, n_query=8)
    ctx.close()
    if rank == 0:
        print(json.dumps(_finite(line)), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    a = parse()
    if a.only:
        import torch
        pk = measure_alu_peaks(torch.device("cuda", 0), 0) if a.only in ("repair", "insert", "batch",
                                                                          "sphere16") else None
        fn = {"backward": extra_backward, "repair": lambda: extra_repair(a.repair_steps, peaks=pk),
              "insert": lambda: extra_insert(a.insert_steps, peaks=pk),
              "batch": lambda: extra_batch(a.batch_shapes, a.batch_scale, peaks=pk),
              "sphere16": lambda: extra_sphere16(pk),
              "scored": lambda: extra_scored(a.scored_every),
              "tangent": lambda: extra_tangent(a.tangent_every),
              "refine_order": extra_refine_order,
              "exact_coverage": lambda: extra_exact_coverage(a.exact_csg, a.exact_only_csg)}[a.only]
        print(json.dumps(_finite({a.only: fn()})), flush=True)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_gfs(a)
