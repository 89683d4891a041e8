"""The multi-replica path of bench.py (one process per GPU, no data-path
collective): whole-job throughput = units of all ranks / slowest rank's
time.  Exercised with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    total_ms = [1000.0, 1500.0][rank]          # rank 1 is the slower replica
    value, ms = bench.aggregate(total_ms, units_per_rank=300, steps=5, world=world)
    out[rank] = (value, ms)
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        value, ms = out[r]
        assert ms == pytest.approx(300.0)                 # 1500 ms / 5 steps: the slowest rank
        assert value == pytest.approx(2 * 300 / 0.3)      # both ranks' units / job time


def test_aggregate_single_process():
    import bench
    value, ms = bench.aggregate(500.0, units_per_rank=100, steps=5, world=1)
    assert ms == pytest.approx(100.0) and value == pytest.approx(1000.0)


def test_json_line_has_no_nonfinite_numbers():
    import json
    import bench
    line = bench._finite({"value": float("nan"), "extras": {"x": [1.0, float("inf")], "y": "ok"}, "n": 3})
    assert json.loads(json.dumps(line, allow_nan=False)) == {"value": None, "extras": {"x": [1.0, None], "y": "ok"},
                                                             "n": 3}


def test_traffic_record_only_for_current_kernel_sources(monkeypatch):
    """The roofline's DRAM traffic comes from the committed ncu summary only
    while the kernel sources still hash to the value recorded beside it."""
    import bench
    current = bench.recorded_traffic("k_query_spheres")
    monkeypatch.setattr(bench, "kernel_hash", lambda: "0000000000000000")
    assert bench.recorded_traffic("k_query_spheres") is None
    assert bench.recorded_traffic("no_such_kernel") is None
    assert current is None or current > 0
