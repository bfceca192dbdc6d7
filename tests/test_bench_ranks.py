"""The multi-rank path of bench.py (replicas, max-over-ranks timing) with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank              # rank 1 is the slowest
    m = bench.max_over_ranks(ms)
    out[rank] = (m, bench.replica_throughput(world, 1_000_000, m))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_replica_throughput_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    # two replicas of 1e6 points each, timed by the slower rank (15 ms)
    assert abs(res[0][1] - 2 * 1e6 / 15e-3 / 1e9) < 1e-12


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference: the timed CPU oracle, one JSON line with the base keys plus
    impl, cpu_baseline and e2e (zero copy bytes), on a bounded sample (seconds, not minutes)."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    assert line["e2e"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_cpu_baseline_uses_every_core_and_names_the_cpu():
    """The oracle's all-core timing: one spawned single-threaded process per core, throughput summed."""
    import bench
    cb = bench.cpu_baseline(seconds=0.3)
    assert cb["cores"] == (os.cpu_count() or 1)
    assert cb["kind"] == "oracle" and cb["unit"] == bench.UNIT
    assert cb["value"] > 0 and cb["single_thread_value"] > 0
    assert isinstance(cb["cpu"], str) and cb["cpu"]
