"""The N > 1 path of bench.py runs independent replicas (the solver does not shard: one mesh
hierarchy per GPU, no collective on the data path).  Its host logic, the max over ranks of the
step time and the whole-job throughput, runs here on two gloo ranks on the CPU."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")

_RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, os.environ["BENCH_ROOT"])
import torch.distributed as dist
import bench
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:" + os.environ["PORT"], rank=rank, world_size=world)
local_ms = [41.0, 57.5][rank]
t = bench.max_over_ranks(local_ms, world)
dist.barrier()
dist.destroy_process_group()
print(json.dumps({"rank": rank, "max_ms": t, "value": bench.replica_throughput(t / 10, world, 3, 859812)}))
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return str(s.getsockname()[1])


def test_step_time_is_the_max_over_two_gloo_ranks():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", PORT=port, BENCH_ROOT=ROOT,
                   MASTER_ADDR="127.0.0.1", CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", _RANK_SCRIPT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["max_ms"] == 57.5
        # 2 replicas x 3 solves x 859,812 DoFs in 5.75 ms per step
        assert o["value"] == pytest.approx(2 * 3 * 859812 / 5.75e-3 / 1e6)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.replica_throughput(1000.0, 1, 1, 1_000_000) == pytest.approx(1.0)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    import bench
    called = []
    monkeypatch.setattr(bench, "run_oracle_subprocess", lambda *a, **k: called.append(a))
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup = 1, 0
    bench.run_reference(A())
    assert called == []


def test_clock_samples_inside_the_timed_region():
    """Only samples stamped within the timed region (widened by one 200 ms period) count; a
    throttle reason seen there is reported, one outside it is not."""
    import datetime
    import bench
    t0 = datetime.datetime(2026, 1, 1, 12, 0, 0)
    t1 = t0 + datetime.timedelta(seconds=1)

    def line(dt, mhz, thermal):
        ts = (t0 + datetime.timedelta(seconds=dt)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return f"{ts}, 0, {mhz}, 2070, 800.0, 0x0, Not Active, Not Active, {thermal}, Not Active"

    lines = [line(-2.0, 1500, "Active"), line(0.1, 2070, "Not Active"), line(0.5, 2050, "Not Active"),
             line(1.1, 2060, "Not Active"), line(3.0, 1400, "Active"), "garbage"]
    out = bench.parse_clock_samples(lines, t0, t1)
    assert out == {"sm_mhz": 2060.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}
    lines.insert(2, line(0.3, 2000, "Active"))
    assert bench.parse_clock_samples(lines, t0, t1)["reasons"] == ["sw_thermal_slowdown"]
    assert bench.parse_clock_samples([], t0, t1) is None
