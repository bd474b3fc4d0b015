"""Host logic of the benchmark on CPU: one replica per rank, the
job's time is the slowest rank's (all_reduce MAX over two gloo ranks), the
value is every rank's units over that time, and under torchrun only rank 0
runs the oracle arm while the other ranks leave without work, and that arm
prints the contract's line; the stored
ncu traffic figure is reported only for the kernel it was captured on."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["BENCH_ROOT"])
import torch.distributed as dist
import bench
dist.init_process_group("gloo", init_method="env://")
rank = dist.get_rank()
own = [3.0, 5.0][rank]           # this rank's timed region, seconds
t = bench.max_over_ranks(own, dist, "cpu")
v = bench.job_throughput(16 * 20, dist.get_world_size(), t)
print(json.dumps({"rank": rank, "t": t, "value": v}))
dist.barrier()
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_max_over_two_gloo_ranks():
    pytest.importorskip("torch")
    port = free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                   BENCH_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for o in outs:
        assert o["t"] == 5.0                          # the slowest rank's time on every rank
        assert o["value"] == pytest.approx(2 * 16 * 20 / 5.0)


def test_single_process_and_arithmetic():
    assert bench.max_over_ranks(2.5) == 2.5
    assert bench.job_throughput(320, 1, 0.5) == 640.0
    assert bench.job_throughput(320, 4, 2.0) == 640.0


def test_reference_arm_on_other_ranks_does_nothing(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    called = []
    monkeypatch.setattr(bench, "run_reference", lambda *a: called.append(a))
    bench.main()
    assert called == [] and capsys.readouterr().out == ""
    monkeypatch.setenv("RANK", "0")
    bench.main()
    assert len(called) == 1 and called[0][1] == 2     # rank 0 runs it, with the world size


def test_reference_arm_prints_the_contract_line(monkeypatch, capsys):
    """The oracle arm on a 10^3 cube (two steps): one JSON line with the
    metric of the benchmarked workload, its own cpu_baseline and an e2e that
    moves no bytes, in FP64 on the host cores."""
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3",
                                      "--n", "10"])
    bench.main()
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRICS["c3"]
    assert d["unit"] == "evals/s" and d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["value"] > 0
    assert abs(d["ms_per_step"] - 1e3 / d["value"]) < 1e-6 * d["ms_per_step"]
    assert d["config"]["n"] == 10 and d["config"]["n_v"] == 1000
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_stored_traffic_applies_only_to_its_kernel(tmp_path):
    """The ncu traffic figure is reported only for the kernel sources,
    batch size and mesh it was captured on."""
    rec = {"kernel": "k_fim", "kernel_hash": bench.kernel_hash(), "batch": 16, "n": 72,
           "bytes_per_launch": 123456789}
    f = tmp_path / "t.txt"
    f.write_text(json.dumps(rec))
    assert bench.stored_traffic(16, 72, str(f)) == 123456789
    assert bench.stored_traffic(8, 72, str(f)) is None
    assert bench.stored_traffic(16, 40, str(f)) is None
    f.write_text(json.dumps(dict(rec, kernel_hash="0" * 12)))
    assert bench.stored_traffic(16, 72, str(f)) is None
    f.write_text("not json")
    assert bench.stored_traffic(16, 72, str(f)) is None
    assert bench.stored_traffic(16, 72, str(tmp_path / "missing.txt")) is None
