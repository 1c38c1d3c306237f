"""The benchmark's multi-rank reduction on CPU (gloo, world size 2).

A mesh does not shard, so N ranks run N independent replicas; the whole-job
value is N x faces / (slowest rank's time).  No GPU involved."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [40.0, 55.0][rank]                       # rank 1 is the slow one
        got = bench.max_over_ranks(ms, device="cpu")
        out[rank] = (got, bench.weak_value(1_310_720, world, got / 1))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_and_weak_value():
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        ms, v = out[r]
        assert ms == 55.0
        assert v == pytest.approx(2 * 1_310_720 / 0.055 / 1e6)


def test_single_process_identity():
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.weak_value(1e6, 1, 1000.0) == pytest.approx(1.0)


def _run_bench(args, env_extra=None):
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, **(env_extra or {}))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), *args], cwd=root,
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    return [json.loads(ln) for ln in lines]


def test_reference_arm_line_keeps_the_contract():
    """The reference arm (the CPU oracle, steps side by side in worker
    processes) prints one JSON line with the contract's keys; no GPU is needed
    for it.  Level 5 keeps the test short (the benchmark is level 8)."""
    (line,) = _run_bench(["--impl", "reference", "--steps", "2", "--warmup", "0",
                          "--level", "5"])
    assert line["impl"] == "reference" and line["unit"] == "Mfaces/s"
    for k in ("metric", "value", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["value"] > 0 and line["steps"] == 2 and line["higher_is_better"] is True
    assert line["config"]["workload"] == "bumped_icosphere_l5"
    assert line["config"]["faces_in"] == 20480 and line["config"]["target"] == 204
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert cb["nproc"] >= 1 and "cpu_model" in cb
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_print_nothing():
    assert _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0", "--level", "5"],
                      {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []
