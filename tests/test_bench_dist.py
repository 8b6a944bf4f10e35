"""bench.py's multi-rank logic on CPU with the gloo backend, world size 2:
the step time is the max over ranks, the value counts every rank's bytes
(weak scaling), and the reference arm runs on rank 0 only."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        w, r, loc = bench.dist_env()
        local_ms = 2.0 + 3.0 * rank  # rank 1 is the slow one
        ms = bench.timed_max(local_ms, w)
        val = bench.weak_value(1e9, w, ms)
        q.put((r, w, loc, ms, val))
    finally:
        dist.destroy_process_group()


def _free_port():
    import socket

    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_max_over_ranks_and_weak_value():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for r, (rank, world, local, ms, val) in enumerate(got):
        assert (rank, world, local) == (r, 2, r)
        assert ms == 5.0  # the slow rank's time on both ranks
        assert val == pytest.approx(2 * 1e9 / 5e-3 / 1e9)


def test_reference_arm_rank_nonzero_exits_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0
    assert out.stdout.strip() == ""


def test_single_rank_helpers_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.timed_max(4.0, 1) == 4.0
    assert bench.weak_value(2e9, 1, 1.0) == pytest.approx(2000.0)
    json.dumps({"x": bench.weak_value(1.0, 1, 1.0)})


def test_reference_arm_json_line(monkeypatch, capsys):
    """The reference arm (the oracle timed on host cores) prints one JSON line
    with the keys of the bench contract: impl, metric, unit, value, the
    steps and warm-up asked for, its own cpu_baseline, and an e2e entry with
    no host-device copies.  Run on a small stand-in for the 512^3 field."""
    sys.path.insert(0, ROOT)
    import argparse

    import bench
    import synth

    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    shapes = list(synth.PAPER_SHAPES)
    shapes[1] = (20, 24, 32)
    monkeypatch.setattr(synth, "PAPER_SHAPES", tuple(shapes))
    args = argparse.Namespace(gpus=1, steps=2, warmup=3)
    assert bench.run_reference(args) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    assert (line["metric"], line["unit"]) == (bench.METRIC, bench.UNIT)
    assert (line["n_gpus"], line["steps"], line["warmup"]) == (1, 2, 3)
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert line["higher_is_better"] is True and line["vs_baseline"] is None
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"] == bench.WORKLOAD
