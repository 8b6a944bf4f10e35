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
    """The reference arm (the oracle timed on every host core) prints one JSON line
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
    # every host core: one oracle process per core, each on its own slab
    assert cb["kind"] == "oracle" and cb["cores"] == min(os.cpu_count(), 20) and cb["value"] == line["value"]
    assert cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"] == bench.WORKLOAD


def test_clock_samples_summarized():
    """The clock record of the timed region: median and maximum SM clock and
    the throttle reasons that were active; lines that do not parse are
    skipped (nvidia-smi CSV, noheader, nounits)."""
    sys.path.insert(0, ROOT)
    import bench

    idle = "0, 2070, 2070, 812.35, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1965, 2070, 1398.10, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
    slow = "0, 1500, 2070, 1200.00, 0x0000000000000008, Active, Not Active, Not Active, Not Active"
    r = bench.summarize_clock_samples([idle, idle, capped, "garbage", "0, [N/A], 2070, 1, 0, a, b, c, d", idle])
    assert (r["sm_mhz"], r["sm_max_mhz"], r["reasons"], r["samples"]) == (2070.0, 2070.0, ["sw_power_cap"], 4)
    r = bench.summarize_clock_samples([slow, capped, idle])
    assert r["sm_mhz"] == 1965.0 and r["reasons"] == ["hw_slowdown", "sw_power_cap"]
    r = bench.summarize_clock_samples([])
    assert r["sm_mhz"] is None and r["sm_max_mhz"] is None and r["reasons"] == []


def test_profile_traffic_and_peaks(monkeypatch, tmp_path):
    """The roofline's inputs: the headline profile's DRAM traffic per element
    is used while the kernel sources hash as at its capture, and dropped
    (None) once they differ; the HBM peak is the measured one when
    MEASURED_PEAKS.json is present, else the fallback, and says which."""
    sys.path.insert(0, ROOT)
    import bench

    h = bench.csrc_hash()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "k_case.md").write_text("| DRAM traffic per launch (read + write, bytes) | 2000000 |\n"
                                    "elements per launch: 100000\ncsrc_sha256: " + h[:16] + "\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "csrc_hash", lambda: h)
    assert bench.read_profile_traffic("k_case") == 20.0
    monkeypatch.setattr(bench, "csrc_hash", lambda: "0" * 64)
    assert bench.read_profile_traffic("k_case") is None
    assert bench.read_profile_traffic("no_such_profile") is None
    assert bench.measured_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7012.5, "bf16_tflops": 1900}))
    assert bench.measured_peaks() == (7012.5, "measured")


def test_clock_sampler_keeps_the_timed_region():
    """ClockSampler.stop keeps the samples taken inside the marked region
    (with a stand-in for the nvidia-smi process) and summarizes those."""
    sys.path.insert(0, ROOT)
    import bench

    class _Proc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    class _Thread:
        def join(self, timeout=None):
            pass

    s = bench.ClockSampler(0)
    s.proc, s.thread = _Proc(), _Thread()
    row = "0, {}, 2070, 900.0, 0x0, Not Active, Not Active, {}, Not Active"
    s.lines = [(0.0, row.format(1000, "Active")),  # before the region
               (10.0, row.format(2070, "Not Active")), (10.5, row.format(2055, "Not Active")),
               (11.0, row.format(2070, "Not Active")),
               (99.0, row.format(900, "Active"))]  # after it
    s.t0, s.t1 = 9.9, 11.0
    r = s.stop()
    assert (r["sm_mhz"], r["sm_max_mhz"], r["reasons"], r["samples"]) == (2070.0, 2070.0, [], 3)
