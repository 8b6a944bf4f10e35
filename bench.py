"""Benchmark: homomorphic operations on compressed paper-like fields, GB300.

One step = every homomorphic operation of the hot path on every field of the
paper-like workload, each field resident in HBM in compressed form: the
derivative along every axis, the gradient magnitude, the Laplacian and the
exact mean / variance, for five float32 fields shaped like the paper's
datasets (k^-3 Gaussian random field + 5% spikes, value-range-relative
eb = 1e-3, block 32).  The step runs one pass per field (hc_op_multi: the
stream is decoded once and every operation is written from the same
neighbourhood, "decompress once, many ops").

value    = original bytes of one pass over the fields / step time (GB/s of
           original data, the paper's throughput definition) on the device
           with the compressed inputs already resident; value_op_weighted
           counts those bytes once per operation;
per_field = the one-pass kernel's rooflines field by field;
per_op_launches = the same operations as one fused kernel per operation
           (the paper's per-operation form: mean at stage 2, the rest at
           stage 3), with that form's own roofline and kernel shares;
per_op_cold = every per-operation kernel of every field cold (median of 30,
           L2 flushed before each run), with its roofline, the plain path and
           Table 4's decompress / operate split; field_512 singles out the
           512^3 field and its error-bound sweep (eb 1e-2, 1e-4);
configs  = the other configurations, time-bounded: HSZx, HSZp-nd / HSZp,
           HSZx-nd, the 64-field batched launch, the wide-code field and the
           serving saturation curve;
e2e      = the one-pass step through the C ABI from pinned host memory: the
           compressed streams are copied in and every output field and the
           statistics copied out inside the timed region;
plain    = full decompression to float32 followed by the same operations on
           the same GPU (the "generic flow"), once per field or once per
           operation, for the speedups;
roofline = the one-pass kernel's algorithmic bytes (compressed input +
           output fields) over its CUDA-event time, against the measured HBM
           copy bandwidth;
cpu_baseline = the oracle on every host core (one process per core, each on
           its own slab of the 512^3 field) and on one core.

Launch: python bench.py [--gpus N --steps K --warmup W] [--impl reference].
With torchrun (WORLD_SIZE > 1) every rank runs its own copy of the workload
on its own GPU (independent problems, weak scaling, no data-path collective);
the step time is the maximum over ranks.  Other modes print one
configuration alone: --batched, --serving, --hszx, --lorenzo, --boxes,
--wide; --no-extras skips the cold tables, the sweep and the configurations;
--profile-small / --profile-batch / --profile-lorenzo / --profile-boxes run
the small ncu cases.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "homomorphic-op GB/s of original data & speedup vs full decompress+op; %HBM peak"
UNIT = "GB/s"
EB = 1e-3
BLOCK = 32
WORKLOAD = ("paper-like scale: five float32 fields 100x500x500, 512x512x512, 256x384x384, 98x1200x1200, "
            "1800x3600 (2-D); seeded k^-3 Gaussian random fields + 5% spikes normalised to [0,1]; "
            "value-range-relative eb=1e-3; block 32; every homomorphic op (derivative per axis, gradient "
            "magnitude, Laplacian, exact mean and variance, all at stage 3) fused on the compressed stream, "
            "one pass per field")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(value: float, world: int) -> float:
    """Max of a per-rank float over the process group (identity when world == 1)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(bytes_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job GB/s: every rank processes bytes_per_rank in its step, the
    job's step time is the slowest rank's (ms_max)."""
    return bytes_per_rank * world / (ms_max * 1e-3) / 1e9


def timed_max(local_ms: float, world: int) -> float:
    """The step time the job reports: the max over ranks, after a barrier."""
    barrier(world)
    return reduce_max(local_ms, world)


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


# -------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle-reason samples (every 50 ms) around the
    timed region.  Started before the warm-up so that sampling is running when
    the timed region begins; mark() brackets the region and stop() keeps the
    samples that arrived inside it (or the one nearest to it when the region
    is shorter than the sampling period)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []  # (host time, line)
        self.t0 = self.t1 = None

    def start(self, wait_first: float = 3.0):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        t = time.monotonic()
        while not self.lines and time.monotonic() - t < wait_first:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def mark(self):
        if self.t0 is None:
            self.t0 = time.monotonic()
        else:
            self.t1 = time.monotonic()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        if self.t1 is None:
            self.mark()
        time.sleep(0.06)  # let the sample that covers the region's end arrive
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        t0 = self.t0 if self.t0 is not None else -1e30
        inside = [ln for t, ln in self.lines if t0 <= t <= self.t1 + 0.05]
        if not inside and self.lines:
            mid = (t0 + self.t1) / 2
            inside = [min(self.lines, key=lambda tl: abs(tl[0] - mid))[1]]
        return summarize_clock_samples(inside)


def summarize_clock_samples(lines) -> dict:
    """Median SM clock, maximum SM clock and the throttle reasons seen, from
    nvidia-smi CSV lines (ClockSampler.FIELDS, noheader, nounits); lines that
    do not parse are skipped."""
    sm, smax, reasons = [], [], set()
    names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
    for ln in lines:
        parts = [p.strip() for p in ln.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            smax.append(float(parts[2]))
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons), "samples": len(sm), "period_ms": 50}


def smi_index(local: int) -> str:
    """nvidia-smi -i argument for this rank's GPU (honours CUDA_VISIBLE_DEVICES)."""
    vis = [v.strip() for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    if local < len(vis):
        return vis[local]
    return str(local)


# ------------------------------------------------------------------ workload
def make_fields():
    import synth

    return [(shape, synth.grf_field(shape, 1000 + i)) for i, shape in enumerate(synth.PAPER_SHAPES)]


def op_list(ndim):
    return [("mean", None), ("variance", None)] + [("derivative", a) for a in range(ndim)] + \
        [("gradmag", None), ("laplacian", None)]


class Workload:
    """Compressed fields resident on the device plus preallocated outputs."""

    def __init__(self, hc, torch, dev, fields, eb=EB, S=BLOCK):
        self.hc, self.torch, self.dev = hc, torch, dev
        self.items = []
        for shape, x in fields:
            xd = torch.from_numpy(x).to(dev)
            c = hc.compress(xd, eb, rel=True, S=S)
            # keep only the stream bytes resident (the compressor's bound-sized buffer is freed)
            stream = c.stream[: c.nbytes].clone()
            c = hc.Compressed(stream, c.header, c.nbytes)
            del xd
            out = torch.empty(shape, dtype=torch.float32, device=dev)
            scal = torch.empty(hc.SCALAR_BYTES, dtype=torch.uint8, device=dev)
            self.items.append({"shape": shape, "c": c, "out": out, "scal": scal, "n": int(np.prod(shape))})
        torch.cuda.synchronize()

    @property
    def orig_bytes_per_step(self):
        return sum(it["n"] * 4 * len(op_list(len(it["shape"]))) for it in self.items)

    @property
    def launches_per_step(self):
        return sum(len(op_list(len(it["shape"]))) for it in self.items)

    def run_op(self, it, op, ax, src=None, level_q="q"):
        hc = self.hc
        inp = it["c"] if src is None else src
        if op == "mean":
            hc.mean(inp, level="p", out=it["scal"])
        elif op == "variance":
            hc.variance(inp, level=level_q, out=it["scal"])
        elif op == "derivative":
            hc.derivative(inp, ax, out=it["out"])
        elif op == "gradmag":
            hc.gradmag(inp, out=it["out"])
        else:
            hc.laplacian(inp, out=it["out"])

    def step(self, events=None):
        for fi, it in enumerate(self.items):
            for op, ax in op_list(len(it["shape"])):
                if events is not None:
                    e0 = self.torch.cuda.Event(enable_timing=True)
                    e0.record()
                self.run_op(it, op, ax)
                if events is not None:
                    e1 = self.torch.cuda.Event(enable_timing=True)
                    e1.record()
                    events.append((fi, op, e0, e1))


# timing protocol of the per-operation and plain forms: the L2 is flushed
# (a 512 MB write, four times the L2) before every timed run, and the median
# of REPS runs is kept
REPS = 30


def flush_l2(torch, dev, buf=[]):
    if not buf:
        buf.append(torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev))
    buf[0].fill_(1.0)


def time_call(torch, dev, fn, reps=REPS):
    """Median CUDA-event time (ms) of fn() with an L2 flush before each rep."""
    ts = []
    for _ in range(reps):
        flush_l2(torch, dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def op_specs(ndim):
    """Every per-operation kernel of a field: (label, operation, level or axis)."""
    specs = [("mean_stage2", "mean", "p"), ("mean_stage3", "mean", "q"),
             ("variance_stage2", "variance", "p"), ("variance_stage3", "variance", "q")]
    specs += [(f"derivative{a}", "derivative", a) for a in range(ndim)]
    return specs + [("gradmag", "gradmag", None), ("laplacian", "laplacian", None)]


def run_spec(hc, inp, kind, arg, out, scal):
    if kind == "mean":
        hc.mean(inp, level=arg or "p", out=scal)
    elif kind == "variance":
        hc.variance(inp, level=arg or "q", out=scal)
    elif kind == "derivative":
        hc.derivative(inp, arg, out=out)
    elif kind == "gradmag":
        hc.gradmag(inp, out=out)
    else:
        hc.laplacian(inp, out=out)


def cold_table(hc, torch, dev, c, shape, peak, plain=True, split=True):
    """Every operation of one compressed field on its own, cold (REPS runs,
    L2 flushed before each): the fused kernel's time, GB/s of original data
    and roofline fraction (compressed stream + output over the measured HBM
    peak); the plain path (decompress to float32, then the operation on the
    floats) and the speedup; and Table 4's split of the unfused stages:
    decompression to D_p / D_q / D_f and the operation on that array."""
    n = int(np.prod(shape))
    nd = len(shape)
    out = torch.empty(shape, dtype=torch.float32, device=dev)
    scal = torch.empty(hc.SCALAR_BYTES, dtype=torch.uint8, device=dev)
    arrs, t_dec = {}, {}
    if plain or split:
        for s in ("p", "q", "f"):
            arrs[s] = hc.decompress(c, s)
            t_dec[s] = time_call(torch, dev, lambda s=s: hc.decompress(c, s, out=arrs[s]))
        stages = {s: hc.as_stage(c, s, arrs[s]) for s in arrs}
    rows = {}
    for label, kind, arg in op_specs(nd):
        run_spec(hc, c, kind, arg, out, scal)
        ms = time_call(torch, dev, lambda: run_spec(hc, c, kind, arg, out, scal))
        field_op = kind in ("derivative", "gradmag", "laplacian")
        alg = c.nbytes + (4 * n if field_op else 64)
        r = {"ms": round(ms, 5), "gbs_orig": round(n * 4 / ms / 1e6, 1), "alg_bytes": alg,
             "roofline_frac": round(alg / (ms * 1e-3) / 1e9 / peak, 4)}
        aarg = arg if kind == "derivative" else None  # arrays: the axis only (no level)
        if plain:
            op_f = time_call(torch, dev, lambda: run_spec(hc, stages["f"], kind, aarg, out, scal))
            r["plain_ms"] = round(t_dec["f"] + op_f, 5)
            r["speedup_vs_plain"] = round((t_dec["f"] + op_f) / ms, 3)
            r["plain_split_ms"] = {"decompress_f": round(t_dec["f"], 5), "op_on_f": round(op_f, 5)}
        if split:
            st = arg if kind in ("mean", "variance") else "q"
            op_a = time_call(torch, dev, lambda: run_spec(hc, stages[st], kind, aarg, out, scal))
            r["unfused_split_ms"] = {"stage": st, "decompress": round(t_dec[st], 5), "op_on_array": round(op_a, 5),
                                     "total": round(t_dec[st] + op_a, 5)}
        rows[label] = r
    del arrs, out, scal
    res = {"field": "x".join(map(str, shape)), "compressed_bytes": c.nbytes, "wmax": int(c.header.wmax),
           "ops": rows}
    if t_dec:
        res["decompress_ms"] = {s: round(v, 5) for s, v in t_dec.items()}
    return res


def one_pass_cold(hc, torch, dev, c, shape, peak):
    """The one-pass kernel (every operation from one decode) cold on one field."""
    n = int(np.prod(shape))
    nd = len(shape)
    mo = {"derivative": [torch.empty(shape, dtype=torch.float32, device=dev) for _ in range(nd)],
          "gradmag": torch.empty(shape, dtype=torch.float32, device=dev),
          "laplacian": torch.empty(shape, dtype=torch.float32, device=dev),
          "stats": torch.empty(hc.SCALAR_BYTES, dtype=torch.uint8, device=dev)}
    hc.multi(c, outs=mo)
    ms = time_call(torch, dev, lambda: hc.multi(c, outs=mo))
    alg = c.nbytes + (nd + 2) * 4 * n + 64
    del mo
    return {"ms": round(ms, 5), "gbs_orig": round(n * 4 / ms / 1e6, 1), "alg_bytes": alg,
            "roofline_frac": round(alg / (ms * 1e-3) / 1e9 / peak, 4)}


def eb_sweep(hc, torch, dev, x, shape, peak, ebs=(1e-2, 1e-4)):
    """The 512^3 field at the other error bounds of the paper-like
    configuration: stream size and widths, the one-pass kernel and every
    per-operation kernel cold, against the plain path."""
    out = {}
    for eb in ebs:
        xd = torch.from_numpy(x).to(dev)
        c = hc._trim(hc.compress(xd, eb, rel=True, S=BLOCK))
        del xd
        row = cold_table(hc, torch, dev, c, shape, peak, plain=True, split=False)
        row["one_pass"] = one_pass_cold(hc, torch, dev, c, shape, peak)
        out[f"{eb:g}"] = row
        del c
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- roofline
def read_profile_traffic(kernel_tag: str):
    """DRAM bytes per element of the kernel's committed ncu capture
    (profiles/<kernel_tag>.md), if the CUDA sources are unchanged since the
    capture; else None."""
    path = os.path.join(ROOT, "profiles", kernel_tag + ".md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"DRAM traffic per launch \(read \+ write, bytes\) \| ([0-9.]+)", text)
    n = re.search(r"elements per launch: ([0-9]+)", text)
    h = re.search(r"csrc_sha256: ([0-9a-f]{16,64})", text)
    if not m or not n or not h or h.group(1) != csrc_hash()[: len(h.group(1))]:
        return None
    return float(m.group(1)) / float(n.group(1))


# device sources of the profiled kernels (the one-pass and single-operation
# stencils, their tile helpers, and the block-size-32 statistics): a
# profile's traffic is used only while these are unchanged since its capture
KERNEL_SOURCES = ("hc_stencil_pipe.cu", "hc_stencil_pipe.cuh", "hc_stencil_tile.cuh", "hc_internal.cuh",
                  "hc_finish.cuh", "hc_group.cuh", "hc_reduce32.cu")


def csrc_hash():
    d = hashlib.sha256()
    for fn in KERNEL_SOURCES:
        d.update(fn.encode())
        d.update(open(os.path.join(ROOT, "paper_2603_25206_gb300", "csrc", fn), "rb").read())
    return d.hexdigest()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        j = json.load(open(p))
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------- CPU baseline
def oracle_sample(sub):
    """Compress a sample with the oracle (outside any timed region)."""
    import oracle

    s, eps = oracle.compress(np.ascontiguousarray(sub), EB, True, BLOCK)
    return s, eps


def oracle_ops(s, eps, ndim):
    """The oracle, as it stands, on one compressed sample: decode to D_p and
    D_q and run every operation.  Returns (seconds, original bytes of the
    sample: one pass)."""
    import oracle

    t0 = time.perf_counter()
    dp = oracle.decode(s, "p")
    oracle.mean_p_sum(dp, BLOCK)
    q = oracle.decode(s, "q")
    s1, s2 = oracle.sums_q(q)
    oracle.finalize(q.size, s1, s2, eps)
    for ax in range(ndim):
        oracle.stencil_q(q, oracle.KIND_DERIV, eps, ax)
    oracle.stencil_q(q, oracle.KIND_GRADMAG, eps)
    oracle.stencil_q(q, oracle.KIND_LAPLACIAN, eps)
    dt = time.perf_counter() - t0
    return dt, q.size * 4


def cpu_sample_run(field, shape, planes):
    """The oracle on the first `planes` planes of a field (single thread)."""
    s, eps = oracle_sample(field[:planes])
    return oracle_ops(s, eps, len(shape))


def _oracle_worker(rank, sub, inbox, outbox):
    """One process of the all-cores oracle pool: compresses its slab once,
    then runs the oracle on it at every 'go' (spawned: no CUDA state)."""
    sys.path.insert(0, ROOT)
    s, eps = oracle_sample(sub)
    outbox.put(("ready", rank, 0.0, 0))
    while True:
        msg = inbox.get()
        if msg != "go":
            break
        dt, b = oracle_ops(s, eps, sub.ndim)
        outbox.put(("done", rank, dt, b))


class OraclePool:
    """The unmodified oracle on every host core: one spawned process per core,
    each on its own slab of planes of the field (the operations run on each
    slab as a field of its own; the slabs together cover the sample).  step()
    starts every process at once and returns (wall seconds until the last one
    finished, original bytes of the whole sample)."""

    def __init__(self, x, planes, nproc=None):
        import multiprocessing as mp

        self.nproc = nproc or os.cpu_count() or 1
        ctx = mp.get_context("spawn")
        per = max(1, planes // self.nproc)
        self.nproc = min(self.nproc, max(1, planes // per))
        self.planes = per * self.nproc
        self.inboxes = [ctx.Queue() for _ in range(self.nproc)]
        self.outbox = ctx.Queue()
        self.procs = []
        for r in range(self.nproc):
            sub = np.ascontiguousarray(x[r * per:(r + 1) * per])
            p = ctx.Process(target=_oracle_worker, args=(r, sub, self.inboxes[r], self.outbox), daemon=True)
            p.start()
            self.procs.append(p)
        for _ in range(self.nproc):
            self.outbox.get(timeout=600)

    def step(self):
        t0 = time.perf_counter()
        for q in self.inboxes:
            q.put("go")
        b = 0
        for _ in range(self.nproc):
            _, _, _, nb = self.outbox.get(timeout=600)
            b += nb
        return time.perf_counter() - t0, b

    def close(self):
        for q in self.inboxes:
            q.put("stop")
        for p in self.procs:
            p.join(timeout=30)


def cpu_baseline(fields, target_s=10.0):
    """The oracle timed on the host cores, on samples of the 512^3 field: one
    thread on its first planes (about target_s of work), and every core at
    once on the whole field (one slab per process; median of 3 passes)."""
    shape, x = fields[1]  # the 512^3 field
    planes = 8
    dt, b = cpu_sample_run(x, shape, planes)
    planes = int(max(8, min(shape[0], planes * target_s / max(dt, 1e-3))))
    dt, b = cpu_sample_run(x, shape, planes)
    single = {"value": b / dt / 1e9, "cores": 1,
              "sample": f"first {planes} planes of the 512x512x512 field ({planes * 512 * 512} elements), "
                        f"single thread, {dt:.1f} s"}
    pool = OraclePool(x, shape[0])
    try:
        runs = [pool.step() for _ in range(3)]
    finally:
        pool.close()
    wall = float(np.median([w for w, _ in runs]))
    ball = runs[0][1]
    return {"value": ball / wall / 1e9, "unit": UNIT, "cores": pool.nproc, "kind": "oracle",
            "sample": f"the whole 512x512x512 field split into {pool.nproc} slabs of {pool.planes // pool.nproc} "
                      f"planes, one oracle process per host core (spawned), each decoding its slab to D_p and "
                      f"D_q and running the mean, variance, 3 derivatives, gradient magnitude and Laplacian; "
                      f"median of 3 passes, {wall:.2f} s each; GB/s of original data (one pass)",
            "single_thread": single}


def _setup():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2603_25206_gb300 import hc

    return hc, torch, torch.device("cuda", torch.cuda.current_device())


def guarded(fn):
    """fn()'s result, or the error it raised: a failing extra measurement
    never takes the benchmark line down."""
    try:
        return fn()
    except Exception as e:  # noqa: BLE001
        import traceback

        return {"error": f"{type(e).__name__}: {e}", "where": traceback.format_exc().splitlines()[-4:]}


SERVING_QPS = (2000.0, 8000.0, 11000.0, 14000.0, 17000.0, 32000.0)
SERVING_P99_MS = 20.0


def run_extras(hc, torch, dev, fields, peak, args):
    """The other configurations of the paper-like benchmark, each bounded in
    time, as sub-objects of the benchmark line: the block-mean (HSZx), global
    predictor (HSZp-nd, HSZp) and box-mean (HSZx-nd) forms of the five fields,
    the 64-field batched launch, the wide-code float64 field, the serving
    loop's saturation curve and the small PR1 reference field."""
    out = {}
    jobs = (("hszx", lambda: measure_hszx(hc, torch, dev, fields)),
            ("lorenzo", lambda: measure_lorenzo(hc, torch, dev, fields)),
            ("boxes", lambda: measure_boxes(hc, torch, dev, fields)),
            ("batched", lambda: measure_batched(hc, torch, dev, steps=max(3, args.steps), warmup=3,
                                                device_fields=True, sample_clocks=False)),
            ("wide", lambda: measure_wide(hc, torch, dev, device_field=True)),
            ("pr1", lambda: measure_pr1(hc, torch, dev)),
            ("serving", lambda: measure_serving(hc, torch, dev, nfields=args.fields, qps_list=SERVING_QPS,
                                                duration=args.serving_duration, p99_ms=SERVING_P99_MS)))
    for name, fn in jobs:
        t = time.perf_counter()
        r = guarded(fn)
        r["wall_s"] = round(time.perf_counter() - t, 1)
        out[name] = r
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    return out


# -------------------------------------------------------------------- arms
def run_reference(args):
    """The oracle as the reference arm: K timed steps, each the oracle on
    every host core at once over a bounded sample of the 512^3 field (one
    slab per process)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import synth

    shape = synth.PAPER_SHAPES[1]
    x = synth.grf_field(shape, 1001)
    nproc = os.cpu_count() or 1
    pool = OraclePool(x, min(shape[0], 16 * nproc), nproc)
    try:
        for _ in range(args.warmup):
            pool.step()
        tot_t, tot_b = 0.0, 0
        for _ in range(args.steps):
            dt, b = pool.step()
            tot_t += dt
            tot_b += b
    finally:
        pool.close()
    value = tot_b / tot_t / 1e9
    sample = (f"the first {pool.planes} planes of the 512x512x512 field per step, {pool.nproc} oracle processes "
              f"(one per host core) on {pool.planes // pool.nproc} planes each")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_t / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.nproc, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", torch.cuda.current_device())
    import __graft_entry__

    __graft_entry__.build()
    from paper_2603_25206_gb300 import hc

    hc.lib()
    fields = make_fields()
    wl = Workload(hc, torch, dev, fields)
    # original bytes of one pass over every field (the metric's unit of work);
    # the operation-weighted figure (x the operations per field) is reported
    # under its own key
    bytes_pass = sum(it["n"] * 4 for it in wl.items)
    bytes_step = wl.orig_bytes_per_step
    comp_bytes = sum(it["c"].nbytes for it in wl.items)
    # the library's autotuner picks the fused stencil's tile height per field and op
    tiles = {}
    for it in wl.items:
        for op in ("derivative", "gradmag", "laplacian", "multi"):
            tiles["x".join(map(str, it["shape"])) + ":" + op] = hc.autotune(
                it["c"], op, "float32", out=None if op == "multi" else it["out"])

    peak, peak_src = measured_peaks()
    # outputs of the one-pass step: every derivative, the gradient magnitude,
    # the Laplacian and the statistics of each field
    mouts = []
    for it in wl.items:
        nd = len(it["shape"])
        mouts.append({"derivative": [torch.empty(it["shape"], dtype=torch.float32, device=dev) for _ in range(nd)],
                      "gradmag": torch.empty(it["shape"], dtype=torch.float32, device=dev),
                      "laplacian": it["out"], "stats": it["scal"]})

    def one_pass_step(evs=None, items=None):
        for fi, it in enumerate(wl.items):
            if evs is not None:
                e0 = torch.cuda.Event(enable_timing=True)
                e0.record()
            hc.multi(it["c"] if items is None else items[fi], outs=mouts[fi])
            if evs is not None:
                e1 = torch.cuda.Event(enable_timing=True)
                e1.record()
                evs.append((fi, e0, e1))

    sampler = ClockSampler(smi_index(local))
    sampler.start()
    for _ in range(args.warmup):
        one_pass_step()
    torch.cuda.synchronize()

    # ---- headline, device-resident: one pass per field computes every
    # operation from one decode (hc_op_multi)
    barrier(world)
    torch.cuda.synchronize()
    sampler.mark()
    mev = []
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(args.steps):
        one_pass_step(mev)
    t1.record()
    torch.cuda.synchronize()
    sampler.mark()
    barrier(world)
    clocks = sampler.stop()
    ms = reduce_max(t0.elapsed_time(t1) / args.steps, world)
    value = weak_value(bytes_pass, world, ms)
    value_op_weighted = weak_value(bytes_step, world, ms)
    m_ms = sum(x.elapsed_time(y) for _, x, y in mev)
    m_bytes = sum(wl.items[fi]["c"].nbytes + (len(wl.items[fi]["shape"]) + 2) * 4 * wl.items[fi]["n"] + 64
                  for fi, _, _ in mev)
    achieved = m_bytes / (m_ms * 1e-3) / 1e9
    per_elem = read_profile_traffic("stencil_multi_256x384x384")
    m_elems = sum(wl.items[fi]["n"] for fi, _, _ in mev) / max(1, len(mev))
    per_field = {}
    for fi, x, y in mev:
        it = wl.items[fi]
        d = per_field.setdefault("x".join(map(str, it["shape"])), {"ms": 0.0, "launches": 0, "n": it["n"],
                                                                    "alg": it["c"].nbytes + (len(it["shape"]) + 2) * 4 * it["n"] + 64})
        d["ms"] += x.elapsed_time(y)
        d["launches"] += 1
    for k, d in per_field.items():
        a = d["ms"] / d["launches"]
        per_field[k] = {"kernel": "k_stencil_multi", "avg_launch_ms": round(a, 5),
                        "gbs_orig": round(d["n"] * 4 / a / 1e6, 1), "algorithmic_bytes_per_launch": d["alg"],
                        "achieved_gbs": round(d["alg"] / (a * 1e-3) / 1e9, 1),
                        "roofline_frac": round(d["alg"] / (a * 1e-3) / 1e9 / peak, 4)}
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": per_elem * m_elems if per_elem is not None else None,
                "kernel": "k_stencil_multi", "peak_source": peak_src,
                "algorithmic_bytes_per_launch": m_bytes / len(mev), "avg_launch_ms": m_ms / len(mev),
                "algorithmic_bytes": "compressed stream + (ndim + 2) float32 output fields + 64 B of statistics"}

    # ---- the same operations as one fused kernel per operation (the paper's
    # per-operation form), device-resident
    for _ in range(args.warmup):
        wl.step()
    torch.cuda.synchronize()
    barrier(world)
    events = []
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        wl.step(events)
    b.record()
    torch.cuda.synchronize()
    op_ms = reduce_max(a.elapsed_time(b) / args.steps, world)
    per = {}
    for fi, op, x, y in events:
        d = per.setdefault(op, {"ms": 0.0, "bytes": 0.0, "launches": 0})
        it = wl.items[fi]
        d["ms"] += x.elapsed_time(y)
        d["bytes"] += it["c"].nbytes + (it["n"] * 4 if op in ("derivative", "gradmag", "laplacian") else 64)
        d["launches"] += 1
    dom = max(per, key=lambda k: per[k]["ms"])
    op_ach = per[dom]["bytes"] / (per[dom]["ms"] * 1e-3) / 1e9
    # DRAM traffic: the dominant kernel's bytes per element from its committed
    # ncu capture on the 256x384x384 case, scaled to this launch's elements
    tag = {"derivative": "stencil_pipe_derivative_256x384x384", "gradmag": "stencil_pipe_gradmag_256x384x384",
           "laplacian": "stencil_pipe_laplacian_256x384x384",
           "variance": "reduce32_variance_256x384x384", "mean": "reduce32_mean_stage2_256x384x384"}.get(dom, "")
    op_pe = read_profile_traffic(tag) if tag else None
    elems = sum(wl.items[fi]["n"] for fi, op, _, _ in events if op == dom) / max(1, per[dom]["launches"])
    per_op_launches = {
        "what": "one fused kernel per operation (mean at stage 2, the rest at stage 3), 35 launches per step",
        "ms_per_step": op_ms, "value": weak_value(bytes_pass, world, op_ms),
        "value_op_weighted": weak_value(bytes_step, world, op_ms),
        "one_pass_speedup": op_ms / ms,
        "roofline": {"bound": "hbm", "achieved": op_ach, "peak": peak, "unit": "GB/s", "frac": op_ach / peak,
                     "traffic": op_pe * elems if op_pe is not None else None, "kernel": dom,
                     "algorithmic_bytes_per_launch": per[dom]["bytes"] / per[dom]["launches"],
                     "avg_launch_ms": per[dom]["ms"] / per[dom]["launches"]},
        "kernel_time_share": {k: v["ms"] / sum(x["ms"] for x in per.values()) for k, v in per.items()}}

    # ---- plain path: every op on a full decompression to float32 (the
    # paper's "decompress, then operate" per operation), and, for reference,
    # one decompression per field shared by all its ops
    plain_ms = plain_once_ms = None
    if not args.skip_plain:
        df = {fi: torch.empty(it["shape"], dtype=torch.float32, device=dev) for fi, it in enumerate(wl.items)}

        def plain_step(once):
            for fi, it in enumerate(wl.items):
                st = hc.as_stage(it["c"], "f", df[fi])
                if once:
                    hc.decompress(it["c"], "f", out=df[fi])
                for op, ax in op_list(len(it["shape"])):
                    if not once:
                        hc.decompress(it["c"], "f", out=df[fi])
                    wl.run_op(it, op, ax, src=st)

        def timed(fn):
            for _ in range(max(1, args.warmup)):
                fn()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(args.steps):
                fn()
            b.record()
            torch.cuda.synchronize()
            return reduce_max(a.elapsed_time(b) / args.steps, world)

        plain_ms = timed(lambda: plain_step(False))
        plain_once_ms = timed(lambda: plain_step(True))
        del df

    # ---- end to end through the ABI from pinned host memory: every step
    # copies the compressed streams in, runs the one-pass step and copies
    # every output field and the statistics out
    host_streams = [it["c"].stream.cpu().pin_memory() for it in wl.items]
    dev_streams = [torch.empty_like(it["c"].stream) for it in wl.items]
    e2e_items = [hc.Compressed(ds, it["c"].header, it["c"].nbytes) for ds, it in zip(dev_streams, wl.items)]
    host_out = [[torch.empty(it["shape"], dtype=torch.float32).pin_memory() for _ in range(len(it["shape"]) + 2)]
                for it in wl.items]
    host_scal = [torch.empty(hc.SCALAR_BYTES, dtype=torch.uint8).pin_memory() for _ in wl.items]
    d2h = 0

    # outputs go back on four copy streams: a field's copies overlap the next
    # field's kernel and can use several copy engines
    copy_streams = [torch.cuda.Stream(device=dev) for _ in range(4)]

    def e2e_step():
        nonlocal d2h
        d2h = 0
        main = torch.cuda.current_stream(dev)
        for fi, it in enumerate(wl.items):
            dev_streams[fi].copy_(host_streams[fi], non_blocking=True)
        k = 0
        for fi, it in enumerate(wl.items):
            hc.multi(e2e_items[fi], outs=mouts[fi])
            done = torch.cuda.Event()
            done.record(main)
            mo = mouts[fi]
            pairs = list(zip(host_out[fi], mo["derivative"] + [mo["gradmag"], mo["laplacian"]]))
            pairs.append((host_scal[fi], mo["stats"]))
            for dst, src in pairs:
                cs = copy_streams[k % len(copy_streams)]
                k += 1
                cs.wait_event(done)
                with torch.cuda.stream(cs):
                    dst.copy_(src, non_blocking=True)
                d2h += src.numel() * src.element_size()
        for cs in copy_streams:
            main.wait_stream(cs)

    # the same step with the one-pass kernel writing every output field and
    # statistic straight into the pinned host buffers (host memory is mapped
    # into the device's address space), so no copy engine pass is needed
    host_mouts = []
    for fi, it in enumerate(wl.items):
        nd = len(it["shape"])
        host_mouts.append({"derivative": host_out[fi][:nd], "gradmag": host_out[fi][nd],
                           "laplacian": host_out[fi][nd + 1], "stats": host_scal[fi]})

    def e2e_direct_step():
        for fi, it in enumerate(wl.items):
            dev_streams[fi].copy_(host_streams[fi], non_blocking=True)
        for fi, it in enumerate(wl.items):
            hc.multi(e2e_items[fi], outs=host_mouts[fi])

    def time_e2e(fn):
        for _ in range(max(1, args.warmup)):
            fn()
        torch.cuda.synchronize()
        barrier(world)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.steps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return reduce_max(a.elapsed_time(b) / args.steps, world)

    copy_ms = time_e2e(e2e_step)
    copied = [[h.clone() for h in hs] for hs in host_out]
    try:
        direct_ms = time_e2e(e2e_direct_step)
        # both ways must deliver the same bytes to the host
        same = all(torch.equal(a_, b_) for hs_a, hs_b in zip(copied, host_out) for a_, b_ in zip(hs_a, hs_b))
    except hc.HcError:  # a host buffer the library does not accept (alignment): copies only
        direct_ms, same = None, False
    del copied
    e2e_ms = min(copy_ms, direct_ms) if same else copy_ms
    direct_won = same and direct_ms < copy_ms
    e2e = {"value": weak_value(bytes_pass, world, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": comp_bytes,
           "value_op_weighted": weak_value(bytes_step, world, e2e_ms),
           "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
           "mode": "kernel writes to pinned host memory" if direct_won
           else "device outputs copied back on four copy streams",
           "copy_engines_ms_per_step": copy_ms, "direct_host_write_ms_per_step": direct_ms,
           "direct_equals_copied": same}

    # per-operation kernels cold (REPS runs, L2 flushed before each) on every
    # field, with the plain path and Table 4's decompress / operate split;
    # the 512^3 field at the other error bounds; the other configurations
    cold = sweep = extras = None
    if rank == 0 and world == 1 and args.extras:
        cold = []
        for it in wl.items:
            def field_rows(it=it):
                row = cold_table(hc, torch, dev, it["c"], it["shape"], peak, plain=not args.skip_plain, split=True)
                row["one_pass"] = one_pass_cold(hc, torch, dev, it["c"], it["shape"], peak)
                return row
            cold.append(guarded(field_rows))
        sweep = guarded(lambda: eb_sweep(hc, torch, dev, fields[1][1], fields[1][0], peak))
        extras = run_extras(hc, torch, dev, fields, peak, args)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "value_op_weighted": value_op_weighted,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "fields": ["x".join(map(str, it["shape"])) for it in wl.items],
                           "eb_rel": EB, "block": BLOCK, "compressed_bytes": comp_bytes,
                           "original_bytes_per_pass": bytes_pass,
                           "value": "original bytes of one pass over the five fields / step time (each pass "
                                    "computes every operation of every field); value_op_weighted counts "
                                    "those bytes once per operation",
                           "l2": "no flush: every step streams 5 compressed fields and writes ~6.9 GB of output "
                                 "fields, far larger than the 129 MB L2",
                           "parallelism": f"replicas x{world} (independent fields per GPU)",
                           "autotuned_tile_rows": tiles},
                "step": "one pass per field: hc_op_multi decodes the stream once and writes the derivative "
                        "along every axis, the gradient magnitude, the Laplacian and the exact stage-3 "
                        "mean / variance (5 launches per step)",
                "plain": None if plain_ms is None else {
                    "what": "decompress to float32 on the GPU, then the same operations on the floats",
                    "decompress_once_ms_per_step": plain_once_ms,
                    "decompress_once_value": weak_value(bytes_pass, world, plain_once_ms),
                    "speedup_vs_decompress_once": plain_once_ms / ms,
                    "decompress_per_op_ms_per_step": plain_ms,
                    "decompress_per_op_value": weak_value(bytes_pass, world, plain_ms),
                    "speedup_vs_decompress_per_op": plain_ms / ms},
                "per_op_launches": per_op_launches,
                "e2e": e2e, "gpu_launches": len(wl.items) * args.steps,
                "roofline": roofline, "clocks": clocks}
        if args.cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(fields)
        line["per_field"] = per_field
        if cold is not None:
            line["per_op_cold"] = {"timing": f"median of {REPS} CUDA-event runs per kernel, a 512 MB write "
                                             "(4x L2) before each", "eb_rel": EB, "fields": cold}
            f512 = next((r for r in cold if r.get("field") == "512x512x512"), None)
            if f512 is not None:
                line["field_512"] = {"one_pass": f512["one_pass"],
                                     "ops": {k: {"roofline_frac": v["roofline_frac"], "ms": v["ms"],
                                                 "speedup_vs_plain": v.get("speedup_vs_plain")}
                                             for k, v in f512["ops"].items()},
                                     "eb_sweep": sweep}
        if extras is not None:
            line["configs"] = extras
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def measure_batched(hc, torch, dev, steps, warmup, device_fields=False, sample_clocks=True):
    """The batched form: 64 float32 fields of uneven sizes (every axis drawn
    log-uniformly from [32, 384], seed 3; k^-3 field + 5% spikes), value-range-
    relative eb = 1e-3.  Mean, variance and Laplacian of every field in ONE
    persistent fused launch replayed from a CUDA graph, with the block size S
    and threads per CTA picked by the library's autotuner.  value = original
    bytes of all fields / step time (each field is read once for its three
    operations).  Compared on the same GPU with the same streams: the three
    one-field fused calls per field (192 launches), and the plain path
    (decompress each field to float32, then the three operations)."""
    import synth

    shapes = synth.log_uniform_shapes(64, 32, 384, 3)
    if device_fields:  # the same recipe drawn on the device (fast; different numbers)
        raw = [synth.grf_field_device(sh, 3000 + j, dev) for j, sh in enumerate(shapes)]
    else:
        raw = [torch.from_numpy(synth.grf_field(sh, 3000 + j)).to(dev) for j, sh in enumerate(shapes)]
    n_total = sum(int(x.numel()) for x in raw)
    flush = lambda: flush_l2(torch, dev)  # noqa: E731
    best, table = hc.batch_autotune(raw, EB, True, "mean|variance|laplacian", flush=flush)
    del raw
    b, comps = best["batch"], best["comps"]
    comp_bytes = sum(c.nbytes for c in comps)
    sampler = ClockSampler(smi_index(0)) if sample_clocks else None
    if sampler:
        sampler.start()
    for _ in range(warmup):
        b.replay()
    torch.cuda.synchronize()
    if sampler:
        sampler.mark()
    ev = []
    for _ in range(steps):
        flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        b.replay()
        e1.record()
        ev.append((e0, e1))
    torch.cuda.synchronize()
    clocks = None
    if sampler:
        sampler.mark()
        clocks = sampler.stop()
    ms = sum(a.elapsed_time(z) for a, z in ev) / steps
    assert b.status() == 0
    value = n_total * 4 / (ms * 1e-3) / 1e9

    # the same work as one-field calls, and the plain path
    outs = [torch.empty(c.shape, dtype=torch.float32, device=dev) for c in comps]
    scal = torch.empty(hc.SCALAR_BYTES, dtype=torch.uint8, device=dev)

    def separate():
        for c, o in zip(comps, outs):
            hc.mean(c, level="q", out=scal)
            hc.variance(c, level="q", out=scal)
            hc.laplacian(c, out=o)

    def plain():
        for c, o in zip(comps, outs):
            f = hc.decompress(c, "f", out=o)
            sf = hc.as_stage(c, "f", f)
            hc.mean(sf, out=scal)
            hc.variance(sf, out=scal)
            hc.laplacian(sf, out=o)

    separate()
    plain()
    t_sep = time_call(torch, dev, separate)
    t_plain = time_call(torch, dev, plain)
    peak, peak_src = measured_peaks()
    alg = comp_bytes + n_total * 4 + 64 * len(comps)
    achieved = alg / (ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": 1, "steps": steps,
        "warmup": warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": "batched: 64 float32 fields, every axis log-uniform in [32, 384] (seed 3), k^-3 "
                               "GRF + 5% spikes, value-range-relative eb=1e-3; mean + variance + Laplacian per "
                               "field in one persistent fused launch under a CUDA graph; S and threads autotuned",
                   "elements": n_total, "compressed_bytes": comp_bytes, "S": best["S"],
                   "threads": best["threads"], "ty": best["ty"], "grid": b.grid,
                   "l2": "flushed between timed iterations",
                   "fields_drawn_on": "device" if device_fields else "host"},
        "gpu_launches": steps,
        "autotune": table,
        "one_field_calls_ms": round(t_sep, 4), "speedup_vs_one_field_calls": round(t_sep / ms, 3),
        "plain_ms": round(t_plain, 4), "speedup_vs_plain": round(t_plain / ms, 3),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": None,
                     "peak_source": peak_src,
                     "algorithmic_bytes": "compressed streams + float32 Laplacian outputs + 64 B per field"},
        "clocks": clocks,
    }
    b.close()
    return line


def run_batched(args):
    hc, torch, dev = _setup()
    print(json.dumps(measure_batched(hc, torch, dev, args.steps, args.warmup)))
    return 0


def serving_fields(hc, torch, dev, nfields):
    """The serving set: nfields compressed float32 fields resident on the
    device (cube side log-uniform in [64, 512], k^-3 Gaussian random fields
    drawn on the device, eb uniform over {1e-2, 1e-3, 1e-4} value-range-
    relative, block 32)."""
    import synth

    rng = np.random.default_rng(4)
    fields, fbytes = [], {}
    for j in range(nfields):
        side = int(round(math.exp(rng.uniform(math.log(64), math.log(512)))))
        eb = float(rng.choice([1e-2, 1e-3, 1e-4]))
        x = synth.grf_field_device((side, side, side), 5000 + j, dev, spikes=0.0)
        fields.append(hc._trim(hc.compress(x, eb, rel=True, S=BLOCK)))
        fbytes[j] = x.numel() * 4
        del x
    torch.cuda.synchronize()
    return fields, fbytes


def serve_once(hc, torch, fields, fbytes, qps, duration, plain):
    """One seeded Poisson stream served to the end: p50 / p99 latency and
    throughput (120 GB admission budget, 4 stream slots, <= 64 queries per step)."""
    from paper_2603_25206_gb300 import serving

    budget = 120 * 10**9
    qs = serving.poisson_queries(len(fields), qps, duration, 4, plain=plain)
    # warm-up on a short prefix (kernels, allocator, plans)
    serving.run(hc, fields, qs[:64], budget, slots=4, max_batch=64)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    recs, sch = serving.run(hc, fields, qs, budget, slots=4, max_batch=64)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    summ = serving.summarize(recs, qs, fbytes, wall=wall)
    summ["offered_qps"] = qps
    summ["offered"] = len(qs)
    summ["refused"] = len(sch.refused)
    summ["peak_reserved_gb"] = round(sch.peak_bytes / 1e9, 3)
    return {k: (round(v, 4) if isinstance(v, float) else v) for k, v in summ.items()}


def measure_serving(hc, torch, dev, nfields, qps_list, duration, p99_ms=SERVING_P99_MS):
    """The serving form: a seeded Poisson stream of mean / variance /
    gradient-magnitude queries at random stages on the resident serving set,
    served by the homomorphic path and by the plain path (every query
    decompresses to float32 first), at each offered rate of qps_list.  The
    saturation point of a path is the highest offered rate it serves with
    p99 <= p99_ms and a completed rate of at least 95% of the offered one."""
    t_gen = time.perf_counter()
    fields, fbytes = serving_fields(hc, torch, dev, nfields)
    t_gen = time.perf_counter() - t_gen
    out = {"metric": "serving: query latency p50/p99 and throughput, homomorphic vs plain, per offered rate",
           "config": {"workload": f"serving: {nfields} float32 fields, cube side log-uniform 64..512, k^-3 "
                                  f"GRF, eb in {{1e-2,1e-3,1e-4}} (REL), block 32; Poisson queries (seed 4) of "
                                  f"mean/variance/gradmag at random stages for {duration:g} s per rate; 120 GB "
                                  f"admission budget, 4 slots, <= 64 queries per step",
                      "raw_bytes": sum(fbytes.values()), "compressed_bytes": sum(c.nbytes for c in fields),
                      "setup_s": round(t_gen, 1), "p99_bound_ms": p99_ms},
           "data": "synthetic", "rates": {}}
    sat = {"homomorphic": 0.0, "plain": 0.0}
    for qps in qps_list:
        row = {}
        for name, plain in (("homomorphic", False), ("plain", True)):
            r = serve_once(hc, torch, fields, fbytes, qps, duration, plain)
            row[name] = r
            if r.get("p99_ms", 1e9) <= p99_ms and r.get("qps", 0.0) >= 0.95 * qps:
                sat[name] = max(sat[name], qps)
        out["rates"][f"{qps:g}"] = row
    out["saturation_qps"] = sat
    del fields
    return out


def run_serving(args):
    """The serving form at one offered rate (--qps, --duration) or, with
    --qps 0, the saturation curve over the default rates."""
    hc, torch, dev = _setup()
    qps = SERVING_QPS if args.qps <= 0 else (args.qps,)
    print(json.dumps(measure_serving(hc, torch, dev, args.fields, qps, args.duration)))
    return 0


def measure_hszx(hc, torch, dev, fields):
    """The block-mean (HSZx) form of the paper-like workload: the same five
    fields compressed with block means as metadata (block 32, eb 1e-3
    value-range relative).  Per field and operation: the fused time at every
    stage it is defined at (mean at stages 1, 2, 3; standard deviation at 2
    and 3; all stencils in one pass at 3) and the plain path (decompress to
    float32, then the operation), median CUDA-event time over REPS runs with
    an L2 flush before each.  GB/s counts the field's original bytes."""
    rows = []
    tot = {}
    for shape, x in fields:
        xd = torch.from_numpy(x).to(dev)
        cx = hc._trim(hc.compress(xd, EB, rel=True, S=BLOCK, predictor="mean"))
        cd = hc._trim(hc.compress(xd, EB, rel=True, S=BLOCK))
        del xd
        n = int(np.prod(shape))
        scal = torch.empty(hc.SCALAR_BYTES, dtype=torch.uint8, device=dev)
        df = torch.empty(shape, dtype=torch.float32, device=dev)
        nd = len(shape)
        mo = {"derivative": [torch.empty(shape, dtype=torch.float32, device=dev) for _ in range(nd)],
              "gradmag": torch.empty(shape, dtype=torch.float32, device=dev),
              "laplacian": torch.empty(shape, dtype=torch.float32, device=dev), "stats": scal}
        sf = hc.as_stage(cx, "f", df)

        def plain_stat(fn):
            hc.decompress(cx, "f", out=df)
            fn(sf, out=scal)

        def plain_all():
            hc.decompress(cx, "f", out=df)
            hc.mean(sf, out=scal)
            hc.variance(sf, out=scal)
            for a in range(nd):
                hc.derivative(sf, a, out=mo["derivative"][a])
            hc.gradmag(sf, out=mo["gradmag"])
            hc.laplacian(sf, out=mo["laplacian"])

        t = {
            "mean_stage1": time_call(torch, dev, lambda: hc.mean(cx, level="m", out=scal)),
            "mean_stage2": time_call(torch, dev, lambda: hc.mean(cx, level="p", out=scal)),
            "mean_stage3": time_call(torch, dev, lambda: hc.mean(cx, level="q", out=scal)),
            "mean_plain": time_call(torch, dev, lambda: plain_stat(hc.mean)),
            "std_stage2": time_call(torch, dev, lambda: hc.variance(cx, level="p", out=scal)),
            "std_stage3": time_call(torch, dev, lambda: hc.variance(cx, level="q", out=scal)),
            "std_plain": time_call(torch, dev, lambda: plain_stat(hc.variance)),
            "all_ops_one_pass_stage3": time_call(torch, dev, lambda: hc.multi(cx, outs=mo)),
            "all_ops_plain_decompress_once": time_call(torch, dev, plain_all),
        }
        r = {"field": "x".join(map(str, shape)), "hszx_bytes": cx.nbytes, "delta_bytes": cd.nbytes,
             "ms": {k: round(v, 4) for k, v in t.items()},
             "gbs_orig": {k: round(n * 4 / v / 1e6, 1) for k, v in t.items()},
             "speedup_vs_plain": {"mean_stage1": round(t["mean_plain"] / t["mean_stage1"], 2),
                                  "mean_stage2": round(t["mean_plain"] / t["mean_stage2"], 2),
                                  "mean_stage3": round(t["mean_plain"] / t["mean_stage3"], 2),
                                  "std_stage2": round(t["std_plain"] / t["std_stage2"], 2),
                                  "std_stage3": round(t["std_plain"] / t["std_stage3"], 2),
                                  "all_ops_one_pass": round(t["all_ops_plain_decompress_once"] /
                                                            t["all_ops_one_pass_stage3"], 2)}}
        rows.append(r)
        for k, v in t.items():
            tot[k] = tot.get(k, 0.0) + v
        del cx, cd, df, mo
    orig = sum(int(np.prod(sh)) * 4 for sh in synth_shapes())
    line = {"metric": "HSZx (block-mean) operations: GB/s of original data per stage, vs the plain path",
            "unit": "GB/s", "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("block 32;", "block 32, block-mean predictor (HSZx);"),
                       "timing": f"median of {REPS} CUDA-event runs per op, L2 flushed before each"},
            "totals_ms": {k: round(v, 4) for k, v in tot.items()},
            "totals_gbs_orig": {k: round(orig / v / 1e6, 1) for k, v in tot.items()},
            "per_field": rows}
    return line



def run_hszx(args):
    hc, torch, dev = _setup()
    print(json.dumps(measure_hszx(hc, torch, dev, make_fields())))
    return 0

def measure_lorenzo(hc, torch, dev, fields):
    """The global predictors on the paper-like workload: the same five fields
    compressed as HSZp-nd (Lorenzo over the field's axes) and as HSZp (delta
    across blocks over the flattened field), block 32, eb 1e-3 value-range
    relative.  Per field: the stream sizes beside the block-head stream; the
    fused stage-2 mean (weighted sum), the statistics and the derivative along
    the first axis and the Laplacian at stages 2 and 3, against the plain path
    (decompress to float32, then the operation); decompression to D_q.
    Median CUDA-event time over REPS runs with an L2 flush before each; GB/s
    counts the field's original bytes.  The roofline line is the stage-2 mean
    kernel (k_reduce32 on the global predictors) at its algorithmic bytes, the
    compressed stream."""
    peak, peak_src = measured_peaks()
    rows, tot = [], {}
    mean_bytes = 0
    for shape, x in fields:
        xd = torch.from_numpy(x).to(dev)
        cl = hc._trim(hc.compress(xd, EB, rel=True, S=BLOCK, predictor="lorenzo"))
        cg = hc._trim(hc.compress(xd, EB, rel=True, S=BLOCK, predictor="global"))
        cd = hc._trim(hc.compress(xd, EB, rel=True, S=BLOCK))
        del xd
        n = int(np.prod(shape))
        scal = torch.empty(hc.SCALAR_BYTES, dtype=torch.uint8, device=dev)
        df = torch.empty(shape, dtype=torch.float32, device=dev)
        dq = torch.empty(shape, dtype=torch.int32, device=dev)
        fo = torch.empty(shape, dtype=torch.float32, device=dev)
        sf = hc.as_stage(cl, "f", df)

        def plain(op, c=cl):
            hc.decompress(c, "f", out=df)
            op()

        t = {
            "decompress_q": time_call(torch, dev, lambda: hc.decompress(cl, "q", out=dq)),
            "mean_stage2": time_call(torch, dev, lambda: hc.mean(cl, level="p", out=scal)),
            "mean_stage3": time_call(torch, dev, lambda: hc.mean(cl, level="q", out=scal)),
            "mean_plain": time_call(torch, dev, lambda: plain(lambda: hc.mean(sf, out=scal))),
            "std_stage2": time_call(torch, dev, lambda: hc.variance(cl, level="p", out=scal)),
            "std_plain": time_call(torch, dev, lambda: plain(lambda: hc.variance(sf, out=scal))),
            "deriv0_stage2": time_call(torch, dev, lambda: hc.derivative(cl, 0, level="p", out=fo)),
            "deriv0_stage3": time_call(torch, dev, lambda: hc.derivative(cl, 0, level="q", out=fo)),
            "deriv0_plain": time_call(torch, dev, lambda: plain(lambda: hc.derivative(sf, 0, out=fo))),
            "lap_stage2": time_call(torch, dev, lambda: hc.laplacian(cl, level="p", out=fo)),
            "lap_stage3": time_call(torch, dev, lambda: hc.laplacian(cl, level="q", out=fo)),
            "lap_plain": time_call(torch, dev, lambda: plain(lambda: hc.laplacian(sf, out=fo))),
            "hszp_mean_stage2": time_call(torch, dev, lambda: hc.mean(cg, level="p", out=scal)),
            "hszp_mean_plain": time_call(torch, dev, lambda: plain(lambda: hc.mean(sf, out=scal), cg)),
        }
        mean_bytes += cl.nbytes + 64
        sp = lambda a, b: round(t[a] / t[b], 2)
        rows.append({"field": "x".join(map(str, shape)), "lorenzo_bytes": cl.nbytes, "hszp_bytes": cg.nbytes,
                     "delta_bytes": cd.nbytes, "ms": {k: round(v, 4) for k, v in t.items()},
                     "gbs_orig": {k: round(n * 4 / v / 1e6, 1) for k, v in t.items()},
                     "speedup_vs_plain": {"mean_stage2": sp("mean_plain", "mean_stage2"),
                                          "mean_stage3": sp("mean_plain", "mean_stage3"),
                                          "std_stage2": sp("std_plain", "std_stage2"),
                                          "deriv0_stage2": sp("deriv0_plain", "deriv0_stage2"),
                                          "deriv0_stage3": sp("deriv0_plain", "deriv0_stage3"),
                                          "lap_stage2": sp("lap_plain", "lap_stage2"),
                                          "lap_stage3": sp("lap_plain", "lap_stage3"),
                                          "hszp_mean_stage2": sp("hszp_mean_plain", "hszp_mean_stage2")}})
        for k, v in t.items():
            tot[k] = tot.get(k, 0.0) + v
        del cl, cg, cd, df, dq, fo
    orig = sum(int(np.prod(sh)) * 4 for sh in synth_shapes())
    achieved = mean_bytes / (tot["mean_stage2"] * 1e-3) / 1e9
    line = {"metric": "global predictors (HSZp-nd, HSZp): GB/s of original data per stage, vs the plain path",
            "unit": "GB/s", "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("block 32;", "block 32, Lorenzo predictor (HSZp-nd) and "
                                                                 "delta across blocks (HSZp);"),
                       "timing": f"median of {REPS} CUDA-event runs per op, L2 flushed before each"},
            "roofline": {"kernel": "k_reduce32 (global mean)", "bound": "hbm", "achieved": round(achieved, 1),
                         "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_source": peak_src,
                         "algorithmic_bytes": "compressed stream + 64 B per field"},
            "totals_ms": {k: round(v, 4) for k, v in tot.items()},
            "totals_gbs_orig": {k: round(orig / v / 1e6, 1) for k, v in tot.items()},
            "per_field": rows}
    return line



def run_lorenzo(args):
    hc, torch, dev = _setup()
    print(json.dumps(measure_lorenzo(hc, torch, dev, make_fields())))
    return 0

def measure_boxes(hc, torch, dev, fields):
    """HSZx-nd (block means over boxes of codes) on the paper-like workload:
    the five fields in 4x4x4 boxes (8x8 for the 2-D field), eb 1e-3 value-range
    relative.  Per field: the stream size beside 1-D HSZx (block 64) and the
    block-head stream; the mean at stages 1, 2 and 3, the standard deviation
    at stages 2 and 3, the derivative along the first axis and the Laplacian
    at stages 2 and 3, against the plain path (decompress to float32, then the
    operation).  Median CUDA-event time over REPS runs with an L2 flush before
    each; GB/s counts the field's original bytes.  The roofline line is the
    stage-3 variance kernel (k_reduce32 on 64-slot boxes) at its algorithmic
    bytes, the compressed stream."""
    peak, peak_src = measured_peaks()
    rows, tot = [], {}
    var_bytes = 0
    for shape, x in fields:
        block = (4, 4, 4) if len(shape) == 3 else (8, 8)
        xd = torch.from_numpy(x).to(dev)
        cb = hc._trim(hc.compress(xd, EB, rel=True, predictor="mean-nd", block=block))
        cx = hc._trim(hc.compress(xd, EB, rel=True, S=64, predictor="mean"))
        cd = hc._trim(hc.compress(xd, EB, rel=True, S=BLOCK))
        del xd
        n = int(np.prod(shape))
        scal = torch.empty(hc.SCALAR_BYTES, dtype=torch.uint8, device=dev)
        df = torch.empty(shape, dtype=torch.float32, device=dev)
        fo = torch.empty(shape, dtype=torch.float32, device=dev)
        sf = hc.as_stage(cb, "f", df)

        def plain(op):
            hc.decompress(cb, "f", out=df)
            op()

        t = {
            "mean_stage1": time_call(torch, dev, lambda: hc.mean(cb, level="m", out=scal)),
            "mean_stage2": time_call(torch, dev, lambda: hc.mean(cb, level="p", out=scal)),
            "mean_plain": time_call(torch, dev, lambda: plain(lambda: hc.mean(sf, out=scal))),
            "std_stage2": time_call(torch, dev, lambda: hc.variance(cb, level="p", out=scal)),
            "std_stage3": time_call(torch, dev, lambda: hc.variance(cb, level="q", out=scal)),
            "std_plain": time_call(torch, dev, lambda: plain(lambda: hc.variance(sf, out=scal))),
            "deriv0_stage2": time_call(torch, dev, lambda: hc.derivative(cb, 0, level="p", out=fo)),
            "deriv0_stage3": time_call(torch, dev, lambda: hc.derivative(cb, 0, level="q", out=fo)),
            "deriv0_plain": time_call(torch, dev, lambda: plain(lambda: hc.derivative(sf, 0, out=fo))),
            "lap_stage2": time_call(torch, dev, lambda: hc.laplacian(cb, level="p", out=fo)),
            "lap_stage3": time_call(torch, dev, lambda: hc.laplacian(cb, level="q", out=fo)),
            "lap_plain": time_call(torch, dev, lambda: plain(lambda: hc.laplacian(sf, out=fo))),
        }
        var_bytes += cb.nbytes + 64
        sp = lambda a, b: round(t[a] / t[b], 2)  # noqa: E731
        rows.append({"field": "x".join(map(str, shape)), "block": list(block), "box_bytes": cb.nbytes,
                     "hszx_s64_bytes": cx.nbytes, "delta_bytes": cd.nbytes,
                     "ms": {k: round(v, 4) for k, v in t.items()},
                     "gbs_orig": {k: round(n * 4 / v / 1e6, 1) for k, v in t.items()},
                     "speedup_vs_plain": {"mean_stage1": sp("mean_plain", "mean_stage1"),
                                          "mean_stage2": sp("mean_plain", "mean_stage2"),
                                          "std_stage2": sp("std_plain", "std_stage2"),
                                          "std_stage3": sp("std_plain", "std_stage3"),
                                          "deriv0_stage2": sp("deriv0_plain", "deriv0_stage2"),
                                          "deriv0_stage3": sp("deriv0_plain", "deriv0_stage3"),
                                          "lap_stage2": sp("lap_plain", "lap_stage2"),
                                          "lap_stage3": sp("lap_plain", "lap_stage3")}})
        for k, v in t.items():
            tot[k] = tot.get(k, 0.0) + v
        del cb, cx, cd, df, fo
    orig = sum(int(np.prod(sh)) * 4 for sh in synth_shapes())
    achieved = var_bytes / (tot["std_stage3"] * 1e-3) / 1e9
    line = {"metric": "HSZx-nd (box means): GB/s of original data per stage, vs the plain path",
            "unit": "GB/s", "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("block 32;", "boxes of 4x4x4 (8x8 in 2-D), box-mean predictor "
                                                                 "(HSZx-nd);"),
                       "timing": f"median of {REPS} CUDA-event runs per op, L2 flushed before each"},
            "roofline": {"kernel": "k_reduce32 (64-slot boxes)", "bound": "hbm", "achieved": round(achieved, 1),
                         "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_source": peak_src,
                         "algorithmic_bytes": "compressed stream + 64 B per field"},
            "totals_ms": {k: round(v, 4) for k, v in tot.items()},
            "totals_gbs_orig": {k: round(orig / v / 1e6, 1) for k, v in tot.items()},
            "per_field": rows}
    return line



def run_boxes(args):
    hc, torch, dev = _setup()
    print(json.dumps(measure_boxes(hc, torch, dev, make_fields())))
    return 0

def run_profile_boxes():
    """Small case for ncu captures of the HSZx-nd kernels: one 256x384x384
    float32 field in 4x4x4 boxes (compressed ~44 MB, float32 output 151 MB),
    the stage-3 variance three times, then the one-pass Laplacian at stage 2
    (border-corrected) and at stage 3."""
    import torch

    import __graft_entry__
    import synth

    __graft_entry__.build()
    from paper_2603_25206_gb300 import hc

    x = synth.grf_field((256, 384, 384), 1002)
    c = hc.compress(torch.from_numpy(x).cuda(), EB, rel=True, predictor="mean-nd", block=(4, 4, 4))
    out = torch.empty(x.shape, dtype=torch.float32, device="cuda")
    for _ in range(3):
        hc.variance(c, level="q")
    hc.laplacian(c, level="p", out=out)
    hc.laplacian(c, level="q", out=out)
    torch.cuda.synchronize()
    print(json.dumps({"profile_boxes": "ok", "compressed_bytes": c.nbytes, "wmax": int(c.header.wmax)}))
    return 0


def run_hbm_probe():
    """Context for the roofline: HBM write, read and copy bandwidth of plain
    torch operations (fill, sum, copy) on a 4 GiB float32 buffer, CUDA-event
    time over 10 repetitions after 3 warm-ups.  Not a roofline denominator
    (that stays MEASURED_PEAKS.json's copy bandwidth)."""
    import torch

    n = 1 << 30
    x = torch.empty(n, dtype=torch.float32, device="cuda")
    y = torch.empty(n, dtype=torch.float32, device="cuda")

    def t(fn, reps=10):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    w, r, c = t(lambda: x.fill_(1.0)), t(lambda: x.sum()), t(lambda: y.copy_(x))
    print(json.dumps({"hbm_probe": {"write_gbs": round(4 * n / w / 1e6, 1), "read_gbs": round(4 * n / r / 1e6, 1),
                                    "copy_gbs": round(8 * n / c / 1e6, 1), "buffer_bytes": 4 * n}}))
    return 0


def run_profile_lorenzo():
    """Small case for ncu captures of the global-predictor kernels: one
    256x384x384 float32 field as HSZp-nd (compressed ~40 MB, D_q 151 MB), the
    stage-2 mean three times, then decompression to D_q and the stage-2
    derivative along the first axis."""
    import torch

    import __graft_entry__
    import synth

    __graft_entry__.build()
    from paper_2603_25206_gb300 import hc

    x = synth.grf_field((256, 384, 384), 1002)
    c = hc.compress(torch.from_numpy(x).cuda(), EB, rel=True, S=BLOCK, predictor="lorenzo")
    dq = torch.empty(x.shape, dtype=torch.int32, device="cuda")
    out = torch.empty(x.shape, dtype=torch.float32, device="cuda")
    for _ in range(3):
        hc.mean(c, level="p")
    hc.decompress(c, "q", out=dq)
    hc.derivative(c, 0, level="p", out=out)
    torch.cuda.synchronize()
    print(json.dumps({"profile_lorenzo": "ok", "compressed_bytes": c.nbytes, "wmax": int(c.header.wmax)}))
    return 0


def measure_pr1(hc, torch, dev):
    """The small reference configuration: one 64^3 float32 field, the sum of
    8 seeded plane sinusoids plus N(0, 0.01^2) noise, min-max normalised,
    value-range-relative eb 1e-3, block 32.  Every operation fused at stages
    2 and 3, on a materialised stage-3 array, and on the plain path (stage 4),
    each the median of REPS runs with an L2 flush before each.  The field
    (1 MB) fits in L2, so the line is reported for completeness and is not a
    roofline figure."""
    import synth

    peak, _ = measured_peaks()
    shape = (64, 64, 64)
    x = torch.from_numpy(synth.sinusoid_field(shape)).to(dev)
    c = hc._trim(hc.compress(x, EB, rel=True, S=BLOCK))
    del x
    row = cold_table(hc, torch, dev, c, shape, peak, plain=True, split=True)
    return {"metric": "PR1 reference field: ms per operation, fused at stages 2 / 3, on the stage-3 array, "
                      "and on the plain path",
            "config": {"workload": "PR1: 64x64x64 float32, 8 seeded plane sinusoids + N(0, 0.01^2) noise, "
                                   "min-max normalised; value-range-relative eb=1e-3; block 32",
                       "timing": f"median of {REPS} CUDA-event runs per op, L2 flushed before each",
                       "note": "the 1 MB field fits in L2: not a roofline figure"},
            "data": "synthetic", "field": row}


def measure_wide(hc, torch, dev, device_field=False):
    """The wide-code configuration: one float64 512 x 512 x 1024 field (k^-3
    field times 1e4 plus a linear trend), block 64, value-range-relative
    eb 1e-6, and its ABS companion (eps = range / 2^31, block widths in the
    upper 20s).  Per form and operation: fused time (mean, variance with exact
    128-bit sums, derivative per axis into float32 and float64) against the
    plain path (decompress to float64, then the operation), median of REPS
    CUDA-event runs with an L2 flush before each.  GB/s counts the field's
    original bytes (8 per element)."""
    import synth

    shape = (512, 512, 1024)
    if device_field:  # the same recipe drawn on the device (fast; different numbers)
        x = synth.wide_field_device(shape, 3000, dev)
    else:
        x = torch.from_numpy(synth.wide_field(shape, 3000)).to(dev)
    forms = {}
    for form in ("rel_1e-6", "abs_2^-31"):
        if form == "rel_1e-6":
            c = hc._trim(hc.compress(x, 1e-6, rel=True, S=64))
        else:
            lo, hi = float(x.min()), float(x.max())
            xc = x - (hi + lo) / 2
            c = hc._trim(hc.compress(xc, float(xc.max() - xc.min()) / 2**31, rel=False, S=64))
            del xc
        n = int(np.prod(shape))
        scal = torch.empty(hc.SCALAR_BYTES, dtype=torch.uint8, device=dev)
        o32 = torch.empty(shape, dtype=torch.float32, device=dev)
        o64 = torch.empty(shape, dtype=torch.float64, device=dev)
        df = torch.empty(shape, dtype=torch.float64, device=dev)
        sf = hc.as_stage(c, "f", df)

        def plain(fn):
            hc.decompress(c, "f", out=df)
            fn()

        t = {"mean_stage2": time_call(torch, dev, lambda: hc.mean(c, level="p", out=scal)),
             "variance_stage3": time_call(torch, dev, lambda: hc.variance(c, level="q", out=scal)),
             "variance_plain": time_call(torch, dev, lambda: plain(lambda: hc.variance(sf, out=scal)))}
        for a in range(3):
            t[f"derivative{a}_f32"] = time_call(torch, dev, lambda a=a: hc.derivative(c, a, out=o32))
            t[f"derivative{a}_f64"] = time_call(torch, dev, lambda a=a: hc.derivative(c, a, out=o64))
            t[f"derivative{a}_plain_f64"] = time_call(torch, dev, lambda a=a: plain(lambda: hc.derivative(sf, a, out=o64)))
        forms[form] = {"compressed_bytes": c.nbytes, "wmax": int(c.header.wmax), "qmax": int(c.header.qmax),
                       "ms": {k: round(v, 4) for k, v in t.items()},
                       "gbs_orig": {k: round(n * 8 / v / 1e6, 1) for k, v in t.items()}}
        del c, o32, o64, df, sf
    del x
    return {"metric": "wide-code field: GB/s of original data per operation, fused vs plain",
            "unit": "GB/s", "data": "synthetic",
            "config": {"workload": "wide-code: float64 512x512x1024 k^-3 GRF x 1e4 + linear trend, block 64; "
                                   "REL 1e-6 and ABS range/2^31",
                       "timing": f"median of {REPS} CUDA-event runs per op, L2 flushed before each",
                       "field_drawn_on": "device" if device_field else "host"},
            "forms": forms}


def run_wide(args):
    hc, torch, dev = _setup()
    print(json.dumps(measure_wide(hc, torch, dev)))
    return 0


def synth_shapes():
    import synth

    return synth.PAPER_SHAPES


def run_profile_small():
    """Small case for ncu captures: one 256x384x384 float32 field (compressed
    ~44 MB, float32 outputs 151 MB each: larger than L2), each operation 3
    times, then the one-pass call (5 output fields + statistics)."""
    import torch

    import __graft_entry__
    import synth

    __graft_entry__.build()
    from paper_2603_25206_gb300 import hc

    x = synth.grf_field((256, 384, 384), 1002)
    c = hc.compress(torch.from_numpy(x).cuda(), EB, rel=True, S=BLOCK)
    out = torch.empty(x.shape, dtype=torch.float32, device="cuda")
    mouts = {"derivative": [torch.empty(x.shape, dtype=torch.float32, device="cuda") for _ in range(3)],
             "gradmag": torch.empty(x.shape, dtype=torch.float32, device="cuda"), "laplacian": out}
    for _ in range(3):
        hc.derivative(c, 2, out=out)
        hc.gradmag(c, out=out)
        hc.laplacian(c, out=out)
        hc.variance(c, level="q")
        hc.mean(c, level="p")
        hc.decompress(c, "f", out=out)
        hc.multi(c, outs=mouts)
    torch.cuda.synchronize()
    print(json.dumps({"profile_small": "ok", "compressed_bytes": c.nbytes, "wmax": int(c.header.wmax)}))
    return 0


def run_profile_batch():
    """Small case for an ncu capture of the batched kernel: the 64-field
    batched workload at block 32, 256 threads, no tile-height limit (the
    tuned choice), launched 3 times without the autotuner."""
    import torch

    import __graft_entry__
    import synth

    __graft_entry__.build()
    from paper_2603_25206_gb300 import hc

    dev = torch.device("cuda", torch.cuda.current_device())
    shapes = synth.log_uniform_shapes(64, 32, 384, 3)
    comps = []
    for j, sh in enumerate(shapes):
        x = torch.from_numpy(synth.grf_field(sh, 3000 + j)).to(dev)
        comps.append(hc._trim(hc.compress(x, EB, rel=True, S=BLOCK)))
        del x
    b = hc.Batch([(c, "mean|variance|laplacian") for c in comps], threads=256, ty=0)
    for _ in range(3):
        b.run()
    torch.cuda.synchronize()
    assert b.status() == 0
    print(json.dumps({"profile_batch": "ok", "compressed_bytes": sum(c.nbytes for c in comps),
                      "elements": sum(int(np.prod(c.shape)) for c in comps), "grid": b.grid, "smem": b.smem}))
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--profile-small", action="store_true", help="run the small ncu case and exit")
    ap.add_argument("--batched", action="store_true", help="the batched form (64 uneven fields, one launch)")
    ap.add_argument("--profile-batch", action="store_true", help="run the small batched ncu case and exit")
    ap.add_argument("--serving", action="store_true", help="the serving form (200 resident fields, Poisson queries)")
    ap.add_argument("--hszx", action="store_true", help="the block-mean (HSZx) form of the paper-like workload")
    ap.add_argument("--wide", action="store_true", help="the wide-code float64 configuration")
    ap.add_argument("--lorenzo", action="store_true",
                    help="the global predictors (HSZp-nd, HSZp) on the paper-like workload")
    ap.add_argument("--profile-lorenzo", action="store_true", help="run the small global-predictor ncu case")
    ap.add_argument("--boxes", action="store_true", help="HSZx-nd (box means) on the paper-like workload")
    ap.add_argument("--profile-boxes", action="store_true", help="run the small HSZx-nd ncu case")
    ap.add_argument("--hbm-probe", action="store_true", help="HBM write/read/copy bandwidth of plain torch ops")
    ap.add_argument("--fields", type=int, default=200)
    ap.add_argument("--qps", type=float, default=2000.0)
    ap.add_argument("--duration", type=float, default=30.0)
    ap.add_argument("--serving-duration", type=float, default=2.0,
                    help="seconds of queries per offered rate in the default run's saturation curve")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="skip the cold per-operation tables, the error-bound sweep and the other configurations")
    args = ap.parse_args(argv)
    if args.profile_small:
        return run_profile_small()
    if args.profile_batch:
        return run_profile_batch()
    if args.serving:
        return run_serving(args)
    if args.hszx:
        return run_hszx(args)
    if args.wide:
        return run_wide(args)
    if args.lorenzo:
        return run_lorenzo(args)
    if args.profile_lorenzo:
        return run_profile_lorenzo()
    if args.boxes:
        return run_boxes(args)
    if args.profile_boxes:
        return run_profile_boxes()
    if args.hbm_probe:
        return run_hbm_probe()
    if args.batched:
        if args.warmup < 3:
            args.warmup = 3
        return run_batched(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
