"""Serving loop: homomorphic queries on device-resident compressed fields.

Every field stays resident on the device in compressed form.  Queries
(field, operation, stage) arrive over time; the server admits them as CUDA
stream slots and memory under a budget free up, and launches the admitted
queries of each scheduling step together.  Several steps run at once on
separate streams: queries that arrive while earlier ones are on the GPU are
admitted into free slots, and their work overlaps on the device (continuous
batching, not a queue served one request at a time).

Stages follow Table 1's numbering: a query at stage "q" runs the fused
operation on the codes q (Section V, "Operation with D_q"); at stage "p" the
fused stage-2 form (the block-weighted mean of Section V-A, or the variance
through the eta accumulator); at stage "f" the plain path (decompress to
floats, then the operation).  The stage-"q" queries of a step go into one
batched fused launch (hc_batch_run); the others run as one-field calls on the
same stream.

Latency is the time from a query's arrival to the host observing its step
complete (a CUDA event); throughput counts completed queries and the
original bytes of the fields they covered.

The admission policy (`Scheduler`) is plain Python with no CUDA, so it can be
exercised with a simulated executor; `GpuExecutor` runs the steps on the
device through the C ABI.
"""
from __future__ import annotations

import collections
import ctypes
import time
from dataclasses import dataclass, field

import numpy as np

OPS = ("mean", "variance", "gradmag")
# stages a query of each operation may ask for
STAGES = {"mean": ("p", "q", "f"), "variance": ("p", "q", "f"), "gradmag": ("q", "f")}


@dataclass
class Query:
    qid: int
    t_arrive: float  # seconds from the start of the run
    field: int
    op: str
    stage: str


@dataclass
class Record:
    qid: int
    t_arrive: float
    t_admit: float
    t_done: float
    batch: int
    result: object = None

    @property
    def latency(self):
        return self.t_done - self.t_arrive


def poisson_queries(n_fields: int, rate: float, duration: float, seed: int, ops=OPS, stages=STAGES,
                    plain: bool = False):
    """A seeded Poisson arrival stream: exponential gaps of mean 1/rate over
    `duration` seconds; each query picks a field, an operation and a stage
    uniformly (the stage among those its operation supports, or "f" for
    every query when plain=True)."""
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        f = int(rng.integers(n_fields))
        op = ops[int(rng.integers(len(ops)))]
        st = stages[op][int(rng.integers(len(stages[op])))]
        out.append(Query(len(out), t, f, op, "f" if plain else st))
    return out


class Scheduler:
    """Admission and batching policy (no CUDA).

    - Queries wait in arrival order.
    - A step takes the oldest waiting queries, up to `max_batch`, while the
      memory they need fits in what the budget leaves free; it needs a free
      slot (at most `slots` steps in flight).
    - A query that alone exceeds the budget is refused (recorded as such).
    """

    def __init__(self, budget_bytes: int, slots: int, max_batch: int, need_bytes):
        self.budget = int(budget_bytes)
        self.slots = int(slots)
        self.max_batch = int(max_batch)
        self.need = need_bytes
        self.waiting = collections.deque()
        self.in_use = 0  # bytes reserved by steps in flight
        self.in_flight = 0
        self.refused = []
        self.peak_bytes = 0

    def arrive(self, q: Query):
        if self.need(q) > self.budget:
            self.refused.append(q)
        else:
            self.waiting.append(q)

    def next_step(self):
        """The queries of the next step (and their bytes), or None."""
        if self.in_flight >= self.slots or not self.waiting:
            return None
        batch, mem = [], 0
        while self.waiting and len(batch) < self.max_batch:
            need = self.need(self.waiting[0])
            if self.in_use + mem + need > self.budget:
                break
            batch.append(self.waiting.popleft())
            mem += need
        if not batch:
            return None
        self.in_use += mem
        self.in_flight += 1
        self.peak_bytes = max(self.peak_bytes, self.in_use)
        return batch, mem

    def finish(self, mem: int):
        self.in_use -= mem
        self.in_flight -= 1


class StepTimeout(RuntimeError):
    """A step stayed in flight longer than serve's step_timeout.  Its memory
    and slot stay reserved (the device may still be using them); the caller
    decides whether to wait longer or to abandon the device."""

    def __init__(self, step: int, qids, waited: float):
        super().__init__(f"step {step} (queries {list(qids)}) still in flight after {waited:.3f} s")
        self.step, self.qids, self.waited = step, list(qids), waited


def serve(queries, executor, scheduler: Scheduler, clock=time.perf_counter, idle=None, step_timeout=None):
    """Run the arrival stream through the scheduler and executor.  Returns
    the records of the completed queries in completion order.

    executor.launch(batch) -> handle; executor.done(handle) -> bool;
    executor.results(handle) -> list of per-query results (or Nones).
    Every wait for a step is a poll; with step_timeout (seconds) a step still
    in flight that long raises StepTimeout instead of being polled forever."""
    queries = sorted(queries, key=lambda q: q.t_arrive)
    n = len(queries)
    t0 = clock()
    i = 0
    inflight = []  # (handle, batch, mem, t_admit, step)
    records = []
    step = 0
    while i < n or scheduler.waiting or inflight:
        now = clock() - t0
        while i < n and queries[i].t_arrive <= now:
            scheduler.arrive(queries[i])
            i += 1
        keep = []
        for h, batch, mem, t_admit, k in inflight:
            if executor.done(h):
                t_done = clock() - t0
                res = executor.results(h)
                for q, r in zip(batch, res):
                    records.append(Record(q.qid, q.t_arrive, t_admit, t_done, k, r))
                scheduler.finish(mem)
            else:
                waited = clock() - t0 - t_admit
                if step_timeout is not None and waited > step_timeout:
                    raise StepTimeout(k, [q.qid for q in batch], waited)
                keep.append((h, batch, mem, t_admit, k))
        inflight = keep
        while True:
            nxt = scheduler.next_step()
            if nxt is None:
                break
            batch, mem = nxt
            t_admit = clock() - t0
            inflight.append((executor.launch(batch), batch, mem, t_admit, step))
            step += 1
        if idle is not None and not inflight and i < n and not scheduler.waiting:
            idle(queries[i].t_arrive - (clock() - t0))
    return records


def summarize(records, queries, field_bytes, wall: float = None):
    """p50 / p99 latency (ms), throughput (queries/s) and original bytes per
    second (each query counts its field's original bytes once)."""
    if not records:
        return {"completed": 0}
    lat = np.array([r.latency for r in records]) * 1e3
    by_id = {q.qid: q for q in queries}
    span = wall if wall is not None else max(r.t_done for r in records) - min(r.t_arrive for r in records)
    orig = sum(field_bytes[by_id[r.qid].field] for r in records)
    return {"completed": len(records), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
            "span_s": float(span), "qps": len(records) / span, "orig_gbs": orig / span / 1e9,
            "steps": len({r.batch for r in records}),
            "mean_batch": len(records) / max(1, len({r.batch for r in records}))}


# ------------------------------------------------------------------ device
class _Slot:
    def __init__(self, hc, torch, dev, max_batch):
        self.stream = torch.cuda.Stream(device=dev)
        cap = int(hc.lib().hc_batch_plan_bytes(max_batch))
        self.h_plan = torch.empty(cap, dtype=torch.uint8).pin_memory()
        self.d_plan = torch.empty(cap, dtype=torch.uint8, device=dev)
        self.ws = torch.zeros(int(hc.lib().hc_batch_workspace_bytes(max_batch)), dtype=torch.uint8, device=dev)
        self.scal = torch.zeros((max_batch, hc.SCALAR_BYTES), dtype=torch.uint8, device=dev)
        self.items = (hc.HcBatchItem * max_batch)()
        self.event = torch.cuda.Event()


class GpuExecutor:
    """Runs scheduler steps on the device.  fields: list of hc.Compressed
    (resident).  keep_results: copy every result back (scalars as parsed
    dicts, field outputs as device tensors) for checking."""

    def __init__(self, hc, fields, slots: int = 4, max_batch: int = 64, keep_results: bool = False, device=None,
                 batch_max_elems: int = 1 << 21):
        import torch

        self.hc, self.torch = hc, torch
        self.fields = fields
        self.dev = device if device is not None else fields[0].stream.device
        self.slots = [_Slot(hc, torch, self.dev, max_batch) for _ in range(slots)]
        self.free = list(range(slots))
        self.keep = keep_results
        self.max_batch = max_batch
        # stage-q queries on fields up to this size share the step's batched
        # launch; larger fields (whose one-field kernels fill the GPU on their
        # own) and lone queries use the one-field entry points
        self.batch_max_elems = batch_max_elems
        self.sizes = []
        for c in fields:
            n = 1
            for d in c.shape:
                n *= int(d)
            self.sizes.append(n)
        # the operation workspace each one-field call allocates on the slot
        # stream (the field's own size: global predictors need scratch)
        self.ws_bytes = [int(hc.lib().hc_workspace_bytes_for(ctypes.byref(c.header))) for c in fields]
        self.op_ws_bytes = int(hc.lib().hc_workspace_bytes())

    def need_bytes(self, q: Query) -> int:
        c = self.fields[q.field]
        n = 1
        for d in c.shape:
            n *= int(d)
        # the 64-byte statistic, the field output of a gradient query (the
        # batched path allocates it too), the float array of the plain path and
        # the workspace of every one-field call the query makes (a batched
        # query uses the slot's preallocated batch workspace; counting a
        # workspace for it as well keeps the bound an upper bound)
        need = 64 + self.ws_bytes[q.field]
        if q.op == "gradmag":
            need += 4 * n
        if q.stage == "f":
            need += (8 if c.dtype == "float64" else 4) * n + self.op_ws_bytes
        return need

    def launch(self, batch):
        hc, torch = self.hc, self.torch
        k = self.free.pop()
        sl = self.slots[k]
        outs = [None] * len(batch)
        scal_rows = [None] * len(batch)
        nq = 0
        small_q = [q for q in batch if q.stage == "q" and self.sizes[q.field] <= self.batch_max_elems]
        use_batch = len(small_q) > 1
        with torch.cuda.stream(sl.stream):
            for j, q in enumerate(batch):
                c = self.fields[q.field]
                if q.stage == "q" and not (use_batch and self.sizes[q.field] <= self.batch_max_elems):
                    if q.op == "gradmag":
                        outs[j] = hc.gradmag(c, stream=sl.stream)
                    else:
                        fn = hc.mean if q.op == "mean" else hc.variance
                        fn(c, level="q", out=sl.scal[j], stream=sl.stream)
                        scal_rows[j] = j
                elif q.stage == "q":
                    it = sl.items[nq]
                    it.d_stream = c.stream.data_ptr()
                    it.hdr = c.header
                    it.axis = 0
                    if q.op == "gradmag":
                        o = torch.empty(c.shape, dtype=torch.float32, device=self.dev)
                        outs[j] = o
                        it.ops = hc.HC_BATCH_GRADMAG
                        it.d_scalar = None
                        it.d_field = o.data_ptr()
                        it.field_dtype = hc.HC_F32
                    else:
                        it.ops = hc.HC_BATCH_MEAN if q.op == "mean" else hc.HC_BATCH_VARIANCE
                        it.d_scalar = sl.scal[j].data_ptr()
                        it.d_field = None
                        scal_rows[j] = j
                    nq += 1
                elif q.stage == "p":
                    fn = hc.mean if q.op == "mean" else hc.variance
                    fn(c, level="p", out=sl.scal[j], stream=sl.stream)
                    scal_rows[j] = j
                else:  # plain path: decompress to floats, then the operation
                    f = hc.decompress(c, "f", stream=sl.stream)
                    sf = hc.as_stage(c, "f", f)
                    if q.op == "gradmag":
                        outs[j] = hc.gradmag(sf, stream=sl.stream)
                    else:
                        fn = hc.mean if q.op == "mean" else hc.variance
                        fn(sf, out=sl.scal[j], stream=sl.stream)
                        scal_rows[j] = j
                    del f, sf
            if nq:
                used = ctypes.c_size_t()
                tune = hc.HcBatchTune(0, 0, 0, 0, 0)
                hc._check(hc.lib().hc_batch_plan(sl.items, nq, ctypes.byref(tune),
                                                 ctypes.c_void_p(sl.h_plan.data_ptr()), sl.h_plan.numel(),
                                                 ctypes.byref(used)))
                sl.d_plan[: used.value].copy_(sl.h_plan[: used.value], non_blocking=True)
                hc._check(hc.lib().hc_batch_run(ctypes.c_void_p(sl.h_plan.data_ptr()),
                                                ctypes.c_void_p(sl.d_plan.data_ptr()),
                                                ctypes.c_void_p(sl.ws.data_ptr()), sl.ws.numel(),
                                                hc._stream_ptr(sl.stream)))
            sl.event.record(sl.stream)
        return (k, batch, outs, scal_rows)

    def done(self, h) -> bool:
        return self.slots[h[0]].event.query()

    def results(self, h):
        k, batch, outs, rows = h
        sl = self.slots[k]
        res = [None] * len(batch)
        if self.keep:
            raw = sl.scal[: len(batch)].cpu().numpy()
            for j in range(len(batch)):
                if rows[j] is not None:
                    res[j] = self.hc.parse_scalar(raw[rows[j]].tobytes())
                elif outs[j] is not None:
                    res[j] = outs[j]
        self.free.append(k)
        return res


def run(hc, fields, queries, budget_bytes: int, slots: int = 4, max_batch: int = 64, keep_results: bool = False,
        batch_max_elems: int = 1 << 21):
    """Serve `queries` on the resident `fields`; returns (records, scheduler)."""
    ex = GpuExecutor(hc, fields, slots=slots, max_batch=max_batch, keep_results=keep_results,
                     batch_max_elems=batch_max_elems)
    sch = Scheduler(budget_bytes, slots, max_batch, ex.need_bytes)
    recs = serve(queries, ex, sch)
    return recs, sch
