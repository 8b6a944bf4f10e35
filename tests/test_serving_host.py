"""Serving loop policy on the host (no GPU): admission under a memory budget
and a slot limit, arrival order, continuous batching, and the statistics."""
import numpy as np
import pytest

from paper_2603_25206_gb300 import serving


class FakeClock:
    """Deterministic clock: every reading advances time by `tick` seconds."""

    def __init__(self, tick=1e-5):
        self.t = 0.0
        self.tick = tick

    def __call__(self):
        self.t += self.tick
        return self.t


class FakeExecutor:
    """A step finishes `base + per_query * len(batch)` seconds after launch."""

    def __init__(self, clock, base=2e-4, per_query=5e-5, need=lambda q: 100):
        self.clock = clock
        self.base, self.per = base, per_query
        self.need_bytes = need
        self.launches = []  # (t_launch, t_finish, qids)
        self.running = 0
        self.max_running = 0

    def launch(self, batch):
        now = self.clock.t
        fin = now + self.base + self.per * len(batch)
        self.launches.append((now, fin, [q.qid for q in batch]))
        self.running += 1
        self.max_running = max(self.max_running, self.running)
        return len(self.launches) - 1

    def done(self, h):
        if self.clock.t >= self.launches[h][1]:
            return True
        return False

    def results(self, h):
        self.running -= 1
        return [("r", qid) for qid in self.launches[h][2]]


def _run(queries, budget=10_000, slots=3, max_batch=8, need=lambda q: 100, **kw):
    clk = FakeClock()
    ex = FakeExecutor(clk, need=need, **kw)
    sch = serving.Scheduler(budget, slots, max_batch, need)
    recs = serving.serve(queries, ex, sch, clock=clk)
    return recs, sch, ex


def test_poisson_stream_seeded_and_valid():
    a = serving.poisson_queries(10, 2000.0, 1.0, 4)
    b = serving.poisson_queries(10, 2000.0, 1.0, 4)
    assert [(q.t_arrive, q.field, q.op, q.stage) for q in a] == [(q.t_arrive, q.field, q.op, q.stage) for q in b]
    assert abs(len(a) - 2000) < 5 * np.sqrt(2000)
    assert all(0 <= q.field < 10 and q.stage in serving.STAGES[q.op] for q in a)
    assert all(x.t_arrive < y.t_arrive for x, y in zip(a, a[1:]))
    assert {q.op for q in a} == set(serving.OPS)
    p = serving.poisson_queries(10, 2000.0, 1.0, 4, plain=True)
    assert all(q.stage == "f" for q in p) and [q.field for q in p] == [q.field for q in a]


def test_every_query_completes_once_in_arrival_order():
    qs = serving.poisson_queries(5, 20000.0, 0.05, 1)
    recs, sch, ex = _run(qs)
    assert sorted(r.qid for r in recs) == [q.qid for q in qs]
    # admission follows arrival order
    by_admit = sorted(recs, key=lambda r: (r.t_admit, r.qid))
    assert [r.qid for r in by_admit] == sorted(r.qid for r in recs)
    assert all(r.t_arrive <= r.t_admit <= r.t_done for r in recs)
    assert sch.in_use == 0 and sch.in_flight == 0


def test_slots_and_budget_respected_and_work_overlaps():
    qs = serving.poisson_queries(5, 50000.0, 0.02, 2)
    need = lambda q: 1000 if q.op == "gradmag" else 10  # noqa: E731
    recs, sch, ex = _run(qs, budget=2500, slots=3, max_batch=16, need=need)
    assert sch.peak_bytes <= 2500
    assert ex.max_running <= 3
    # continuous batching: some step starts while an earlier one is still running
    overlap = any(ex.launches[k][0] < ex.launches[k - 1][1] for k in range(1, len(ex.launches)))
    assert overlap
    assert all(len(ids) <= 16 for _, _, ids in ex.launches)
    # every step's memory fits the budget on its own
    for _, _, ids in ex.launches:
        assert sum(need(qs[i]) for i in ids) <= 2500


def test_over_budget_query_refused_not_blocking():
    qs = [serving.Query(0, 0.0, 0, "gradmag", "q"), serving.Query(1, 0.0, 1, "mean", "q"),
          serving.Query(2, 1e-4, 0, "mean", "p")]
    need = lambda q: 10**9 if q.qid == 0 else 10  # noqa: E731
    recs, sch, ex = _run(qs, budget=1000, need=need)
    assert [q.qid for q in sch.refused] == [0]
    assert sorted(r.qid for r in recs) == [1, 2]


def test_summary_percentiles():
    qs = [serving.Query(i, 0.0, i % 2, "mean", "q") for i in range(100)]
    recs = [serving.Record(i, 0.0, 0.0, (i + 1) * 1e-3, i // 10) for i in range(100)]
    s = serving.summarize(recs, qs, {0: 4000, 1: 8000})
    assert s["completed"] == 100
    assert s["p50_ms"] == pytest.approx(np.percentile(np.arange(1, 101), 50))
    assert s["p99_ms"] == pytest.approx(np.percentile(np.arange(1, 101), 99))
    assert s["qps"] == pytest.approx(100 / 0.1)
    assert s["orig_gbs"] == pytest.approx((50 * 4000 + 50 * 8000) / 0.1 / 1e9)
    assert s["steps"] == 10 and s["mean_batch"] == 10


def test_step_timeout_raises_instead_of_polling_forever():
    """A step whose completion never comes (its event never fires) ends the
    loop with StepTimeout after step_timeout seconds, naming the step and its
    queries; without a timeout nothing changes for steps that finish."""
    class Stuck(FakeExecutor):
        def done(self, h):
            return False if h == 1 else super().done(h)

    qs = [serving.Query(i, 1e-3 * i, 0, "mean", "q") for i in range(3)]
    clk = FakeClock(tick=1e-4)
    ex = Stuck(clk, base=1e-4, per_query=0.0)
    sch = serving.Scheduler(10_000, 4, 1, lambda q: 100)
    with pytest.raises(serving.StepTimeout) as e:
        serving.serve(qs, ex, sch, clock=clk, step_timeout=0.05)
    assert e.value.step == 1 and e.value.qids == [1] and 0.05 < e.value.waited < 0.06
    assert sch.in_flight >= 1  # the stuck step keeps its slot and memory
    recs, sch2, _ = _run(qs)
    assert sorted(r.qid for r in recs) == [0, 1, 2]
