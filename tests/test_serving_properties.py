"""Serving policy invariants under drawn workloads (no GPU): for any arrival
stream, memory budget, slot count, batch limit and per-query memory need,
the scheduler and the serve loop

* complete every query that fits the budget exactly once and refuse exactly
  those that alone exceed it;
* never reserve more than the budget, never run more steps than slots, and
  never put more than max_batch queries in a step;
* admit in arrival order (continuous batching never lets a later query
  overtake an earlier one);
* end drained: nothing reserved, nothing in flight.

The executor and clock are the deterministic fakes of test_serving_host.
"""
import pytest

pytest.importorskip("hypothesis")
from hypothesis import HealthCheck, given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

from paper_2603_25206_gb300 import serving  # noqa: E402
from test_serving_host import FakeClock, FakeExecutor  # noqa: E402


@st.composite
def workloads(draw):
    n = draw(st.integers(0, 60))
    gaps = draw(st.lists(st.floats(0.0, 5e-4, allow_nan=False), min_size=n, max_size=n))
    t, qs = 0.0, []
    for i, g in enumerate(gaps):
        t += g
        op = draw(st.sampled_from(serving.OPS))
        stage = draw(st.sampled_from(serving.STAGES[op]))
        qs.append(serving.Query(i, t, draw(st.integers(0, 4)), op, stage))
    sizes = draw(st.lists(st.integers(1, 3000), min_size=max(n, 1), max_size=max(n, 1)))
    budget = draw(st.integers(1, 4000))
    slots = draw(st.integers(1, 5))
    max_batch = draw(st.integers(1, 12))
    base = draw(st.floats(1e-5, 1e-3))
    per = draw(st.floats(0.0, 2e-4))
    return qs, sizes, budget, slots, max_batch, base, per


@settings(max_examples=150, deadline=None, derandomize=True, suppress_health_check=[HealthCheck.too_slow])
@given(w=workloads())
def test_scheduler_invariants(w):
    qs, sizes, budget, slots, max_batch, base, per = w
    need = lambda q: sizes[q.qid]  # noqa: E731
    clk = FakeClock()
    ex = FakeExecutor(clk, base=base, per_query=per, need=need)
    sch = serving.Scheduler(budget, slots, max_batch, need)
    recs = serving.serve(qs, ex, sch, clock=clk)
    fits = [q.qid for q in qs if need(q) <= budget]
    assert sorted(r.qid for r in recs) == fits
    assert sorted(q.qid for q in sch.refused) == [q.qid for q in qs if need(q) > budget]
    assert sch.peak_bytes <= budget
    assert ex.max_running <= slots
    assert all(0 < len(ids) <= max_batch for _, _, ids in ex.launches)
    assert all(sum(sizes[i] for i in ids) <= budget for _, _, ids in ex.launches)
    admitted = [qid for _, _, ids in ex.launches for qid in ids]
    assert admitted == fits  # arrival order (queries are numbered in arrival order)
    assert all(r.t_arrive <= r.t_admit <= r.t_done for r in recs)
    assert sch.in_use == 0 and sch.in_flight == 0 and not sch.waiting
