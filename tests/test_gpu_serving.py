"""Serving loop on the device (needs a GPU): every result served in a mix of
concurrent, batched queries equals the same query served alone, and the
statistics equal the oracle's exact sums."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2603_25206_gb300 import hc

    hc.lib()
    return hc, torch, torch.device("cuda:0")


def test_results_same_alone_and_in_the_mix(env, orc):
    import synth
    from paper_2603_25206_gb300 import serving

    hc, torch, dev = env
    rng = np.random.default_rng(5)
    fields, refs = [], []
    for j in range(12):
        shape = tuple(int(v) for v in rng.integers(16, 72, size=3))
        eb = (1e-2, 1e-3, 1e-4)[j % 3]
        x = synth.grf_field(shape, 4000 + j)
        ref, eps = orc.compress(x, eb, True, 32)
        c = hc.compress(torch.from_numpy(x).to(dev), eb, rel=True, S=32)
        fields.append(hc._trim(c))
        refs.append((orc.decode(ref, "q"), eps))
    # a burst: far more queries than one step holds, arriving while earlier steps run
    qs = serving.poisson_queries(len(fields), 40000.0, 0.01, 4)
    assert len(qs) > 200
    recs, sch = serving.run(hc, fields, qs, budget_bytes=64 << 20, slots=4, max_batch=16, keep_results=True)
    assert sorted(r.qid for r in recs) == [q.qid for q in qs]
    assert len({r.batch for r in recs}) > 4  # several steps ...
    assert max(sum(1 for r in recs if r.batch == b) for b in {r.batch for r in recs}) > 1  # ... of several queries
    assert sch.peak_bytes <= 64 << 20
    by_id = {r.qid: r for r in recs}
    for q in qs:
        mixed = by_id[q.qid].result
        alone, _ = serving.run(hc, fields, [serving.Query(0, 0.0, q.field, q.op, q.stage)], budget_bytes=64 << 20,
                               slots=1, max_batch=1, keep_results=True)
        alone = alone[0].result
        qf, eps = refs[q.field]
        if q.op == "gradmag":
            assert torch.equal(mixed, alone)
            if q.stage == "q":
                val = orc.stencil_q(qf, orc.KIND_GRADMAG, eps)
                assert np.all(np.abs(mixed.cpu().numpy() - val) <= 1e-6 * np.maximum(np.abs(val), eps))
        else:
            for k in ("mean", "variance", "s1", "s2", "status"):
                a, b = mixed[k], alone[k]
                assert a == b or (isinstance(a, float) and np.isnan(a) and np.isnan(b)), (q, k)
            if q.stage in ("p", "q"):
                s1, s2 = orc.sums_q(qf)
                assert mixed["s1"] == s1
                if q.op == "variance":
                    assert mixed["s2"] == s2
                m_ref, v_ref, _ = orc.finalize(qf.size, s1, s2, eps)
                assert abs(mixed["mean"] - m_ref) <= 1e-12 * max(abs(m_ref), eps)
