"""Shard plans over drawn fields (no GPU): for any length, block size,
predictor (block heads or block means) and number of ranks, the ranks'
shards tile the field in rank order, each is the oracle's own compression
of its slice of codes (but for the two header bounds kept from the whole
field), and the exact sums add up to the whole field's."""
import numpy as np
import pytest

pytest.importorskip("hypothesis")
from hypothesis import HealthCheck, given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

from test_abi_host import _header_from_oracle_stream  # noqa: E402
from test_shard import _build_shard, _chunks  # noqa: E402


@pytest.fixture(scope="module")
def hc():
    from paper_2603_25206_gb300 import build as b

    b.build()
    from paper_2603_25206_gb300 import hc as mod

    mod.lib()
    return mod


@settings(max_examples=200, deadline=None, derandomize=True,
          suppress_health_check=[HealthCheck.too_slow, HealthCheck.function_scoped_fixture])
@given(small=st.booleans(), S=st.sampled_from([1, 3, 8, 32, 33, 64, 500, 4096]), pred=st.integers(0, 1),
       world=st.integers(1, 9), seed=st.integers(0, 2**31 - 1), f64=st.booleans())
def test_shards_tile_the_field(hc, orc, small, S, pred, world, seed, f64):
    # the length is drawn by the seeded generator: spread evenly up to 15 chunks, or small
    rng = np.random.default_rng(seed)
    n = 1 + int(rng.integers(0, 300 if small else 60000))
    dtype = np.float64 if f64 else np.float32
    x = np.cumsum(rng.standard_normal(n)).astype(dtype)
    s, eps = orc.compress(x, 1e-3, True, S, pred=pred)
    h = _header_from_oracle_stream(hc, orc, s)
    q = orc.decode(s, "q").reshape(-1)
    chunks = _chunks(orc, s, h)
    pos, t1, t2 = 0, 0, 0
    for rank in range(world):
        c0, c1 = hc.shard_range(int(h.nchunks), rank, world)
        if c1 <= c0:
            continue
        plan, rebased = hc.shard_plan(h, chunks, c0, c1)
        assert int(plan.first) == pos
        sh = _build_shard(s, plan, rebased)
        m = int(plan.hdr.N)
        alone = orc.compress_codes(q[pos:pos + m], eps, S, dtype, eb=1e-3, rel=True, pred=pred)
        assert alone.size == sh.size
        assert set(np.nonzero(alone != sh)[0].tolist()) <= set(range(60, 64)) | set(range(136, 140))
        a, b = orc.sums_q(q[pos:pos + m])
        t1, t2, pos = t1 + a, t2 + b, pos + m
    assert pos == n
    assert (t1, t2) == orc.sums_q(q)


@settings(max_examples=200, deadline=None, derandomize=True,
          suppress_health_check=[HealthCheck.too_slow, HealthCheck.function_scoped_fixture])
@given(data=st.data(), seed=st.integers(0, 2**31 - 1))
def test_plan_copies_stay_inside_both_streams(hc, orc, data, seed):
    """Whatever an ascending chunk index from 0 to the payload size says (a
    stream's index may be corrupt), the plan is either refused as corrupt (a
    range holding more payload than any stream of its size can) or every copy
    it asks for lies inside the whole stream and inside the shard, after the
    shard's header and before its end; so hc.shard's device copies never
    leave their buffers."""
    rng = np.random.default_rng(seed)
    n = 1 + int(rng.integers(4096 * 2, 4096 * 12))
    S = data.draw(st.sampled_from([1, 32, 100]))
    x = np.cumsum(rng.standard_normal(n)).astype(np.float32)
    s, _ = orc.compress(x, 1e-3, True, S, pred=data.draw(st.integers(0, 1)))
    h = _header_from_oracle_stream(hc, orc, s)
    nc, pw = int(h.nchunks), int(h.payload_words)
    inner = np.sort(rng.integers(0, pw + 1, size=nc - 1)) if nc > 1 else np.zeros(0, np.int64)
    chunks = np.concatenate([[0], inner, [pw]]).astype(np.uint64)
    c0 = data.draw(st.integers(0, nc - 1))
    c1 = data.draw(st.integers(c0 + 1, nc))
    try:
        plan, rebased = hc.shard_plan(h, chunks, c0, c1)
    except hc.HcError as e:
        assert e.status == hc.HC_ERR_CORRUPT
        return
    total, shard_total = int(h.total_bytes), int(plan.hdr.total_bytes)
    for k in range(3):
        so, do, nb = int(plan.src_off[k]), int(plan.dst_off[k]), int(plan.nbytes[k])
        assert nb >= 0 and 0 <= so and so + nb <= total
        assert 256 <= do and do + nb <= shard_total
    co = int(plan.chunks_off)
    assert 256 <= co and co + 8 * rebased.size <= shard_total
    assert rebased[0] == 0 and np.all(np.diff(rebased.astype(np.int64)) >= 0)
    assert int(rebased[-1]) == int(plan.hdr.payload_words)
