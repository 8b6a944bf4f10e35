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
