"""The library and the oracle agree on the stream layout, over drawn inputs
(no GPU): for any shape (1-D to 3-D), block size or box extents, predictor
and field type, the library's host header reader (hc_read_header_host, the
parser hc_read_header uses) accepts the stream the oracle writes with the
same fields, refuses it truncated, and the library's compress bound covers
it.  The two sides compute the section layout independently."""
import ctypes

import numpy as np
import pytest

pytest.importorskip("hypothesis")
from hypothesis import HealthCheck, given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

from test_abi_host import _header_from_oracle_stream  # noqa: E402


@pytest.fixture(scope="module")
def hc():
    from paper_2603_25206_gb300 import build as b

    b.build()
    from paper_2603_25206_gb300 import hc as mod

    mod.lib()
    return mod


@settings(max_examples=150, deadline=None, derandomize=True,
          suppress_health_check=[HealthCheck.too_slow, HealthCheck.function_scoped_fixture])
@given(data=st.data(), ndim=st.integers(1, 3), pred=st.integers(0, 4), f64=st.booleans(),
       seed=st.integers(0, 2**31 - 1))
def test_library_reads_every_oracle_header(hc, orc, data, ndim, pred, f64, seed):
    rng = np.random.default_rng(seed)
    shape = tuple(int(rng.integers(1, 70 if ndim < 3 else 20)) for _ in range(ndim))
    q = np.cumsum(rng.integers(-40, 41, size=shape), axis=-1).astype(np.int32)
    dtype = np.float64 if f64 else np.float32
    L = hc.lib()
    dims = (ctypes.c_int64 * 3)(*shape)
    if pred == 4:
        block = tuple(data.draw(st.integers(1, 9)) for _ in range(ndim))
        s = orc.compress_codes_nd(q, block, 0.5, dtype)
        bound = int(L.hc_compress_bound_nd(ndim, dims, (ctypes.c_int32 * 3)(*block)))
    else:
        S = data.draw(st.sampled_from([1, 2, 5, 16, 32, 64, 129, 4096]))
        s = orc.compress_codes(q, 0.5, S, dtype, pred=pred)
        bound = int(L.hc_compress_bound(q.size, S))
    assert 0 < s.size <= bound
    got = hc.header_of(s)
    want = _header_from_oracle_stream(hc, orc, s)
    assert bytes(got) == bytes(want)
    with pytest.raises(hc.HcError) as e:
        hc.header_of(s[:-16])
    assert e.value.status == hc.HC_ERR_CORRUPT
