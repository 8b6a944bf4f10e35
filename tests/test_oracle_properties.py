"""Property-based checks of the CPU oracle: invariants that the paper's
definitions fix at any size, drawn by hypothesis over small shapes (1-D to
3-D, ragged), block sizes, box extents, predictors and code magnitudes.

* Every stage of every predictor round-trips to the codes (Algorithm 2).
* Section V-A: the stage-2 sums (block-weighted, eta accumulator, the HSZx
  and HSZx-nd forms, the global predictors' weighted sums and Algorithm 4)
  equal the exact stage-3 sums; the stage-1 sum of the block means is within
  N/2 of them (Section V-D: each block mean is off by at most 1/2 per code).
* Section V-B: the stage-2 derivative and Laplacian numerators of HSZp-nd and
  HSZx-nd equal the stage-3 numerators on the same codes.
* Section IV: every reconstructed value is within eps of the input.

Draws are derandomized, so the suite is reproducible.
"""
import numpy as np
import pytest

pytest.importorskip("hypothesis")
from hypothesis import HealthCheck, assume, given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

SETTINGS = settings(max_examples=200, deadline=None, derandomize=True,
                    suppress_health_check=[HealthCheck.too_slow, HealthCheck.function_scoped_fixture])


@st.composite
def codes(draw):
    """Codes of a small field: a smooth walk or noise, with magnitudes from 0
    (constant) to 2^26 (the residual of the 3-D Lorenzo predictor stays below
    2^31), optionally a few spikes."""
    ndim = draw(st.integers(1, 3))
    shape = tuple(draw(st.integers(1, 11 if ndim == 3 else (40 if ndim == 2 else 300))) for _ in range(ndim))
    amp = draw(st.sampled_from([0, 1, 5, 300, 1 << 16, 1 << 26]))
    smooth = draw(st.booleans())
    spikes = draw(st.booleans())
    rng = np.random.default_rng(draw(st.integers(0, 2**31 - 1)))
    if smooth:
        q = np.cumsum(rng.integers(-3, 4, size=shape), axis=-1) * max(1, amp // 64)
    else:
        q = rng.integers(-amp, amp + 1, size=shape)
    if spikes and q.size > 3:
        idx = rng.integers(0, q.size, size=3)
        q.reshape(-1)[idx] = rng.choice([-1, 1], size=3) * amp
    return np.clip(q, -(1 << 26), 1 << 26).astype(np.int32)


@SETTINGS
@given(q=codes(), S=st.sampled_from([1, 2, 3, 7, 16, 32, 33, 64, 100]), pred=st.integers(0, 3))
def test_every_stage_round_trips(orc, q, S, pred):
    eps = 0.25
    s = orc.compress_codes(q, eps, S, np.float64, pred=pred)
    h = orc.read_header(s)
    assert (h["N"], h["nb"], h["pred"]) == (q.size, -(-q.size // S), pred)
    np.testing.assert_array_equal(orc.decode(s, "q"), q)
    np.testing.assert_array_equal(orc.decode(s, "f"), orc.dequantize(q, eps, np.float64))
    assert orc.compress_codes(orc.decode(s, "q"), eps, S, np.float64, pred=pred).tobytes() == s.tobytes()


@SETTINGS
@given(q=codes(), S=st.sampled_from([1, 4, 16, 32, 37, 128]), pred=st.integers(0, 3))
def test_stage2_sums_equal_stage3(orc, q, S, pred):
    s = orc.compress_codes(q, 0.5, S, np.float32, pred=pred)
    dp = orc.decode(s, "p")
    s1, s2 = orc.sums_q(q)
    assert s1 == int(q.astype(np.int64).sum())
    if pred == 0:
        assert orc.mean_p_sum(dp, S) == s1
        assert orc.var_p_sums(dp, S) == (s1, s2)
    elif pred == 1:
        M = orc.decode(s, "m")
        assert orc.mean_p_sum_x(dp, M, S) == s1
        assert 2 * abs(orc.mean_m_sum(M, S, q.size) - s1) <= q.size
    else:
        assert orc.lorenzo_mean_p(dp, pred) == s1
        assert orc.lorenzo_var_p(dp, pred) == (s1, s2)


@SETTINGS
@given(q=codes())
def test_hszp_nd_stage2_stencils_equal_stage3(orc, q):
    s = orc.compress_codes(q, 0.5, 32, np.float32, pred=orc.PRED_LORENZO)
    dp = orc.decode(s, "p")
    for a in range(q.ndim):
        np.testing.assert_array_equal(orc.lorenzo_deriv_p(dp, a), orc.deriv_q(q, a))
    np.testing.assert_array_equal(orc.lorenzo_lap_p(dp), orc.lap_q(q))


@st.composite
def boxes(draw, q):
    ext = [draw(st.integers(1, 6)) for _ in range(q.ndim)]
    return tuple(ext)


@SETTINGS
@given(data=st.data(), q=codes())
def test_hszx_nd_stages_sums_and_stencils(orc, data, q):
    block = data.draw(boxes(q))
    s = orc.compress_codes_nd(q, block, 0.5)
    h = orc.read_header(s)
    assert h["pred"] == orc.PRED_MEAN_ND and h["block"] == block
    np.testing.assert_array_equal(orc.decode(s, "q"), q)
    dp, M = orc.decode(s, "p"), orc.decode(s, "m")
    s1 = int(q.astype(np.int64).sum())
    assert orc.xnd_mean_p(dp, M, block) == s1
    assert 2 * abs(orc.xnd_mean_m(M, q.shape, block) - s1) <= q.size
    for a in range(q.ndim):
        np.testing.assert_array_equal(orc.xnd_deriv_p(dp, M, block, a), orc.deriv_q(q, a))
    np.testing.assert_array_equal(orc.xnd_lap_p(dp, M, block), orc.lap_q(q))


@SETTINGS
@given(q=codes(), dtype=st.sampled_from([np.float32, np.float64]), eb=st.sampled_from([1e-1, 1e-3, 1e-5]),
       rel=st.booleans(), pred=st.integers(0, 3), S=st.sampled_from([3, 32, 64]))
def test_error_bound_holds(orc, q, dtype, eb, rel, pred, S):
    x = (q.astype(np.float64) * 1e-4 + np.sin(np.arange(q.size)).reshape(q.shape)).astype(dtype)
    # codes below 2^27 keep every predictor's residual inside the encoder's 31 bits
    assume(int(np.abs(orc.quantize(x, orc.eps_for(x, eb, rel)).astype(np.int64)).max()) < (1 << 27))
    s, eps = orc.compress(x, eb, rel, S, pred=pred)
    f = orc.decode(s, "f")
    err = np.abs(f.astype(np.float64) - x.astype(np.float64))
    slack = 0.0 if dtype == np.float64 else np.spacing(np.abs(f)).astype(np.float64)
    assert np.all(err <= eps * (1 + 1e-12) + slack)


@SETTINGS
@given(q=codes(), eps=st.sampled_from([1e-6, 1e-3, 0.5, 7.0]))
def test_homomorphic_equals_generic_flow(orc, q, eps):
    """Section V-D: on the same codes, the homomorphic results (integer sums
    and numerators, scaled once) equal the generic flow on D_f = 2 eps q in
    float64 up to rounding: a few units in the last place of the field's
    scale 2 eps max|q| (its square for the variance)."""
    f = orc.dequantize(q, eps, np.float64)
    ulp = 2.0**-52 * 2 * eps * max(1, int(np.abs(q.astype(np.int64)).max()))
    for a in range(q.ndim):
        np.testing.assert_allclose(orc.stencil_q(q, orc.KIND_DERIV, eps, a), orc.stencil_f(f, orc.KIND_DERIV, a),
                                   rtol=0, atol=8 * ulp)
    np.testing.assert_allclose(orc.stencil_q(q, orc.KIND_GRADMAG, eps), orc.stencil_f(f, orc.KIND_GRADMAG),
                               rtol=0, atol=16 * ulp)
    np.testing.assert_allclose(orc.stencil_q(q, orc.KIND_LAPLACIAN, eps), orc.stencil_f(f, orc.KIND_LAPLACIAN),
                               rtol=0, atol=32 * q.ndim * ulp)
    mean, var, _ = orc.finalize(q.size, *orc.sums_q(q), eps)
    mf, vf = orc.stats_f(f)
    assert abs(mean - mf) <= 4 * ulp
    if q.size > 1:
        assert abs(var - vf) <= 16 * ulp * ulp / 2.0**-52 + 1e-12 * vf
