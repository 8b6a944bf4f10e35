"""Pins of the CPU oracle to what the paper and the mathematics fix.

Each test ties one oracle function to something other than itself: values
printed in the paper (tests/golden), a hand-derived byte image of the stream
layout, closed forms, exact rational arithmetic, library routines (numpy,
scipy) and brute force on tiny arrays.  No GPU is used.
"""
import math
import struct
from fractions import Fraction

import numpy as np
import pytest

from conftest import read_golden_table, GOLDEN

SIZES_S = (1, 2, 3, 4, 7, 16, 31, 32, 33, 64, 100, 128)


# --------------------------------------------------------------- quantization
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_worked_example_codes(orc, dtype):
    """Section IV worked example: Y with eps = 0.1 quantizes to the printed Y_q."""
    g = read_golden_table("worked_example.txt")
    eps = float(g["eps"][0])
    Y = np.array([float(v) for v in g["Y"]], dtype).reshape(2, 4)
    Yq = np.array([int(v) for v in g["Yq"]], np.int32).reshape(2, 4)
    np.testing.assert_array_equal(orc.quantize(Y, eps), Yq)


def test_round_half_up_on_exact_halves(orc):
    """round(t) = floor(t + 1/2): exact half-integers go up (-12.5 -> -12, 12.5 -> 13)."""
    eps = 0.25  # 2 eps = 0.5 is exact, so x / (2 eps) is exact
    k = np.arange(-40, 41)
    x = ((k + 0.5) * 0.5).astype(np.float64)
    np.testing.assert_array_equal(orc.quantize(x, eps), (k + 1).astype(np.int32))
    x2 = (k * 0.5).astype(np.float64)
    np.testing.assert_array_equal(orc.quantize(x2, eps), k.astype(np.int32))


def _err_bound_exact(x, q, eps, sample):
    """max over a sample of |x - 2 eps q| / eps in exact rational arithmetic."""
    e = Fraction(eps)
    worst = Fraction(0)
    for i in sample:
        d = abs(Fraction(float(x.flat[i])) - 2 * e * int(q.flat[i]))
        worst = max(worst, d / e)
    return worst


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("eb,rel", [(1e-2, True), (1e-3, True), (1e-4, True), (0.37, False), (1e-6, True)])
def test_error_bound_every_element(orc, rng, dtype, eb, rel):
    """|d - d'| <= eps for every point (Section III-A and IV), d' = 2 eps q.

    The division x / (2 eps) is rounded once, so the bound holds up to one
    rounding of a double near a half-integer (relative 2^-52)."""
    x = (rng.standard_normal(20000) * 3.0 + rng.uniform(-5, 5)).astype(dtype)
    eps = orc.eps_for(x, eb, rel)
    if rel:
        assert eps == eb * (float(x.max()) - float(x.min()))
    else:
        assert eps == eb
    q = orc.quantize(x, eps)
    err = np.abs(x.astype(np.float64) - q.astype(np.float64) * (2 * eps))
    assert np.all(err <= eps * (1 + 1e-9) + 4 * np.spacing(np.abs(x.astype(np.float64))))
    sample = rng.choice(x.size, 300, replace=False)
    assert _err_bound_exact(x, q, eps, sample) <= 1 + Fraction(1, 2**40)


def test_error_bound_float_field_after_dequantize(orc, rng):
    """The float32 reconstruction stays within eps plus the float32 rounding of d'."""
    x = rng.uniform(-1, 1, 50000).astype(np.float32)
    s, eps = orc.compress(x, 1e-3, True, 32)
    f = orc.decode(s, "f")
    err = np.abs(f.astype(np.float64) - x.astype(np.float64))
    assert np.all(err <= eps + 2 * np.spacing(np.abs(f)).astype(np.float64))


def test_range_and_argument_errors(orc):
    with pytest.raises(orc.OracleError) as e:
        orc.quantize(np.array([1.0, 2.0**31], np.float64), 0.5)
    assert e.value.status == 2
    with pytest.raises(orc.OracleError) as e:
        orc.quantize(np.array([np.nan], np.float64), 0.5)
    assert e.value.status == 2
    with pytest.raises(orc.OracleError) as e:
        orc.compress(np.ones(8, np.float32), -1.0, False, 4)
    assert e.value.status == 1
    # constant field with a relative bound: eps falls back to eb
    assert orc.eps_for(np.full(10, 3.0, np.float32), 1e-3, True) == 1e-3


def test_quantize_limit_is_two_to_the_thirty(orc):
    """Codes satisfy |q| < 2^30 (the stream's code range): with 2 eps = 1,
    x = +-(2^30 - 1) quantises and x = +-2^30, or 2^30 - 1/2 (which rounds up
    to 2^30), is refused as out of range."""
    ok = orc.quantize(np.array([2.0**30 - 1, -(2.0**30 - 1), 2.0**30 - 0.75], np.float64), 0.5)
    assert [int(v) for v in ok] == [2**30 - 1, -(2**30 - 1), 2**30 - 1]
    for v in (2.0**30, -(2.0**30), 2.0**30 - 0.5):
        with pytest.raises(orc.OracleError) as e:
            orc.quantize(np.array([v], np.float64), 0.5)
        assert e.value.status == 2


def test_header_records_the_bound_as_given(orc, rng):
    """The header keeps the bound as the caller gave it (eb and its mode)
    beside the absolute eps it used: eps = eb (max - min) for a value-range
    relative bound (Section VI-B), eps = eb for an absolute one."""
    x = rng.normal(size=(10, 20)).astype(np.float32)
    for eb, rel in ((1e-3, True), (0.01, False)):
        s, eps = orc.compress(x, eb, rel, 32)
        h = orc.read_header(s)
        assert (h["eb"], h["eb_mode"]) == (eb, 1 if rel else 0)
        assert h["eps"] == eps == (eb * (float(x.max()) - float(x.min())) if rel else eb)


# ---------------------------------------------------------------- the stream
def _golden_stream_bytes():
    out = None
    items = []
    with open(f"{GOLDEN}/stream_s4.txt") as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            parts = line.split()
            if parts[0] == "total":
                out = bytearray(int(parts[1]))
                continue
            items.append((int(parts[0]), parts[1], parts[2]))
    fmt = {"u8": "<B", "u16": "<H", "u32": "<I", "i32": "<i", "u64": "<Q", "f64": "<d"}
    for off, ty, val in items:
        v = float(val) if ty == "f64" else int(val, 0)
        b = struct.pack(fmt[ty], v)
        out[off:off + len(b)] = b
    return bytes(out)


def test_stream_matches_hand_derived_bytes(orc):
    """The oracle writes exactly the documented layout (hand-derived S = 4 example)."""
    q = np.array([5, 3, 4, 4, -1, -1, -1, -1, 7, 9], np.int32)
    x = q.astype(np.float32)  # eps = 0.5 -> 2 eps = 1 -> codes are the values
    s, eps = orc.compress(x, 0.5, False, 4)
    assert eps == 0.5
    assert bytes(s) == _golden_stream_bytes()
    np.testing.assert_array_equal(orc.decode(s, "q"), q)
    np.testing.assert_array_equal(orc.decode(s, "m"), [5, -1, 7])
    np.testing.assert_array_equal(orc.decode(s, "p"), [5, -2, 1, 0, -1, 0, 0, 0, 7, 2])


def _py_decode(stream):
    """Independent reader of the layout (numpy, not the oracle's C loops)."""
    s = np.asarray(stream, np.uint8)
    u32 = lambda o: int(s[o:o + 4].view("<u4")[0])
    u64 = lambda o: int(s[o:o + 8].view("<u8")[0])
    S = u32(32)
    N = u64(64)
    nb = u64(72)
    pred = u32(140)
    ow, oh, oc, op = u64(96), u64(104), u64(112), u64(120)
    widths = s[ow:ow + nb].astype(np.int64)
    heads = s[oh:oh + 4 * nb].view("<i4").astype(np.int64)
    nsw = (S + 31) // 32
    words = np.where(widths > 0, nsw + (S * widths + 31) // 32, 0)
    offs = np.concatenate([[0], np.cumsum(words)])
    pw = u64(88)
    payload = s[op:op + 4 * pw].view("<u4").astype(np.uint64)
    bits = ((payload[:, None] >> np.arange(32, dtype=np.uint64)) & 1).reshape(-1)
    q = np.empty(N, np.int64)
    qs = np.zeros((nb, S), np.int64)  # every slot of every block (predictor 4)
    for b in range(nb):
        first = b * S
        Sb = min(S, N - first)
        w = int(widths[b])
        if pred == 4:
            if w == 0:
                qs[b] = heads[b]
                continue
        elif w == 0:  # every p is 0: q = head (delta) or q = M_b (block mean)
            q[first:first + Sb] = heads[b]
            continue
        if pred in (2, 3):
            assert heads[b] == 0
        base = int(offs[b]) * 32
        k = np.arange(S)
        sign = bits[base + k]
        mb = base + nsw * 32 + (k[:, None] * w + np.arange(w)[None, :])
        mag = (bits[mb] << np.arange(w, dtype=np.uint64)).sum(axis=1).astype(np.int64)
        p = np.where(sign == 1, -mag, mag)
        if pred == 4:
            qs[b] = heads[b] + p
            continue
        assert np.all(p[Sb:] == 0)
        if pred >= 2:  # global predictors: the slots hold residuals, no heads
            q[first:first + Sb] = p[:Sb]
        elif pred == 1:  # block mean: q = M_b + p
            q[first:first + Sb] = heads[b] + p[:Sb]
        else:  # delta inside the block: q = head + prefix sum, p_0 = 0
            assert p[0] == 0
            q[first:first + Sb] = heads[b] + np.cumsum(p[:Sb])
    chunk_g = max(1, 4096 // S)
    chunks = s[oc:oc + 8 * (-(-nb // chunk_g) + 1)].view("<u8").astype(np.int64)
    np.testing.assert_array_equal(chunks, offs[::chunk_g].tolist() + ([offs[-1]] if nb % chunk_g else []))
    if pred == 4:  # HSZx-nd: box slots back to field positions (outside slots dropped)
        d = (u64(8), u64(16), u64(24))
        bd = (u32(144), u32(148), u32(152))
        g = [-(-d[a] // bd[a]) for a in range(3)]
        field = np.empty(d, np.int64)
        for b in range(nb):
            k = (b // (g[1] * g[2]), (b // g[2]) % g[1], b % g[2])
            box = qs[b].reshape(bd)
            sl = tuple(slice(k[a] * bd[a], min(d[a], (k[a] + 1) * bd[a])) for a in range(3))
            ext = tuple(sl[a].stop - sl[a].start for a in range(3))
            field[sl] = box[: ext[0], : ext[1], : ext[2]]
        q = field.reshape(-1)
    if pred == 3:  # HSZp: q is the running sum over the flattened field
        q = np.cumsum(q)
    elif pred == 2:  # HSZp-nd: q is the running sum along every axis
        q = q.reshape(u64(8), u64(16), u64(24))
        for a in range(3):
            q = np.cumsum(q, axis=a)
        q = q.reshape(-1)
    return q, widths


@pytest.mark.parametrize("S", SIZES_S)
def test_roundtrip_and_independent_reader(orc, rng, S):
    """c -> D_q recovers the quantized codes exactly; an independent numpy reader of
    the layout agrees; every width is the bit length of the block's max |p|."""
    n = int(rng.integers(1, 700))
    x = np.cumsum(rng.standard_normal(n)).astype(np.float32)
    if n > 5:
        x[rng.integers(0, n, 3)] += 50.0
    s, eps = orc.compress(x, 1e-2, True, S)
    q_ref = orc.quantize(x, eps)
    np.testing.assert_array_equal(orc.decode(s, "q"), q_ref)
    q_py, widths = _py_decode(s)
    np.testing.assert_array_equal(q_py, q_ref)
    for b in range(widths.size):
        blk = q_ref[b * S:(b + 1) * S].astype(np.int64)
        m = int(np.abs(np.diff(blk)).max()) if blk.size > 1 else 0
        assert widths[b] == m.bit_length()
    h = orc.read_header(s)
    assert h["qmax"] == int(np.abs(q_ref).max())
    assert h["wmax"] == int(widths.max())


@pytest.mark.parametrize("S", SIZES_S)
def test_stage_chain(orc, rng, S):
    """c -> D_p -> D_q -> D_f: the in-block inclusive prefix sum of D_p is D_q, and
    D_f = 2 eps q in the field's arithmetic; encoding the codes again is the identity."""
    shape = (3, 5, int(rng.integers(1, 40)))
    x = rng.normal(size=shape).astype(np.float64)
    s, eps = orc.compress(x, 1e-3, True, S)
    dp = orc.decode(s, "p").reshape(-1).astype(np.int64)
    dq = orc.decode(s, "q").reshape(-1)
    n = dq.size
    q_from_p = np.empty(n, np.int64)
    for first in range(0, n, S):
        q_from_p[first:first + S] = np.cumsum(dp[first:first + S])
    np.testing.assert_array_equal(q_from_p, dq)
    np.testing.assert_array_equal(orc.decode(s, "m"), dq[::S])
    f = orc.decode(s, "f").reshape(-1)
    np.testing.assert_array_equal(f, dq.astype(np.float64) * (2 * eps))
    s2 = orc.compress_codes(dq.reshape(shape), eps, S, np.float64, eb=1e-3, rel=True)
    assert bytes(s2) == bytes(s)


def test_float32_dequantize_rule(orc):
    """float32 reconstruction is (float)q * (float)(2 eps) in float32 arithmetic."""
    q = np.array([0, 1, -1, 3, 12345, -(2**29), 2**29 + 7, 16777217], np.int32)
    eps = 0.1234567
    f = orc.dequantize(q, eps, np.float32)
    expect = q.astype(np.float32) * np.float32(2 * eps)
    np.testing.assert_array_equal(f, expect)


def test_corrupt_streams_are_rejected(orc, rng):
    x = rng.normal(size=1000).astype(np.float32)
    s, _ = orc.compress(x, 1e-3, True, 32)
    bad = s.copy()
    bad[0] ^= 0xFF
    with pytest.raises(orc.OracleError) as e:
        orc.decode(bad, "q")
    assert e.value.status == 3
    with pytest.raises(orc.OracleError):
        orc.decode(s[: s.size // 2], "q")
    h = orc.read_header(s)
    bad = s.copy()
    bad[256] = 40  # width > 31
    with pytest.raises(orc.OracleError):
        orc.decode(bad, "q")
    bad = s.copy()
    bad[256] = (int(bad[256]) + 1) % 32  # width changed: payload walk no longer matches
    with pytest.raises(orc.OracleError):
        orc.decode(bad, "q")
    assert h["N"] == 1000


def test_reader_checks_chunk_index_and_walk_total(orc, rng):
    """The reader checks each chunk's stored base against the running sum of
    the block sizes, and the walk's total against the header.  Two streams
    must be refused as corrupt: one with the base of chunk 1 moved by a word,
    and one whose header and chunk-index end both claim 4 more payload words
    than the blocks hold."""
    x = rng.normal(size=20000).astype(np.float32)
    s, _ = orc.compress(x, 1e-3, True, 32)
    h = orc.read_header(s)
    assert h["nchunks"] >= 3 and s.size == h["total_bytes"]
    r16 = lambda v: (v + 15) & ~15  # noqa: E731
    off_chunks = r16(r16(256 + h["nb"]) + 4 * h["nb"])

    def put_u64(buf, off, v):
        buf[off:off + 8] = np.frombuffer(struct.pack("<Q", v), np.uint8)

    def get_u64(buf, off):
        return struct.unpack("<Q", bytes(buf[off:off + 8]))[0]

    bad = s.copy()
    put_u64(bad, off_chunks + 8, get_u64(bad, off_chunks + 8) + 1)
    with pytest.raises(orc.OracleError) as e:
        orc.decode(bad, "q")
    assert e.value.status == 3
    grown = np.zeros(s.size + 16, np.uint8)
    grown[: s.size] = s
    put_u64(grown, 88, h["payload_words"] + 4)
    put_u64(grown, 128, h["total_bytes"] + 16)
    end = off_chunks + 8 * h["nchunks"]
    put_u64(grown, end, get_u64(grown, end) + 4)
    with pytest.raises(orc.OracleError) as e:
        orc.decode(grown, "q")
    assert e.value.status == 3
    np.testing.assert_array_equal(orc.decode(s, "q"), orc.quantize(x, h["eps"]))


# ------------------------------------------------------------------- statistics
def test_worked_example_std_eq_var_q(orc):
    """Eq. var_q on the printed Y_q: sigma = sqrt((740 - 18^2/8)/7) * 0.2 = 1.99928..."""
    g = read_golden_table("worked_example.txt")
    Yq = np.array([int(v) for v in g["Yq"]], np.int32)
    s1, s2 = orc.sums_q(Yq)
    assert (s1, s2) == (18, 740)
    mean, var, sd = orc.finalize(8, s1, s2, 0.1)
    exact_var = (Fraction(740) - Fraction(18 * 18, 8)) / 7 * Fraction(0.2) ** 2
    assert abs(var - float(exact_var)) <= 1e-15 * float(exact_var)
    assert abs(sd - 1.9992855) < 1e-6
    assert abs(mean - 18 / 8 * 0.2) < 1e-15
    # the HSZx stage-2 value of Section V-A uses the rounded integer mean 2:
    mu_t = round(Fraction(18, 8))
    alt = math.sqrt(sum((int(v) - mu_t) ** 2 for v in Yq) / 7) * 0.2
    assert abs(alt - float(g["sigma_p_hszx"][0])) < 5e-4


def test_stage2_weighted_mean_brute_force(orc, rng):
    """Section V-A: sum_i q_i = sum_i (S_b - i + 1) p_i inside each block (pure Python)."""
    for S in (1, 2, 3, 5, 8):
        n = int(rng.integers(1, 30))
        q = rng.integers(-50, 50, n).astype(np.int32)
        dp = []
        for first in range(0, n, S):
            blk = [int(v) for v in q[first:first + S]]
            dp += [blk[0]] + [blk[k] - blk[k - 1] for k in range(1, len(blk))]
        dp = np.array(dp, np.int32)
        assert orc.mean_p_sum(dp, S) == sum(int(v) for v in q)
        s1, s2 = orc.var_p_sums(dp, S)
        assert s1 == sum(int(v) for v in q)
        assert s2 == sum(int(v) ** 2 for v in q)


def test_exact_sums_wide_codes(orc, rng):
    """Sums of q^2 past 2^64 stay exact (128-bit), checked with Python integers."""
    q = rng.integers(-(2**30) + 1, 2**30, 5000).astype(np.int32)
    s1, s2 = orc.sums_q(q)
    assert s1 == sum(int(v) for v in q)
    assert s2 == sum(int(v) ** 2 for v in q)
    assert s2 > 2**64


@pytest.mark.parametrize("n", [2, 3, 17, 1000])
def test_variance_exact_rational(orc, rng, n):
    """finalize() equals the sample variance of d' = 2 eps q in exact arithmetic."""
    q = rng.integers(-3000, 3000, n).astype(np.int32)
    eps = 0.0123
    s1, s2 = orc.sums_q(q)
    mean, var, sd = orc.finalize(n, s1, s2, eps)
    e2 = Fraction(2 * eps)
    d = [e2 * int(v) for v in q]
    mu = sum(d) / n
    v_exact = sum((t - mu) ** 2 for t in d) / (n - 1)
    assert abs(var - float(v_exact)) <= 1e-14 * float(v_exact)
    assert abs(mean - float(mu)) <= 1e-14 * max(abs(float(mu)), float(e2))
    assert sd == math.sqrt(var)


def test_variance_single_element_is_nan(orc):
    mean, var, sd = orc.finalize(1, 5, 25, 0.5)
    assert mean == 5.0 and math.isnan(var) and math.isnan(sd)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_generic_flow_stats_vs_numpy(orc, rng, dtype):
    x = (rng.standard_normal(100000) + 7.0).astype(dtype)
    m, v = orc.stats_f(x)
    xd = x.astype(np.float64)
    assert abs(m - xd.mean()) <= 1e-13 * abs(xd.mean())
    assert abs(v - xd.var(ddof=1)) <= 1e-12 * xd.var(ddof=1)


@pytest.mark.parametrize("dtype,rtol", [(np.float64, 1e-12), (np.float32, 1e-6)])
def test_homomorphic_stats_equal_generic_flow(orc, rng, dtype, rtol):
    """Section V-D: stage-2/3 mean and std equal the D_f result up to float rounding."""
    import synth

    x = synth.sinusoid_field((24, 20, 18), dtype=dtype)
    s, eps = orc.compress(x, 1e-3, True, 32)
    q = orc.decode(s, "q")
    mean, var, _ = orc.finalize(q.size, *orc.sums_q(q), eps)
    mf, vf = orc.stats_f(orc.decode(s, "f"))
    assert abs(mean - mf) <= rtol * abs(mf)
    assert abs(var - vf) <= rtol * vf


# --------------------------------------------------------------------- stencils
def _gradient(d, axis):
    if d.shape[axis] < 2:
        return np.zeros_like(d)
    return np.gradient(d, axis=axis, edge_order=1)


@pytest.mark.parametrize("shape", [(7,), (2,), (5, 1), (6, 9), (1, 4, 5), (4, 5, 6), (3, 2, 8)])
def test_stencils_generic_flow_vs_library(orc, rng, shape):
    """Eq. derivatives / Eq. laplacian on D_f equal numpy.gradient(edge_order=1) and
    scipy.ndimage.laplace(mode='nearest')."""
    from scipy import ndimage

    f = rng.standard_normal(shape)
    for ax in range(len(shape)):
        np.testing.assert_allclose(orc.stencil_f(f, orc.KIND_DERIV, ax), _gradient(f, ax), rtol=1e-14, atol=1e-14)
    gm = np.sqrt(sum(_gradient(f, ax) ** 2 for ax in range(len(shape))))
    np.testing.assert_allclose(orc.stencil_f(f, orc.KIND_GRADMAG), gm, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(orc.stencil_f(f, orc.KIND_LAPLACIAN), ndimage.laplace(f, mode="nearest"),
                               rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("shape", [(9,), (6, 9), (4, 5, 6), (2, 3, 1)])
def test_integer_stencils_match_library_on_codes(orc, rng, shape):
    """eps * D and 2 eps * L from integer numerators equal the library stencils of 2 eps q."""
    from scipy import ndimage

    q = rng.integers(-1000, 1000, shape).astype(np.int32)
    eps = 0.05
    d = q.astype(np.float64) * (2 * eps)
    for ax in range(len(shape)):
        np.testing.assert_allclose(orc.deriv_q(q, ax) * eps, _gradient(d, ax), rtol=1e-13, atol=1e-12)
        np.testing.assert_allclose(orc.stencil_q(q, orc.KIND_DERIV, eps, ax), _gradient(d, ax), rtol=1e-13,
                                   atol=1e-12)
    np.testing.assert_allclose(orc.lap_q(q) * 2 * eps, ndimage.laplace(d, mode="nearest"), rtol=1e-13, atol=1e-12)
    gm = np.sqrt(sum(_gradient(d, ax) ** 2 for ax in range(len(shape))))
    np.testing.assert_allclose(orc.stencil_q(q, orc.KIND_GRADMAG, eps), gm, rtol=1e-13, atol=1e-12)


def test_stencil_closed_forms(orc):
    """Linear ramp: constant derivative 2a along its axis, 0 elsewhere, Laplacian 0
    inside; quadratic i^2: interior Laplacian numerator 2; constant field: all zero."""
    n0, n1, n2 = 5, 6, 7
    i0, i1, i2 = np.meshgrid(np.arange(n0), np.arange(n1), np.arange(n2), indexing="ij")
    a = 3
    ramp = (a * i1).astype(np.int32)
    np.testing.assert_array_equal(orc.deriv_q(ramp, 1), np.full(ramp.shape, 2 * a))
    np.testing.assert_array_equal(orc.deriv_q(ramp, 0), 0)
    np.testing.assert_array_equal(orc.deriv_q(ramp, 2), 0)
    L = orc.lap_q(ramp)
    np.testing.assert_array_equal(L[:, 1:-1, :], 0)
    quad = (i2 ** 2).astype(np.int32)
    np.testing.assert_array_equal(orc.lap_q(quad)[:, :, 1:-1], 2)
    const = np.full((4, 4, 4), 17, np.int32)
    assert not orc.lap_q(const).any()
    assert not orc.deriv_q(const, 2).any()
    # a one-sided edge is twice the forward difference: D = 2 (q1 - q0)
    line = np.array([0, 5, 6, 20], np.int32)
    np.testing.assert_array_equal(orc.deriv_q(line, 0), [10, 6, 15, 28])


@pytest.mark.parametrize("shape,S", [((13, 17, 19), 32), ((40, 33), 16), ((200,), 7), ((5, 6, 70), 64)])
def test_homomorphic_stencils_equal_generic_flow(orc, rng, shape, S):
    """Section V-D: derivative/Laplacian from codes equal the D_f result up to rounding."""
    import synth

    x = synth.sinusoid_field(shape, dtype=np.float64)
    s, eps = orc.compress(x, 1e-3, True, S)
    q = orc.decode(s, "q")
    f = orc.decode(s, "f")
    for kind in (orc.KIND_DERIV, orc.KIND_GRADMAG, orc.KIND_LAPLACIAN):
        for ax in range(len(shape) if kind == orc.KIND_DERIV else 1):
            hq = orc.stencil_q(q, kind, eps, ax)
            hf = orc.stencil_f(f, kind, ax)
            np.testing.assert_allclose(hq, hf, rtol=1e-12, atol=1e-12 * eps)


def test_sampled_stencils_equal_whole_field(orc, rng):
    """stencil_at evaluates the same numerators and values as the whole-field routines."""
    q = rng.integers(-500, 500, (6, 7, 9)).astype(np.int32)
    idx = np.concatenate([[0, q.size - 1], rng.integers(0, q.size, 50)])
    eps = 0.01
    for ax in range(3):
        num, val = orc.stencil_at(q, orc.KIND_DERIV, eps, idx, ax)
        np.testing.assert_array_equal(num, orc.deriv_q(q, ax).reshape(-1)[idx])
        np.testing.assert_array_equal(val, orc.stencil_q(q, orc.KIND_DERIV, eps, ax).reshape(-1)[idx])
    num, val = orc.stencil_at(q, orc.KIND_LAPLACIAN, eps, idx)
    np.testing.assert_array_equal(num, orc.lap_q(q).reshape(-1)[idx])
    np.testing.assert_array_equal(val, orc.stencil_q(q, orc.KIND_LAPLACIAN, eps).reshape(-1)[idx])
    _, val = orc.stencil_at(q, orc.KIND_GRADMAG, eps, idx)
    np.testing.assert_array_equal(val, orc.stencil_q(q, orc.KIND_GRADMAG, eps).reshape(-1)[idx])


# ------------------------------------------------------------ HSZx (block mean)
def _nearest_tie_zero(a, d):
    """Integer nearest to a / d, ties toward zero (Python integers)."""
    f = Fraction(a, d)
    r = math.floor(abs(f) + Fraction(1, 2))
    if abs(f) - math.floor(abs(f)) == Fraction(1, 2):
        r = math.floor(abs(f))
    return r if a >= 0 else -r


def test_hszx_worked_example(orc):
    """Section IV's HSZx example: 2x2 blocks of the printed Y_q give the block
    means M = 5, -1 and the printed Y_p; Section V-A's stage-2 standard
    deviation about the integer mean round(16/8) = 2 is 2.000.  The two 2x2
    blocks, taken in block order, are blocks of 4 consecutive codes."""
    g = read_golden_table("worked_example.txt")
    Yq = np.array([int(v) for v in g["Yq"]], np.int64).reshape(2, 4)
    Yp = np.array([int(v) for v in g["Yp"]], np.int64).reshape(2, 4)
    M = [int(v) for v in g["M"]]
    blocks = lambda a: np.concatenate([a[:, 0:2].reshape(-1), a[:, 2:4].reshape(-1)])  # noqa: E731
    qb = blocks(Yq).astype(np.int32)
    s = orc.compress_codes(qb, 0.1, 4, np.float64, pred=1)
    assert orc.read_header(s)["pred"] == 1
    np.testing.assert_array_equal(orc.decode(s, "m"), M)
    np.testing.assert_array_equal(orc.decode(s, "p"), blocks(Yp))
    np.testing.assert_array_equal(orc.decode(s, "q"), qb)
    dp = orc.decode(s, "p")
    # stage 1 (Eq. mean_m) and stage 2 means
    assert orc.mean_m_sum(np.array(M, np.int32), 4, 8) == 5 * 4 + (-1) * 4
    assert orc.mean_p_sum_x(dp, np.array(M, np.int32), 4) == int(Yq.sum()) == 18
    mt, ss, sigma = orc.std_p_x(dp, np.array(M, np.int32), 4, 0.1)
    assert mt == 2 and ss == 700  # sum (q - 2)^2 over the printed codes
    assert abs(sigma - 2.0) < 1e-15
    assert f"{sigma:.3f}" == g["sigma_p_hszx"][0]


def test_hszx_block_mean_rounding(orc):
    """Block means: nearest integer, ties toward zero, over the true block size
    (a short last block uses its own size)."""
    q = np.array([-1, -1, -1, -2,   3, 3, 3, 4,   2, 3, 2, 3,   -2, -3, -2, -3,   1, 2], np.int32)
    s = orc.compress_codes(q, 1.0, 4, np.float32, pred=1)
    M = orc.decode(s, "m")
    # -5/4 -> -1; 13/4 -> 3; 10/4 = 2.5 -> 2; -10/4 = -2.5 -> -2; 3/2 = 1.5 -> 1
    np.testing.assert_array_equal(M, [-1, 3, 2, -2, 1])
    for b, (lo, hi) in enumerate([(0, 4), (4, 8), (8, 12), (12, 16), (16, 18)]):
        assert M[b] == _nearest_tie_zero(int(q[lo:hi].astype(np.int64).sum()), hi - lo)
    np.testing.assert_array_equal(orc.decode(s, "p"), q - np.repeat(M, [4, 4, 4, 4, 2]))


@pytest.mark.parametrize("sign", [1, -1])
def test_hszx_mu_tilde_rounds_to_nearest(orc, sign):
    """The integer mean mu~ of Section V-A's stage-2 deviation is the nearest
    integer to T / N (T = sum M_b S_b), not its truncation: block means
    3, 3, 2 over 12 codes give T / N = 32 / 12 = 2.67 -> mu~ = 3 and
    sum (q - 3)^2 = 4 (truncation would give mu~ = 2 and 8).  The same
    codes as one 3x4 field in 1x4 boxes give the same under HSZx-nd."""
    q = (sign * np.array([3, 3, 3, 3, 3, 3, 3, 3, 2, 2, 2, 2])).astype(np.int32)
    eps = 0.5
    s = orc.compress_codes(q, eps, 4, np.float64, pred=1)
    dp, M = orc.decode(s, "p"), orc.decode(s, "m")
    np.testing.assert_array_equal(M, sign * np.array([3, 3, 2]))
    assert orc.mean_m_sum(M, 4, 12) == sign * 32
    mt, ss, sigma = orc.std_p_x(dp, M, 4, eps)
    assert (mt, ss) == (sign * 3, 4)
    assert abs(sigma - math.sqrt(4 / 11)) <= 1e-15
    q2 = q.reshape(3, 4)
    s2 = orc.compress_codes_nd(q2, (1, 4), eps)
    dp2, M2 = orc.decode(s2, "p"), orc.decode(s2, "m")
    mt2, ss2, sigma2 = orc.xnd_std_p(dp2, M2, (1, 4), eps)
    assert (mt2, ss2) == (sign * 3, 4)
    assert abs(sigma2 - math.sqrt(4 / 11)) <= 1e-15


@pytest.mark.parametrize("S", SIZES_S)
def test_hszx_roundtrip_and_independent_reader(orc, rng, S):
    """HSZx streams: D_q is the codes exactly, the independent reader agrees,
    M_b follows the rounding rule and the width is the bit length of
    max |q - M_b|; encoding the decoded codes again is the identity."""
    n = int(rng.integers(1, 700))
    x = np.cumsum(rng.standard_normal(n)).astype(np.float32)
    if n > 5:
        x[rng.integers(0, n, 3)] += 50.0
    s, eps = orc.compress(x, 1e-2, True, S, pred=1)
    q_ref = orc.quantize(x, eps)
    np.testing.assert_array_equal(orc.decode(s, "q"), q_ref)
    q_py, widths = _py_decode(s)
    np.testing.assert_array_equal(q_py, q_ref)
    M = orc.decode(s, "m")
    for b in range(widths.size):
        blk = q_ref[b * S:(b + 1) * S].astype(np.int64)
        assert M[b] == _nearest_tie_zero(int(blk.sum()), blk.size)
        assert widths[b] == int(np.abs(blk - M[b]).max()).bit_length()
    s2 = orc.compress_codes(q_ref, eps, S, np.float32, eb=1e-2, rel=True, pred=1)
    assert bytes(s2) == bytes(s)
    # the same codes under the delta predictor: same header except byte 140
    s0, _ = orc.compress(x, 1e-2, True, S)
    assert orc.read_header(s0)["pred"] == 0


@pytest.mark.parametrize("S", [1, 4, 32, 100])
def test_hszx_statistics_stage_forms(orc, rng, S):
    """Stage 2 mean = exact sum q; stage 1 mean within eps of it (Section V-D:
    |r_b| <= 1/2 per block); stage 2 sigma about mu~ equals the exact rational
    value sum (q - mu~)^2 / (N - 1) and stays within the Section V-D bound
    of the exact sample standard deviation."""
    n = int(rng.integers(2, 3000))
    x = (np.cumsum(rng.standard_normal(n)) * 3).astype(np.float64)
    s, eps = orc.compress(x, 1e-3, True, S, pred=1)
    q = orc.decode(s, "q").astype(np.int64)
    dp = orc.decode(s, "p")
    M = orc.decode(s, "m")
    s1 = int(q.sum())
    assert orc.mean_p_sum_x(dp, M, S) == s1
    T = orc.mean_m_sum(M, S, n)
    assert abs(Fraction(T, n) - Fraction(s1, n)) <= Fraction(1, 2)
    mu1 = T / n * 2 * eps
    assert abs(mu1 - s1 / n * 2 * eps) <= eps * (1 + 1e-12)
    mt, ss, sigma = orc.std_p_x(dp, M, S, eps)
    assert mt == _nearest_tie_zero(T, n)
    assert ss == int(((q - mt) ** 2).sum())
    assert abs(sigma - math.sqrt(ss / (n - 1)) * 2 * eps) <= 1e-12 * sigma + 1e-300
    s2 = int((q * q).sum())
    _, var, sd = orc.finalize(n, s1, s2, eps)
    assert abs(sigma - sd) <= 2 * eps * (math.sqrt(n / (n - 1)) * 0.5 + 0.5) + 1e-12


# ------------------------------------------------------- divergence and curl
@pytest.mark.parametrize("shape", [(9, 11), (5, 6, 7), (2, 40), (1, 8, 3)])
def test_divergence_equals_library_gradients(orc, rng, shape):
    """Section V-C: the divergence is the sum of each component's derivative
    along its own axis; on D_f = 2 eps q it equals numpy.gradient (first-order
    edges) summed over the components, with a common or a per-component eps."""
    qs = [rng.integers(-500, 500, size=shape).astype(np.int32) for _ in shape]
    for eps in ([0.01] * len(shape), [0.01 * (c + 1) for c in range(len(shape))]):
        num, val = orc.divergence_q(qs, eps)
        ref = np.zeros(shape)
        ref_num = np.zeros(shape, np.int64)
        for c, q in enumerate(qs):
            g = np.zeros(shape) if shape[c] < 2 else np.gradient(q.astype(np.float64) * 2 * eps[c], axis=c, edge_order=1)
            ref += g
            ref_num += orc.deriv_q(q, c)
        np.testing.assert_array_equal(num, ref_num)
        np.testing.assert_allclose(val, ref, rtol=1e-12, atol=1e-12)
        if len(set(eps)) == 1:
            np.testing.assert_array_equal(val, num.astype(np.float64) * eps[0])


def test_divergence_and_curl_closed_forms(orc):
    """u = a i, v = b j (codes): divergence 2 (a + b) eps everywhere (centred
    and one-sided differences are exact on linear fields) and curl 0; u = c j,
    v = d i: curl 2 (c - d) eps and divergence 0."""
    n1, n2 = 7, 9
    i = np.arange(n1)[:, None] * np.ones((1, n2), np.int64)
    j = np.ones((n1, 1), np.int64) * np.arange(n2)[None, :]
    a, b, c, d = 3, -5, 4, 7
    num, val = orc.divergence_q([(a * i).astype(np.int32), (b * j).astype(np.int32)], [0.5, 0.5])
    assert np.all(num == 2 * (a + b)) and np.all(val == 2 * (a + b) * 0.5)
    num, val = orc.curl2_q((a * i).astype(np.int32), (b * j).astype(np.int32), 0.5, 0.5)
    assert np.all(num == 0)
    num, val = orc.curl2_q((c * j).astype(np.int32), (d * i).astype(np.int32), 0.5, 0.5)
    assert np.all(num == 2 * (c - d)) and np.all(val == 2 * (c - d) * 0.5)
    num, val = orc.divergence_q([(c * j).astype(np.int32), (d * i).astype(np.int32)], [0.5, 0.5])
    assert np.all(num == 0)


def test_curl_equals_library_gradients(orc, rng):
    qu = rng.integers(-300, 300, size=(12, 10)).astype(np.int32)
    qv = rng.integers(-300, 300, size=(12, 10)).astype(np.int32)
    for eu, ev in ((0.02, 0.02), (0.02, 0.07)):
        num, val = orc.curl2_q(qu, qv, eu, ev)
        ref = np.gradient(qu * 2 * eu, axis=1, edge_order=1) - np.gradient(qv * 2 * ev, axis=0, edge_order=1)
        np.testing.assert_allclose(val, ref, rtol=1e-12, atol=1e-12)
        np.testing.assert_array_equal(num, orc.deriv_q(qu, 1) - orc.deriv_q(qv, 0))


# ------------------------------------------ global predictors (HSZp-nd, HSZp)
GLOBAL_SHAPES = [(1,), (7,), (300,), (5, 9), (33, 40), (1, 6), (4, 6, 7), (1, 5, 3), (2, 1, 9), (3, 4, 1),
                 (9, 10, 11)]


def _residuals_numpy(q, pred):
    """Backward differences with a zero before the field (numpy.diff): along
    every axis for the Lorenzo predictor, over the flattened field for HSZp."""
    r = q.astype(np.int64)
    if pred == 3:
        return np.diff(r.ravel(), prepend=0).reshape(q.shape)
    for a in range(q.ndim):
        r = np.diff(r, axis=a, prepend=0)
    return r


def _smooth_codes(rng, shape, scale=400):
    x = rng.standard_normal(shape)
    for a in range(len(shape)):
        x = np.cumsum(x, axis=a)
    return (x * scale / max(1.0, np.abs(x).max()) + rng.integers(-3, 4, size=shape)).astype(np.int32)


@pytest.mark.parametrize("pred", [2, 3])
@pytest.mark.parametrize("shape", GLOBAL_SHAPES)
def test_global_predictor_residuals_and_roundtrip(orc, rng, pred, shape):
    """Section IV, HSZp and HSZp-nd: D_p is the backward difference across
    block boundaries (numpy.diff), D_q returns the codes, the independent
    reader rebuilds them with numpy.cumsum, each width is the bit length of
    the block's largest |p|, heads are zero and there is no stage 1."""
    q = _smooth_codes(rng, shape)
    for S in (32, 7, 64):
        s = orc.compress_codes(q, 0.01, S, pred=pred)
        assert orc.read_header(s)["pred"] == pred
        p_ref = _residuals_numpy(q, pred)
        np.testing.assert_array_equal(orc.decode(s, "p"), p_ref)
        np.testing.assert_array_equal(orc.decode(s, "q"), q)
        q_py, widths = _py_decode(s)
        np.testing.assert_array_equal(q_py.reshape(shape), q)
        flat = np.abs(p_ref.ravel())
        for b in range(widths.size):
            assert widths[b] == int(flat[b * S:(b + 1) * S].max()).bit_length()
        with pytest.raises(orc.OracleError) as e:
            orc.decode(s, "m")
        assert e.value.status == 4


def test_global_predictor_hand_example(orc):
    """A 2x3 field worked by hand: the 2-D Lorenzo residuals are
    [[1, 2, 3], [1, 1, 1]] (row 1: 2-1, 5-2-3+1, 9-5-6+3) and the flattened
    HSZp residuals are [1, 2, 3, -4, 3, 4]."""
    q = np.array([[1, 3, 6], [2, 5, 9]], np.int32)
    s2 = orc.compress_codes(q, 0.5, 4, pred=2)
    np.testing.assert_array_equal(orc.decode(s2, "p"), [[1, 2, 3], [1, 1, 1]])
    s3 = orc.compress_codes(q, 0.5, 4, pred=3)
    np.testing.assert_array_equal(orc.decode(s3, "p").ravel(), [1, 2, 3, -4, 3, 4])
    # mean on D_p: weights (n1 - i)(n2 - j) = [[6, 4, 2], [3, 2, 1]] for the 2-D form
    assert orc.lorenzo_mean_p(orc.decode(s2, "p"), 2) == 6 + 8 + 6 + 3 + 2 + 1 == int(q.sum())
    assert orc.lorenzo_mean_p(orc.decode(s3, "p"), 3) == 6 * 1 + 5 * 2 + 4 * 3 - 3 * 4 + 2 * 3 + 1 * 4


def test_global_predictor_residual_range(orc):
    """A residual must fit the encoder's 31-bit magnitude: a checkerboard of
    +-A codes has 3-D Lorenzo residuals of magnitude 8 A inside the field."""
    z, y, x = np.meshgrid(np.arange(3), np.arange(3), np.arange(3), indexing="ij")
    sign = 1 - 2 * ((x + y + z) % 2)
    ok = (sign * (2**28 - 1)).astype(np.int32)
    s = orc.compress_codes(ok, 1.0, 32, pred=2)
    assert int(np.abs(orc.decode(s, "p")).max()) == 8 * (2**28 - 1)
    np.testing.assert_array_equal(orc.decode(s, "q"), ok)
    with pytest.raises(orc.OracleError) as e:
        orc.compress_codes((sign * 2**28).astype(np.int32), 1.0, 32, pred=2)
    assert e.value.status == 2


def _box_weights(shape):
    """Brute force: the number of codes whose box [0..i] contains position j."""
    w = np.zeros(shape, np.int64)
    for j in np.ndindex(*shape):
        w[j] = int(np.prod([n - c for n, c in zip(shape, j)]))
    return w


@pytest.mark.parametrize("pred", [2, 3])
@pytest.mark.parametrize("shape", [(1,), (17,), (5, 9), (4, 6, 7), (2, 1, 9), (9, 10, 11)])
def test_global_predictor_stage2_statistics(orc, rng, pred, shape):
    """Section V-A on D_p: the weighted sum equals sum q, the Algorithm 4
    accumulators equal (sum q, sum q^2) exactly, and the weights are the
    brute-force box counts."""
    q = _smooth_codes(rng, shape, scale=3000)
    s = orc.compress_codes(q, 0.01, 32, pred=pred)
    dp = orc.decode(s, "p")
    qi = [int(v) for v in q.ravel()]
    assert orc.lorenzo_mean_p(dp, pred) == sum(qi)
    s1, s2 = orc.lorenzo_var_p(dp, pred)
    assert s1 == sum(qi) and s2 == sum(v * v for v in qi)
    wshape = shape if pred == 2 else (q.size,)
    w = _box_weights(wshape)
    assert int((w.ravel() * dp.ravel().astype(np.int64)).sum()) == sum(qi)


@pytest.mark.parametrize("shape", [(9,), (2,), (5, 9), (2, 7), (4, 6, 7), (1, 5, 3), (2, 1, 9), (3, 4, 2),
                                   (8, 9, 10)])
def test_lorenzo_stage2_derivative_equals_library_gradient(orc, rng, shape):
    """Section V-B on D_p (Eq. derivative_Dp and its box-sum form): the
    numerators equal 2 numpy.gradient of the codes (one-sided edges); an
    axis of length 1 gives 0."""
    q = _smooth_codes(rng, shape, scale=2000)
    dp = orc.decode(orc.compress_codes(q, 0.01, 32, pred=2), "p")
    for a in range(q.ndim):
        D = orc.lorenzo_deriv_p(dp, a)
        if shape[a] == 1:
            assert not D.any()
            continue
        g = 2 * np.gradient(q.astype(np.float64), axis=a)
        np.testing.assert_array_equal(D, g.astype(np.int64))
        np.testing.assert_array_equal(D, orc.deriv_q(q, a))


@pytest.mark.parametrize("shape", [(9,), (2,), (1,), (5, 9), (2, 7), (4, 6, 7), (1, 5, 3), (2, 1, 9),
                                   (8, 9, 10)])
def test_lorenzo_stage2_laplacian_equals_library(orc, rng, shape):
    """Section V-B on D_p (Eq. laplacian_Dp, the xi prefix sums): the
    numerators equal scipy.ndimage.laplace on the codes with replicated
    edges."""
    from scipy import ndimage

    q = _smooth_codes(rng, shape, scale=2000)
    dp = orc.decode(orc.compress_codes(q, 0.01, 32, pred=2), "p")
    L = orc.lorenzo_lap_p(dp)
    ref = ndimage.laplace(q.astype(np.float64), mode="nearest")
    np.testing.assert_array_equal(L, ref.astype(np.int64))
    np.testing.assert_array_equal(L, orc.lap_q(q))


# ------------------------------------------------------- HSZx-nd (boxes of codes)
def test_hszx_nd_worked_example(orc):
    """Section IV's HSZx-nd example as printed: the 2x4 codes Y_q in 2x2 boxes
    give the box means M = 5, -1 and the printed 2x4 Y_p; Section V-A's
    stage-2 standard deviation about round(16/8) = 2 is 2.000."""
    g = read_golden_table("worked_example.txt")
    Yq = np.array([int(v) for v in g["Yq"]], np.int32).reshape(2, 4)
    Yp = np.array([int(v) for v in g["Yp"]], np.int64).reshape(2, 4)
    M = [int(v) for v in g["M"]]
    s = orc.compress_codes_nd(Yq, (2, 2), 0.1, np.float64)
    h = orc.read_header(s)
    assert (h["pred"], h["block"], h["nb"], h["S"]) == (4, (2, 2), 2, 4)
    np.testing.assert_array_equal(orc.decode(s, "m"), M)
    np.testing.assert_array_equal(orc.decode(s, "p"), Yp)
    np.testing.assert_array_equal(orc.decode(s, "q"), Yq)
    dp, Mv = orc.decode(s, "p"), orc.decode(s, "m")
    assert orc.xnd_mean_m(Mv, (2, 4), (2, 2)) == 5 * 4 + (-1) * 4
    assert orc.xnd_mean_p(dp, Mv, (2, 2)) == int(Yq.sum()) == 18
    mt, ss, sigma = orc.xnd_std_p(dp, Mv, (2, 2), 0.1)
    assert (mt, ss) == (2, 700)
    assert f"{sigma:.3f}" == g["sigma_p_hszx"][0]
    q_py, _ = _py_decode(s)
    np.testing.assert_array_equal(q_py.reshape(2, 4), Yq)


ND_CASES = [((7, 10), (2, 3)), ((5, 6, 7), (2, 2, 4)), ((9,), (4,)), ((3, 8, 9), (1, 4, 8)),
            ((4, 5, 6), (8, 8, 8)), ((13, 17, 19), (4, 4, 4)), ((1, 33, 40), (1, 8, 8)), ((50, 3), (16, 4))]


@pytest.mark.parametrize("shape,block", ND_CASES)
def test_hszx_nd_roundtrip_and_reader(orc, rng, shape, block):
    """Boxes cut by the field's end: D_q is the codes, the independent reader
    (box slots back to field positions) agrees, each box mean follows the
    rounding rule over the true box size, each width is the bit length of
    the box's largest |q - M_b|."""
    q = _smooth_codes(rng, shape, scale=900)
    s = orc.compress_codes_nd(q, block, 0.01)
    np.testing.assert_array_equal(orc.decode(s, "q"), q)
    q_py, widths = _py_decode(s)
    np.testing.assert_array_equal(q_py.reshape(shape), q)
    M = orc.decode(s, "m")
    d = (1,) * (3 - len(shape)) + shape
    bd = (1,) * (3 - len(block)) + block
    q3 = q.reshape(d).astype(np.int64)
    g = [-(-d[a] // bd[a]) for a in range(3)]
    assert M.size == widths.size == g[0] * g[1] * g[2]
    b = 0
    for k0 in range(g[0]):
        for k1 in range(g[1]):
            for k2 in range(g[2]):
                box = q3[k0 * bd[0]:(k0 + 1) * bd[0], k1 * bd[1]:(k1 + 1) * bd[1], k2 * bd[2]:(k2 + 1) * bd[2]]
                assert M[b] == _nearest_tie_zero(int(box.sum()), box.size)
                assert widths[b] == int(np.abs(box - M[b]).max()).bit_length()
                b += 1
    np.testing.assert_array_equal(orc.decode(s, "p").reshape(d),
                                  q3 - np.repeat(np.repeat(np.repeat(M.reshape(g), bd[0], 0), bd[1], 1), bd[2], 2)
                                  [: d[0], : d[1], : d[2]])


@pytest.mark.parametrize("S", [1, 7, 32, 100])
def test_hszx_nd_one_axis_equals_hszx(orc, rng, S):
    """Boxes along one axis are HSZx's 1-D blocks: the same widths, means
    and payload; only the predictor byte and the box extents differ."""
    q = _smooth_codes(rng, (1000,), scale=700)
    a = orc.compress_codes(q, 0.01, S, pred=1)
    b = orc.compress_codes_nd(q, (S,), 0.01)
    assert a.size == b.size
    diff = np.nonzero(a != b)[0]
    assert diff.size and diff.min() >= 140 and diff.max() < 156


@pytest.mark.parametrize("shape,block", ND_CASES)
def test_hszx_nd_statistics(orc, rng, shape, block):
    """Section V-A on boxes: the stage-1 sum uses the true box sizes (brute
    force), the stage-2 sum is sum q exactly, the stage-2 deviation is the
    exact sum of (q - mu~)^2 (numpy), and the stage-1 mean is within eps of
    the exact mean (Section V-D)."""
    q = _smooth_codes(rng, shape, scale=5000)
    eps = 0.01
    s = orc.compress_codes_nd(q, block, eps)
    dp, M = orc.decode(s, "p"), orc.decode(s, "m")
    d = (1,) * (3 - len(shape)) + shape
    bd = (1,) * (3 - len(block)) + block
    g = [-(-d[a] // bd[a]) for a in range(3)]
    sizes = [min(bd[0], d[0] - k0 * bd[0]) * min(bd[1], d[1] - k1 * bd[1]) * min(bd[2], d[2] - k2 * bd[2])
             for k0 in range(g[0]) for k1 in range(g[1]) for k2 in range(g[2])]
    T = orc.xnd_mean_m(M, shape, block)
    assert T == sum(int(m) * n for m, n in zip(M, sizes))
    assert orc.xnd_mean_p(dp, M, block) == int(q.astype(np.int64).sum())
    mt, ss, sigma = orc.xnd_std_p(dp, M, block, eps)
    assert mt == _nearest_tie_zero(T, q.size)
    assert ss == sum((int(v) - mt) ** 2 for v in q.ravel())
    assert abs(T / q.size - q.astype(np.int64).sum() / q.size) * 2 * eps <= eps


@pytest.mark.parametrize("shape,block", ND_CASES)
def test_hszx_nd_stage2_stencils_equal_library(orc, rng, shape, block):
    """Section V-B's HSZx-2d stage-2 formulas (p differences plus the box
    means' difference at box borders), for every axis: the derivative
    numerators equal 2 numpy.gradient of the codes and the Laplacian
    numerators scipy.ndimage.laplace with replicated edges."""
    from scipy import ndimage

    q = _smooth_codes(rng, shape, scale=3000)
    s = orc.compress_codes_nd(q, block, 0.01)
    dp, M = orc.decode(s, "p"), orc.decode(s, "m")
    for a in range(q.ndim):
        D = orc.xnd_deriv_p(dp, M, block, a)
        if shape[a] == 1:
            assert not D.any()
            continue
        np.testing.assert_array_equal(D, (2 * np.gradient(q.astype(np.float64), axis=a)).astype(np.int64))
    L = orc.xnd_lap_p(dp, M, block)
    np.testing.assert_array_equal(L, ndimage.laplace(q.astype(np.float64), mode="nearest").astype(np.int64))
