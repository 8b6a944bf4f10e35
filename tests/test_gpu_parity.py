"""CUDA path vs the CPU oracle, through the C ABI (needs a GPU).

Bars (stated once, used everywhere):
* stream bytes, widths, heads, chunk index, D_p, D_q, the exact sums s1 and
  s2, and the integer stencil numerators: bit-exact;
* D_f: bit-exact (the same float arithmetic on both sides);
* mean / variance / std from integer stages: relative 1e-12 (the final
  scaling is the same double arithmetic, so equality is expected);
* float32 stencil fields: |gpu - oracle| <= 1e-6 * max(|oracle|, s) with s = eps
  for derivatives and the gradient magnitude and 2 eps for the Laplacian
  (any nonzero integer numerator is at least that large); float64 fields 1e-12;
* the plain path (statistics and stencils of a float array) computes in the
  field's own precision: relative 1e-5 (float32) / 1e-12 (float64) against
  the oracle's generic flow, plus a few float32 ulps of the field's magnitude
  for the Laplacian's cancellation.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

RTOL_STAT = 1e-12
RTOL_F32 = 1e-6
RTOL_F64 = 1e-12


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2603_25206_gb300 import hc

    hc.lib()
    return hc, torch, torch.device("cuda:0")


def _cases():
    import synth

    r = np.random.default_rng(7)
    yield "pr1_64cubed", synth.sinusoid_field((64, 64, 64)), 1e-3, True, 32
    yield "grf_ragged_3d", synth.grf_field((13, 17, 19), 11), 1e-3, True, 32
    yield "grf_2d_S16", synth.grf_field((40, 33), 12), 1e-2, True, 16
    yield "walk_1d_S7", np.cumsum(r.standard_normal(1000)).astype(np.float32), 1e-2, True, 7
    # rows too long for a whole-row tile of the general kernel, one row per slab
    # (a 1-D field; a 2-D field walked as (n1, 1, n2)): split along x
    yield "walk_1d_long_S16", np.cumsum(r.standard_normal(60001)).astype(np.float32), 1e-3, True, 16
    yield "rows_2d_long_S64", synth.grf_field((3, 70000), 28), 1e-3, True, 64
    yield "grf_S64", synth.grf_field((5, 6, 70), 13), 1e-4, True, 64
    yield "grf_S100", synth.grf_field((9, 10, 31), 14), 1e-3, True, 100
    yield "grf_S128_f64", synth.grf_field((7, 9, 40), 15, dtype=np.float64), 1e-3, True, 128
    yield "S1", synth.grf_field((3, 4, 5), 16), 1e-3, True, 1
    yield "S3", synth.grf_field((4, 6, 7), 17), 1e-3, True, 3
    yield "S4096", synth.grf_field((2, 50, 90), 18), 1e-3, True, 4096
    yield "single", np.array([0.25], np.float32), 1e-3, False, 32
    yield "constant", np.full((8, 9, 10), 3.5, np.float32), 1e-3, True, 32
    yield "two_point_axis", synth.grf_field((2, 3, 40), 19), 1e-3, True, 32
    # a 3-D field whose first axis has length 1 (walked as (n1, 1, n2))
    yield "leading_len1_S32", synth.grf_field((1, 12, 40), 29), 1e-3, True, 32
    yield "leading_len1_S16", synth.grf_field((1, 9, 30), 30), 1e-3, True, 16
    # shapes the pipelined stencil kernel takes (S = 32, rows of a multiple of 8)
    yield "pipe_ragged_3d", synth.grf_field((7, 13, 40), 24), 1e-3, True, 32
    yield "pipe_2d", synth.grf_field((33, 24), 25), 1e-3, True, 32
    yield "pipe_2planes", synth.grf_field((2, 9, 16), 26), 1e-4, True, 32
    yield "pipe_tall", synth.grf_field((40, 70, 8), 27), 1e-2, True, 32
    yield "wide_f64", synth.wide_field((8, 16, 64), 20), 1e-6, True, 64
    x = r.standard_normal((6, 7, 8)).astype(np.float64)
    rng_ = float(x.max() - x.min())
    yield "widest_abs", (x - (x.max() + x.min()) / 2), rng_ / 2**31, False, 32


CASES = list(_cases())


def _close(got, ref, rtol, floor):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    bound = rtol * np.maximum(np.abs(ref), floor)
    bad = np.abs(got - ref) > bound
    assert not bad.any(), f"{bad.sum()} of {bad.size} outside tolerance; worst {np.abs(got - ref)[bad].max()}"


@pytest.mark.parametrize("name,x,eb,rel,S", CASES, ids=[c[0] for c in CASES])
def test_parity(env, orc, name, x, eb, rel, S):
    hc, torch, dev = env
    ref_stream, eps = orc.compress(x, eb, rel, S)
    xd = torch.from_numpy(np.ascontiguousarray(x)).to(dev)

    # compression: the whole stream bit for bit
    c = hc.compress(xd, eb, rel=rel, S=S)
    assert c.nbytes == ref_stream.size
    assert np.array_equal(c.stream[: c.nbytes].cpu().numpy(), ref_stream)
    assert c.eps == eps
    # a stream written by the oracle decodes the same way
    c2 = hc.from_stream(torch.from_numpy(ref_stream).to(dev))
    assert c2.header.N == x.size

    # decompression to every stage
    q = orc.decode(ref_stream, "q")
    for stage in ("m", "p", "q", "f"):
        got = hc.decompress(c2, stage).cpu().numpy()
        assert np.array_equal(got, orc.decode(ref_stream, stage)), stage
    assert hc.workspace_status() == 0

    # statistics: fused at stage 2 and 3, and on materialized P / Q
    s1, s2 = orc.sums_q(q)
    m_ref, v_ref, sd_ref = orc.finalize(q.size, s1, s2, eps)
    dp = hc.decompress(c2, "p")
    dq = hc.decompress(c2, "q")
    inputs = [("fused_p", c2, "p"), ("fused_q", c2, "q"), ("arr_p", hc.as_stage(c2, "p", dp), None),
              ("arr_q", hc.as_stage(c2, "q", dq), None)]
    for tag, inp, level in inputs:
        rm = hc.parse_scalar(hc.mean(inp, level=level or "p"))
        assert rm["status"] == 0 and rm["exact"] == 1, tag
        assert rm["s1"] == s1, tag
        assert abs(rm["mean"] - m_ref) <= RTOL_STAT * max(abs(m_ref), 2 * eps), tag
        rv = hc.parse_scalar(hc.variance(inp, level=level or "q"))
        assert rv["s1"] == s1 and rv["s2"] == s2, tag
        if q.size > 1:
            assert abs(rv["variance"] - v_ref) <= RTOL_STAT * max(abs(v_ref), (2 * eps) ** 2), tag
            assert abs(rv["std"] - sd_ref) <= RTOL_STAT * max(abs(sd_ref), 2 * eps), tag
        else:
            assert np.isnan(rv["variance"])
    # plain path: float statistics of D_f
    df = hc.decompress(c2, "f")
    mf, vf = orc.stats_f(orc.decode(ref_stream, "f"))
    rf = hc.parse_scalar(hc.variance(hc.as_stage(c2, "f", df)))
    tol = 1e-12 if x.dtype == np.float64 else 1e-5
    assert abs(rf["mean"] - mf) <= tol * max(abs(mf), 2 * eps)
    if q.size > 1:
        assert abs(rf["variance"] - vf) <= tol * max(vf, (2 * eps) ** 2) + 1e-7 * abs(mf) * (2 * eps)

    # stencils: fused (stream) and on a materialized D_q, integer and float outputs
    nd = x.ndim
    ops = [("d", a) for a in range(nd)] + [("g", 0), ("l", 0)]
    f_ref = orc.decode(ref_stream, "f")
    for op, ax in ops:
        kind = {"d": orc.KIND_DERIV, "g": orc.KIND_GRADMAG, "l": orc.KIND_LAPLACIAN}[op]
        val_ref = orc.stencil_q(q, kind, eps, ax)
        floor = 2 * eps if op == "l" else eps
        for tag, inp in (("fused", c2), ("arr_q", hc.as_stage(c2, "q", dq))):
            call = {"d": lambda **k: hc.derivative(inp, ax, **k), "g": lambda **k: hc.gradmag(inp, **k),
                    "l": lambda **k: hc.laplacian(inp, **k)}[op]
            if op != "g":
                num = call(out_dtype="int64").cpu().numpy()
                num_ref = orc.deriv_q(q, ax) if op == "d" else orc.lap_q(q)
                assert np.array_equal(num, num_ref), (tag, op, ax)
            _close(call(out_dtype="float32").cpu().numpy(), val_ref, RTOL_F32, floor)
            _close(call(out_dtype="float64").cpu().numpy(), val_ref, RTOL_F64, floor)
        # plain path on D_f
        plain = {"d": lambda: hc.derivative(hc.as_stage(c2, "f", df), ax, out_dtype="float64"),
                 "g": lambda: hc.gradmag(hc.as_stage(c2, "f", df), out_dtype="float64"),
                 "l": lambda: hc.laplacian(hc.as_stage(c2, "f", df), out_dtype="float64")}[op]().cpu().numpy()
        gen = orc.stencil_f(f_ref, kind, ax)
        if x.dtype == np.float64:
            np.testing.assert_allclose(plain, gen, rtol=1e-12, atol=1e-12 * max(1.0, float(np.abs(f_ref).max())))
        else:
            ulp = float(np.spacing(np.float32(np.abs(f_ref).max() + 1e-30)))
            np.testing.assert_allclose(plain, gen, rtol=1e-5, atol=16 * ulp)
    assert hc.workspace_status() == 0


def test_stage2_differentiation_unsupported(env):
    hc, torch, dev = env
    import synth

    c = hc.compress(torch.from_numpy(synth.grf_field((8, 8, 8), 3)).to(dev), 1e-3)
    with pytest.raises(hc.HcError) as e:
        hc.laplacian(c, level="p")
    assert e.value.status == hc.HC_ERR_UNSUPPORTED
    with pytest.raises(hc.HcError) as e:
        hc.derivative(hc.as_stage(c, "p", hc.decompress(c, "p")), 0)
    assert e.value.status == hc.HC_ERR_UNSUPPORTED


def test_extreme_codes_width_31(env, orc):
    """Codes near +-2^30 with alternating signs: widths 31, q^2 sums past 2^64."""
    hc, torch, dev = env
    r = np.random.default_rng(5)
    q = r.integers(-(2**30) + 1, 2**30, (4, 8, 96)).astype(np.int32)
    q[..., ::2] = 2**30 - 1
    q[..., 1::2] = -(2**30) + 1
    eps = 0.5
    for S in (32, 64):
        ref = orc.compress_codes(q, eps, S)
        c = hc.compress_codes(torch.from_numpy(q).to(dev), eps, S=S)
        assert np.array_equal(c.stream[: c.nbytes].cpu().numpy(), ref)
        assert c.header.wmax == 31
        s1, s2 = orc.sums_q(q)
        r3 = hc.parse_scalar(hc.variance(c))
        assert (r3["s1"], r3["s2"]) == (s1, s2)
        assert s2 > 2**64
        assert r3["exact"] == 1
        lap = hc.laplacian(c, out_dtype="int64").cpu().numpy()
        assert np.array_equal(lap, orc.lap_q(q))
        d = hc.derivative(c, 2, out_dtype="int64").cpu().numpy()
        assert np.array_equal(d, orc.deriv_q(q, 2))


def test_range_error(env):
    hc, torch, dev = env
    x = torch.zeros(100, device=dev)
    x[7] = float("nan")
    with pytest.raises(hc.HcError) as e:
        hc.compress(x, 1e-3)
    assert e.value.status == hc.HC_ERR_RANGE
    x = torch.zeros(100, dtype=torch.float64, device=dev)
    x[3] = 2.0**40
    with pytest.raises(hc.HcError) as e:
        hc.compress(x, 1e-3, rel=False)
    assert e.value.status == hc.HC_ERR_RANGE


def test_corrupt_stream_reported_not_faulting(env, orc):
    """A width byte set above the header's max width: the kernels flag the tile
    and skip it (every read stays inside the stream)."""
    hc, torch, dev = env
    import synth

    x = synth.grf_field((16, 16, 64), 4)
    ref, eps = orc.compress(x, 1e-3, True, 32)
    bad = ref.copy()
    bad[256 + 100] = 31
    c = hc.from_stream(torch.from_numpy(bad).to(dev))
    r = hc.parse_scalar(hc.variance(c))
    assert r["status"] == hc.HC_ERR_CORRUPT
    hc.decompress(c, "q")
    assert hc.workspace_status() == hc.HC_ERR_CORRUPT
    hc.laplacian(c)
    assert hc.workspace_status() == hc.HC_ERR_CORRUPT
    assert hc.workspace_status() == 0
    # a corrupt header is refused on the host
    bad = ref.copy()
    bad[64] ^= 1
    with pytest.raises(hc.HcError) as e:
        hc.from_stream(torch.from_numpy(bad).to(dev))
    assert e.value.status == hc.HC_ERR_CORRUPT


def test_repeat_calls_deterministic(env):
    """Same inputs, same bytes: compression, decoding and every operation run twice."""
    hc, torch, dev = env
    import synth

    xd = torch.from_numpy(synth.grf_field((33, 40, 50), 6)).to(dev)
    a = hc.compress(xd, 1e-3)
    b = hc.compress(xd, 1e-3)
    assert torch.equal(a.stream[: a.nbytes], b.stream[: b.nbytes])
    for fn in (lambda: hc.variance(a), lambda: hc.mean(a), lambda: hc.gradmag(a), lambda: hc.laplacian(a),
               lambda: hc.decompress(a, "f")):
        assert torch.equal(fn(), fn())


def test_side_stream_not_current(env, orc):
    """Operations queued on fresh side streams that are never made torch's
    current stream: each stream's workspace is allocated and zeroed on that
    stream, and the results equal the oracle's exactly."""
    hc, torch, dev = env
    import synth

    x = synth.grf_field((20, 30, 40), 31)
    ref, eps = orc.compress(x, 1e-3, True, 32)
    c = hc.compress(torch.from_numpy(x).to(dev), 1e-3)
    q = orc.decode(ref, "q")
    lap_ref = orc.lap_q(q)
    torch.cuda.synchronize()
    for _ in range(3):
        s = torch.cuda.Stream(device=dev)
        r = hc.variance(c, stream=s)
        lap = hc.laplacian(c, out_dtype="int64", stream=s)
        s.synchronize()
        rs = hc.parse_scalar(r)
        assert (rs["s1"], rs["s2"]) == orc.sums_q(q) and rs["status"] == 0
        assert np.array_equal(lap.cpu().numpy(), lap_ref)


def test_kernel_reuse_across_tile_sizes(env, orc):
    """One kernel launched with large, small, then large shared-memory tiles
    (fields of different row lengths) stays valid and exact."""
    hc, torch, dev = env
    import synth

    fields = [synth.grf_field((4, 300, 900), 21), synth.grf_field((6, 20, 40), 22), synth.grf_field((3, 280, 1100), 23)]
    for x in fields + fields[::-1]:
        ref, eps = orc.compress(x, 1e-3, True, 32)
        c = hc.compress(torch.from_numpy(x).to(dev), 1e-3)
        q = orc.decode(ref, "q")
        assert np.array_equal(hc.laplacian(c, out_dtype="int64").cpu().numpy(), orc.lap_q(q))
        assert np.array_equal(hc.decompress(c, "q").cpu().numpy(), q)
        r = hc.parse_scalar(hc.variance(c))
        assert (r["s1"], r["s2"]) == orc.sums_q(q)


def test_autotune_keeps_results_exact(env, orc):
    """hc_autotune times the fused stencil's tile heights; whatever it keeps,
    the outputs stay bit-exact (integer) and within tolerance (float)."""
    hc, torch, dev = env
    import synth

    x = synth.grf_field((6, 40, 96), 31)
    ref, eps = orc.compress(x, 1e-3, True, 32)
    q = orc.decode(ref, "q")
    c = hc.compress(torch.from_numpy(x).to(dev), 1e-3)
    assert hc.autotune(c, "laplacian", "int64") in (1, 2, 4, 8, 16)
    assert np.array_equal(hc.laplacian(c, out_dtype="int64").cpu().numpy(), orc.lap_q(q))
    assert hc.autotune(c, "derivative", "float32") in (1, 2, 4, 8, 16)
    for ax in range(3):
        _close(hc.derivative(c, ax).cpu().numpy(), orc.stencil_q(q, orc.KIND_DERIV, eps, ax), RTOL_F32, eps)
    assert hc.autotune(c, "mean") == 0  # statistics have no tile to tune
