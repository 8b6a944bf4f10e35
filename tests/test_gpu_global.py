"""Global-predictor streams on the GPU against the oracle (needs a GPU).

HSZp-nd (Lorenzo over the field's axes) and HSZp (delta across blocks over
the flattened field), Section IV: stream bytes, every decompression stage,
the stage-2 mean (weighted sum, fused with the decode), the Algorithm 4 and
stage-3 statistics, the stage-2 derivative and Laplacian of HSZp-nd (box sums
of D_p over the other axes) and the stage-3 stencils, one field at a time;
the refusals; and one paper-size field.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

LORENZO, GLOBAL = 2, 3


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

    rng = np.random.default_rng(91)
    yield "grf_3d_S32", synth.grf_field((20, 33, 64), 61), 1e-3, True, 32
    yield "grf_3d_ragged_S32", synth.grf_field((13, 37, 45), 62), 1e-3, True, 32
    yield "grf_3d_S16", synth.grf_field((9, 30, 40), 63), 1e-2, True, 16
    yield "grf_2d_S64", synth.grf_field((70, 90), 64), 1e-2, True, 64
    yield "grf_2d_long_rows", synth.grf_field((5, 5000), 65), 1e-3, True, 32
    yield "walk_1d_S7", np.cumsum(rng.standard_normal(3001)).astype(np.float32), 1e-2, True, 7
    yield "walk_1d_long", np.cumsum(rng.standard_normal(200003)).astype(np.float32), 1e-3, True, 32
    yield "grf_S128_f64", synth.grf_field((10, 16, 50), 66, dtype=np.float64), 1e-4, True, 128
    yield "axis_len_1", synth.grf_field((1, 40, 33), 67), 1e-3, True, 32
    yield "thin_planes", synth.grf_field((70, 2, 3), 68), 1e-3, True, 32
    yield "constant", np.full((5, 6, 7), 2.5, np.float32), 1e-3, True, 32
    yield "single", np.array([3.25], np.float32), 0.1, False, 32


CASES = list(_cases())


def _stage_view(hc, c, stage, out_dtype=None):
    return hc.as_stage(c, stage, hc.decompress(c, stage, out_dtype=out_dtype))


@pytest.mark.parametrize("pred", [LORENZO, GLOBAL])
@pytest.mark.parametrize("name,x,eb,rel,S", CASES, ids=[c[0] for c in CASES])
def test_global_stream_stages_and_statistics(env, orc, pred, name, x, eb, rel, S):
    hc, torch, dev = env
    ref, eps = orc.compress(x, eb, rel, S, pred=pred)
    c = hc.compress(torch.from_numpy(x).to(dev), eb, rel=rel, S=S,
                    predictor="lorenzo" if pred == LORENZO else "global")
    assert c.header.pred == pred
    assert c.nbytes == ref.size
    assert np.array_equal(c.stream[: c.nbytes].cpu().numpy(), ref)
    for st in ("p", "q", "f"):
        got = hc.decompress(c, st).cpu().numpy().reshape(-1)
        want = orc.decode(ref, st).reshape(-1)
        assert np.array_equal(got, want), st
    got64 = hc.decompress(c, "f", out_dtype="float64").cpu().numpy().reshape(-1)
    q = orc.decode(ref, "q")
    assert np.array_equal(got64, orc.dequantize(q, eps, np.float64).reshape(-1))
    with pytest.raises(hc.HcError) as e:
        hc.decompress(c, "m")
    assert e.value.status == hc.HC_ERR_UNSUPPORTED
    n = q.size
    s1, s2 = orc.sums_q(q)
    dp = orc.decode(ref, "p")
    # stage 2 mean: the weighted sum, fused
    r = hc.parse_scalar(hc.mean(c, level="p"))
    assert (r["s1"], r["exact"], r["status"]) == (s1, 1, 0)
    assert s1 == orc.lorenzo_mean_p(dp, pred)
    assert r["mean"] == orc.finalize(n, s1, s2, eps)[0]
    # stage 2 (Algorithm 4) and stage 3 statistics: exact
    want = orc.lorenzo_var_p(dp, pred)
    assert want == (s1, s2)
    m_ref, v_ref, _ = orc.finalize(n, s1, s2, eps)
    for level in ("p", "q"):
        r = hc.parse_scalar(hc.variance(c, level=level))
        assert (r["s1"], r["s2"], r["exact"], r["status"]) == (s1, s2, 1, 0), level
        if n >= 2:
            assert abs(r["variance"] - v_ref) <= 1e-12 * max(v_ref, (2 * eps) ** 2)
        r = hc.parse_scalar(hc.mean(c, level="q"))
        assert r["s1"] == s1
    assert hc.workspace_status() == 0


def _same_codes_delta(hc, torch, dev, q, eps, S, dtype):
    return hc.compress_codes(torch.from_numpy(np.ascontiguousarray(q)).to(dev), eps, S=S,
                             dtype="float64" if dtype == np.float64 else "float32")


@pytest.mark.parametrize("pred", [LORENZO, GLOBAL])
@pytest.mark.parametrize("name,x,eb,rel,S", CASES, ids=[c[0] for c in CASES])
def test_global_stream_stencils(env, orc, pred, name, x, eb, rel, S):
    """Stage 3 on a global stream equals stage 3 on a delta stream of the same
    codes bit for bit; stage 2 of HSZp-nd (Eq. derivative_Dp, Eq.
    laplacian_Dp) gives the oracle's numerators exactly and the same scaled
    values as stage 3."""
    hc, torch, dev = env
    if x.size > 300000:
        pytest.skip("statistics-only case")
    ref, eps = orc.compress(x, eb, rel, S, pred=pred)
    c = hc.from_stream(torch.from_numpy(ref).to(dev))
    q = orc.decode(ref, "q")
    dp = orc.decode(ref, "p")
    d = _same_codes_delta(hc, torch, dev, q, eps, S, x.dtype)
    nd = q.ndim
    for out in ("float32", "float64", "int64"):
        for a in range(nd):
            g3 = hc.derivative(c, a, out_dtype=out, level="q")
            assert torch.equal(g3, hc.derivative(d, a, out_dtype=out, level="q")), (out, a)
            if pred == LORENZO:
                g2 = hc.derivative(c, a, out_dtype=out, level="p")
                assert torch.equal(g2, g3), ("p", out, a)
                if out == "int64":
                    np.testing.assert_array_equal(g2.cpu().numpy(), orc.lorenzo_deriv_p(dp, a))
        l3 = hc.laplacian(c, out_dtype=out, level="q")
        assert torch.equal(l3, hc.laplacian(d, out_dtype=out, level="q")), out
        if pred == LORENZO:
            l2 = hc.laplacian(c, out_dtype=out, level="p")
            assert torch.equal(l2, l3), ("p", out)
            if out == "int64":
                np.testing.assert_array_equal(l2.cpu().numpy(), orc.lorenzo_lap_p(dp))
        if out != "int64":
            assert torch.equal(hc.gradmag(c, out_dtype=out, level="q"), hc.gradmag(d, out_dtype=out, level="q"))
    # the stage-2 derivative values against the oracle's scaled results
    if pred == LORENZO:
        v = hc.derivative(c, 0, out_dtype="float64", level="p").cpu().numpy()
        want = orc.stencil_q(q, orc.KIND_DERIV, eps, axis=0)
        assert np.all(np.abs(v - want) <= 1e-12 * np.maximum(np.abs(want), eps))
        v = hc.laplacian(c, out_dtype="float32", level="p").cpu().numpy()
        want = orc.stencil_q(q, orc.KIND_LAPLACIAN, eps)
        assert np.all(np.abs(v - want) <= 1e-6 * np.maximum(np.abs(want), eps))
    assert hc.workspace_status() == 0


def test_global_refusals(env, orc):
    """What the global predictors do not offer is refused, nothing runs: stage
    1, the stage-2 gradient magnitude, stage-2 differentiation of HSZp (a 1-D
    partition, also inside a divergence), D_p arrays, the batch, the
    allocation-free variance, and a workspace smaller than
    hc_workspace_bytes_for."""
    import ctypes

    import synth

    hc, torch, dev = env
    x = synth.grf_field((8, 20, 24), 71)
    cl = hc.compress(torch.from_numpy(x).to(dev), 1e-3, predictor="lorenzo")
    cg = hc.compress(torch.from_numpy(x).to(dev), 1e-3, predictor="global")
    U = hc.HC_ERR_UNSUPPORTED
    for fn in (lambda: hc.gradmag(cl, level="p"), lambda: hc.derivative(cg, 0, level="p"),
               lambda: hc.laplacian(cg, level="p"), lambda: hc.mean(cl, level="m"),
               lambda: hc.variance_noalloc(cl), lambda: hc.divergence([cg, cg, cg], level="p"),
               lambda: hc.mean(hc.as_stage(cl, "p", hc.decompress(cl, "p")))):
        with pytest.raises(hc.HcError) as e:
            fn()
        assert e.value.status == U
    with pytest.raises(hc.HcError) as e:
        hc.Batch([(cl, "mean")])
    assert e.value.status == U
    # a workspace of hc_workspace_bytes() is too small for a rebuilt D_q
    L = hc.lib()
    need = int(L.hc_workspace_bytes_for(ctypes.byref(cl.header)))
    base = int(L.hc_workspace_bytes())
    assert need >= base + 12 * x.size
    ws = torch.zeros(base, dtype=torch.uint8, device=dev)
    out = torch.empty(x.shape, dtype=torch.int32, device=dev)
    rc = L.hc_decompress_to_stage(ctypes.byref(cl.header), ctypes.c_void_p(cl.stream.data_ptr()), hc.HC_STAGE_Q,
                                  ctypes.c_void_p(out.data_ptr()), hc.HC_F32, ctypes.c_void_p(ws.data_ptr()), base,
                                  None)
    assert rc == hc.HC_ERR_NOMEM
    # a residual beyond the encoder's 31-bit magnitude
    z, y, xx = np.meshgrid(np.arange(3), np.arange(3), np.arange(3), indexing="ij")
    sign = (1 - 2 * ((xx + y + z) % 2)).astype(np.int32)
    with pytest.raises(hc.HcError) as e:
        hc.compress_codes(torch.from_numpy(sign * 2**28).to(dev), 1.0, predictor="lorenzo")
    assert e.value.status == hc.HC_ERR_RANGE
    ok = torch.from_numpy(sign * (2**28 - 1)).to(dev)
    c = hc.compress_codes(ok, 1.0, predictor="lorenzo")
    assert torch.equal(hc.decompress(c, "q").cpu(), ok.cpu())


def test_global_paper_size_field(env, orc):
    """One 256x384x384 paper-like field as HSZp-nd: the stream bit for bit,
    the exact stage-2 sums, and the stage-2 derivative and Laplacian at
    sampled points (edges, corners, random interior) against the oracle."""
    import synth

    hc, torch, dev = env
    shape = synth.PAPER_SHAPES[2]
    x = synth.grf_field(shape, 1002)
    ref, eps = orc.compress(x, 1e-3, True, 32, pred=LORENZO)
    c = hc.compress(torch.from_numpy(x).to(dev), 1e-3, rel=True, S=32, predictor="lorenzo")
    del x
    assert c.nbytes == ref.size
    assert np.array_equal(c.stream[: c.nbytes].cpu().numpy(), ref)
    q = orc.decode(ref, "q")
    del ref
    s1, s2 = orc.sums_q(q)
    assert hc.parse_scalar(hc.mean(c, level="p"))["s1"] == s1
    r = hc.parse_scalar(hc.variance(c, level="p"))
    assert (r["s1"], r["s2"]) == (s1, s2)
    rng = np.random.default_rng(5)
    n = q.size
    idx = np.unique(np.concatenate([rng.integers(0, n, 4000), [0, 1, shape[2] - 1, n - 1, n - shape[2]]]))
    for a in range(3):
        v = hc.derivative(c, a, out_dtype="float32", level="p").reshape(-1)[torch.from_numpy(idx).to(dev)]
        num, val = orc.stencil_at(q, orc.KIND_DERIV, eps, idx, axis=a)
        np.testing.assert_array_equal(
            hc.derivative(c, a, out_dtype="int64", level="p").reshape(-1)[torch.from_numpy(idx).to(dev)]
            .cpu().numpy(), num)
        assert np.all(np.abs(v.cpu().numpy() - val) <= 1e-6 * np.maximum(np.abs(val), eps))
    lap = hc.laplacian(c, out_dtype="int64", level="p").reshape(-1)[torch.from_numpy(idx).to(dev)]
    num, _ = orc.stencil_at(q, orc.KIND_LAPLACIAN, eps, idx)
    np.testing.assert_array_equal(lap.cpu().numpy(), num)
    assert hc.workspace_status() == 0


@pytest.mark.parametrize("pred", [LORENZO, GLOBAL])
def test_global_corrupt_stream_reported_not_faulting(env, orc, pred):
    """A width byte above the header's max width in a global-predictor stream:
    the residual decoder and the fused stage-2 mean flag the tile and skip it
    (every read stays inside the stream); the status comes back on the host."""
    import synth

    hc, torch, dev = env
    x = synth.grf_field((16, 16, 64), 4)
    ref, eps = orc.compress(x, 1e-3, True, 32, pred=pred)
    bad = ref.copy()
    bad[256 + 100] = 31
    c = hc.from_stream(torch.from_numpy(bad).to(dev))
    # a statistic reports in its result; decoders in the workspace status word
    assert hc.parse_scalar(hc.mean(c, level="p"))["status"] == hc.HC_ERR_CORRUPT
    hc.decompress(c, "q")
    assert hc.workspace_status() == hc.HC_ERR_CORRUPT
    if pred == LORENZO:
        hc.laplacian(c, level="p")
        assert hc.workspace_status() == hc.HC_ERR_CORRUPT
    assert hc.workspace_status() == 0


def test_global_multi_equals_one_operation_calls(env):
    """hc_op_multi on global-predictor streams takes the one-operation paths:
    the same bytes as the separate calls, at stage 3 and (HSZp-nd, without the
    gradient magnitude) at stage 2."""
    import synth

    hc, torch, dev = env
    x = synth.grf_field((9, 20, 36), 72)
    for pred in ("lorenzo", "global"):
        c = hc.compress(torch.from_numpy(x).to(dev), 1e-3, predictor=pred)
        r = hc.multi(c, level="q")
        for a in range(3):
            assert torch.equal(r["derivative"][a], hc.derivative(c, a, level="q"))
        assert torch.equal(r["gradmag"], hc.gradmag(c, level="q"))
        assert torch.equal(r["laplacian"], hc.laplacian(c, level="q"))
        assert hc.parse_scalar(r["stats"]) == hc.parse_scalar(hc.variance(c, level="q"))
    c = hc.compress(torch.from_numpy(x).to(dev), 1e-3, predictor="lorenzo")
    r = hc.multi(c, level="p", gradmag=False)
    for a in range(3):
        assert torch.equal(r["derivative"][a], hc.derivative(c, a, level="q"))
    assert torch.equal(r["laplacian"], hc.laplacian(c, level="q"))
    assert hc.workspace_status() == 0
