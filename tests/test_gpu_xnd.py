"""HSZx-nd streams (block means over boxes of codes, Section IV) on the GPU
against the oracle (needs a GPU): stream bytes, every decompression stage,
the stage-1 / 2 / 3 statistics, the stage-2 stencils of Section V-B (p
differences plus the box means' difference at box borders) and the stage-3
stencils, the refusals, and one paper-size field."""
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


def _cases():
    import synth

    rng = np.random.default_rng(123)
    yield "grf_3d_444", synth.grf_field((20, 33, 64), 81), 1e-3, True, (4, 4, 4)
    yield "grf_3d_ragged_244", synth.grf_field((13, 37, 45), 82), 1e-3, True, (2, 4, 4)
    yield "grf_3d_888", synth.grf_field((17, 20, 36), 83), 1e-2, True, (8, 8, 8)
    yield "grf_3d_222", synth.grf_field((9, 10, 11), 84), 1e-3, True, (2, 2, 2)
    yield "grf_2d_88", synth.grf_field((70, 90), 85), 1e-2, True, (8, 8)
    yield "grf_2d_1616", synth.grf_field((50, 75), 86), 1e-3, True, (16, 16)
    yield "grf_2d_48", synth.grf_field((33, 40), 87), 1e-3, True, (4, 8)
    yield "walk_1d_32", np.cumsum(rng.standard_normal(3001)).astype(np.float32), 1e-2, True, (32,)
    yield "f64_3d_448", synth.grf_field((10, 16, 50), 88, dtype=np.float64), 1e-4, True, (4, 4, 8)
    yield "box_larger_than_field", synth.grf_field((3, 5, 6), 89), 1e-3, True, (8, 8, 8)
    yield "leading_len1", synth.grf_field((1, 24, 40), 90), 1e-3, True, (1, 8, 8)
    yield "constant", np.full((5, 6, 7), 2.5, np.float32), 1e-3, True, (2, 2, 2)
    yield "single", np.array([3.25], np.float32), 0.1, False, (4,)
    # one-pass box stencil tiles: boxes of odd extent (divisions, not
    # shifts) with a tile width that is not a multiple of 4 codes; a row of
    # several tiles with a ragged last one; tall fields whose tiles march
    # through more than one box layer (b0 = 1 and b0 = 4)
    yield "grf_3d_333_odd", synth.grf_field((7, 11, 13), 91), 1e-3, True, (3, 3, 3)
    yield "grf_3d_222_odd_cols", synth.grf_field((6, 10, 10), 92), 1e-3, True, (2, 2, 2)
    yield "grf_3d_wide_x", synth.grf_field((12, 20, 300), 93), 1e-3, True, (4, 4, 4)
    yield "grf_3d_tall_144", synth.grf_field((700, 8, 16), 94), 1e-3, True, (1, 4, 4)
    yield "grf_3d_tall_444", synth.grf_field((2500, 8, 8), 95), 1e-3, True, (4, 4, 4)


CASES = list(_cases())


@pytest.mark.parametrize("name,x,eb,rel,block", CASES, ids=[c[0] for c in CASES])
def test_box_stream_stages_and_statistics(env, orc, name, x, eb, rel, block):
    hc, torch, dev = env
    ref, eps = orc.compress_nd(x, block, eb, rel)
    c = hc.compress(torch.from_numpy(x).to(dev), eb, rel=rel, predictor="mean-nd", block=block)
    assert c.header.pred == hc.HC_PRED_MEAN_ND
    assert tuple(c.header.block)[3 - len(block):] == tuple(block)
    assert c.nbytes == ref.size
    assert np.array_equal(c.stream[: c.nbytes].cpu().numpy(), ref)
    for st in ("m", "p", "q", "f"):
        got = hc.decompress(c, st).cpu().numpy().reshape(-1)
        want = orc.decode(ref, st).reshape(-1)
        assert np.array_equal(got, want), st
    q = orc.decode(ref, "q")
    assert np.array_equal(hc.decompress(c, "f", out_dtype="float64").cpu().numpy().reshape(-1),
                          orc.dequantize(q, eps, np.float64).reshape(-1))
    M, dp = orc.decode(ref, "m"), orc.decode(ref, "p")
    n = q.size
    s1, s2 = orc.sums_q(q)
    # stage 1 (Eq. mean_m, true box sizes)
    T = orc.xnd_mean_m(M, x.shape, block)
    r = hc.parse_scalar(hc.mean(c, level="m"))
    assert (r["s1"], r["exact"], r["status"]) == (T, 0, 0)
    assert r["mean"] == (float(T) / n) * (2 * eps)
    # stage 2: the exact mean; the deviation about mu~
    r = hc.parse_scalar(hc.mean(c, level="p"))
    assert (r["s1"], r["exact"]) == (s1, 1) and s1 == orc.xnd_mean_p(dp, M, block)
    mt, ss, sigma = orc.xnd_std_p(dp, M, block, eps)
    r = hc.parse_scalar(hc.variance(c, level="p"))
    assert (r["s1"], r["s2"], r["exact"], r["status"]) == (s1, ss, 0, 0)
    if n >= 2:
        assert abs(r["std"] - sigma) <= 1e-12 * max(sigma, 2 * eps)
    # stage 3: exact
    r = hc.parse_scalar(hc.variance(c, level="q"))
    assert (r["s1"], r["s2"], r["exact"]) == (s1, s2, 1)
    m_ref, v_ref, _ = orc.finalize(n, s1, s2, eps)
    if n >= 2:
        assert abs(r["variance"] - v_ref) <= 1e-12 * max(v_ref, (2 * eps) ** 2)
    assert hc.workspace_status() == 0


@pytest.mark.parametrize("name,x,eb,rel,block", CASES, ids=[c[0] for c in CASES])
def test_box_stream_stencils(env, orc, name, x, eb, rel, block):
    """Stage 2 (Section V-B's HSZx-2d formulas on every axis) gives the
    oracle's numerators exactly and the same scaled values as stage 3; stage
    3 on the box stream equals stage 3 on a block-head stream of the same
    codes bit for bit."""
    hc, torch, dev = env
    ref, eps = orc.compress_nd(x, block, eb, rel)
    c = hc.from_stream(torch.from_numpy(ref).to(dev))
    q = orc.decode(ref, "q")
    M, dp = orc.decode(ref, "m"), orc.decode(ref, "p")
    d = hc.compress_codes(torch.from_numpy(np.ascontiguousarray(q)).to(dev), eps, S=32,
                          dtype="float64" if x.dtype == np.float64 else "float32")
    for out in ("float32", "float64", "int64"):
        for a in range(q.ndim):
            g2 = hc.derivative(c, a, out_dtype=out, level="p")
            g3 = hc.derivative(c, a, out_dtype=out, level="q")
            assert torch.equal(g2, g3), (out, a)
            assert torch.equal(g3, hc.derivative(d, a, out_dtype=out, level="q")), (out, a)
            if out == "int64":
                np.testing.assert_array_equal(g2.cpu().numpy(), orc.xnd_deriv_p(dp, M, block, a))
        l2 = hc.laplacian(c, out_dtype=out, level="p")
        assert torch.equal(l2, hc.laplacian(c, out_dtype=out, level="q")), out
        assert torch.equal(l2, hc.laplacian(d, out_dtype=out, level="q")), out
        if out == "int64":
            np.testing.assert_array_equal(l2.cpu().numpy(), orc.xnd_lap_p(dp, M, block))
        else:
            gm = hc.gradmag(c, out_dtype=out, level="p")
            assert torch.equal(gm, hc.gradmag(c, out_dtype=out, level="q"))
            assert torch.equal(gm, hc.gradmag(d, out_dtype=out, level="q"))
    v = hc.laplacian(c, out_dtype="float32", level="p").cpu().numpy()
    want = orc.stencil_q(q, orc.KIND_LAPLACIAN, eps)
    assert np.all(np.abs(v - want) <= 1e-6 * np.maximum(np.abs(want), 2 * eps))
    assert hc.workspace_status() == 0


def test_box_refusals(env):
    """Box streams are refused where a kernel assumes 1-D blocks: the batch,
    the allocation-free variance, stage arrays of D_p and D_m, and bad box
    extents."""
    import synth

    hc, torch, dev = env
    x = synth.grf_field((8, 20, 24), 91)
    c = hc.compress(torch.from_numpy(x).to(dev), 1e-3, predictor="mean-nd", block=(4, 4, 4))
    U = hc.HC_ERR_UNSUPPORTED
    for fn in (lambda: hc.variance_noalloc(c),
               lambda: hc.mean(hc.as_stage(c, "p", hc.decompress(c, "p"))),
               lambda: hc.mean(hc.as_stage(c, "m", hc.decompress(c, "m")))):
        with pytest.raises(hc.HcError) as e:
            fn()
        assert e.value.status == U
    with pytest.raises(hc.HcError) as e:
        hc.Batch([(c, "mean")])
    assert e.value.status == U
    for bad in ((4, 4), (0, 4, 4), (32, 32, 8)):
        with pytest.raises((hc.HcError, ValueError)):
            hc.compress(torch.from_numpy(x).to(dev), 1e-3, predictor="mean-nd", block=bad)


def test_box_paper_size_field(env, orc):
    """One 256x384x384 paper-like field in 4x4x4 boxes: the stream bit for
    bit, the exact statistics at stages 1-3, and the stage-2 stencils at
    sampled points against the oracle's stage-3 numerators."""
    import synth

    hc, torch, dev = env
    shape = synth.PAPER_SHAPES[2]
    x = synth.grf_field(shape, 1002)
    ref, eps = orc.compress_nd(x, (4, 4, 4), 1e-3, True)
    c = hc.compress(torch.from_numpy(x).to(dev), 1e-3, rel=True, predictor="mean-nd", block=(4, 4, 4))
    del x
    assert c.nbytes == ref.size
    assert np.array_equal(c.stream[: c.nbytes].cpu().numpy(), ref)
    q = orc.decode(ref, "q")
    M = orc.decode(ref, "m")
    del ref
    s1, s2 = orc.sums_q(q)
    assert hc.parse_scalar(hc.mean(c, level="m"))["s1"] == orc.xnd_mean_m(M, shape, (4, 4, 4))
    assert hc.parse_scalar(hc.mean(c, level="p"))["s1"] == s1
    r = hc.parse_scalar(hc.variance(c, level="q"))
    assert (r["s1"], r["s2"]) == (s1, s2)
    rng = np.random.default_rng(6)
    n = q.size
    idx = np.unique(np.concatenate([rng.integers(0, n, 4000), [0, 1, 3, 4, shape[2] - 1, n - 1, n - shape[2]]]))
    ti = torch.from_numpy(idx).to(dev)
    for a in range(3):
        got = hc.derivative(c, a, out_dtype="int64", level="p").reshape(-1)[ti].cpu().numpy()
        num, _ = orc.stencil_at(q, orc.KIND_DERIV, eps, idx, axis=a)
        np.testing.assert_array_equal(got, num)
    got = hc.laplacian(c, out_dtype="int64", level="p").reshape(-1)[ti].cpu().numpy()
    num, _ = orc.stencil_at(q, orc.KIND_LAPLACIAN, eps, idx)
    np.testing.assert_array_equal(got, num)
    assert hc.workspace_status() == 0


def test_box_corrupt_stream_reported_not_faulting(env, orc):
    """A width byte above the header's max width in a box stream: the box
    decoder and the statistics flag the tile and skip it; the status comes
    back on the host."""
    import synth

    hc, torch, dev = env
    x = synth.grf_field((16, 16, 64), 4)
    ref, eps = orc.compress_nd(x, (4, 4, 4), 1e-3, True)
    bad = ref.copy()
    bad[256 + 100] = 31
    c = hc.from_stream(torch.from_numpy(bad).to(dev))
    # a statistic reports in its result; decoders in the workspace status word
    assert hc.parse_scalar(hc.variance(c, level="q"))["status"] == hc.HC_ERR_CORRUPT
    hc.decompress(c, "q")
    assert hc.workspace_status() == hc.HC_ERR_CORRUPT
    hc.laplacian(c, level="p")
    assert hc.workspace_status() == hc.HC_ERR_CORRUPT
    assert hc.workspace_status() == 0


def test_box_multi_equals_one_operation_calls(env):
    """hc_op_multi on a box stream takes the one-operation paths: the same
    bytes as the separate calls at stages 2 and 3 (stage 2 equals stage 3)."""
    import synth

    hc, torch, dev = env
    x = synth.grf_field((9, 20, 36), 73)
    c = hc.compress(torch.from_numpy(x).to(dev), 1e-3, predictor="mean-nd", block=(2, 4, 4))
    for level in ("p", "q"):
        r = hc.multi(c, level=level)
        for a in range(3):
            assert torch.equal(r["derivative"][a], hc.derivative(c, a, level="q"))
        assert torch.equal(r["gradmag"], hc.gradmag(c, level="q"))
        assert torch.equal(r["laplacian"], hc.laplacian(c, level="q"))
    assert hc.workspace_status() == 0
