"""Block-mean (HSZx) streams on the GPU against the oracle (needs a GPU):
stream bytes, every decompression stage, the stage-1 / 2 / 3 statistics and
the stage-3 stencils, one field at a time, in one pass and in a batch."""
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

    rng = np.random.default_rng(77)
    yield "grf_3d_S32", synth.grf_field((20, 33, 64), 51), 1e-3, True, 32
    yield "grf_3d_S16", synth.grf_field((9, 30, 40), 52), 1e-3, True, 16
    yield "grf_2d_S64", synth.grf_field((70, 90), 53), 1e-2, True, 64
    yield "walk_1d_S7", np.cumsum(rng.standard_normal(3001)).astype(np.float32), 1e-2, True, 7
    yield "grf_S1", synth.grf_field((6, 7, 9), 54), 1e-3, True, 1
    yield "grf_S128_f64", synth.grf_field((10, 16, 50), 55, dtype=np.float64), 1e-4, True, 128
    yield "constant", np.full((5, 6, 7), 2.5, np.float32), 1e-3, True, 32
    yield "single", np.array([3.25], np.float32), 0.1, False, 32
    x = synth.wide_field((4, 8, 64), 56)
    yield "widest_abs", (x - (x.max() + x.min()) / 2), float(x.max() - x.min()) / 2**31, False, 32


CASES = list(_cases())


@pytest.mark.parametrize("name,x,eb,rel,S", CASES, ids=[c[0] for c in CASES])
def test_hszx_stream_stages_and_statistics(env, orc, name, x, eb, rel, S):
    hc, torch, dev = env
    ref, eps = orc.compress(x, eb, rel, S, pred=1)
    c = hc.compress(torch.from_numpy(x).to(dev), eb, rel=rel, S=S, predictor="mean")
    assert c.header.pred == hc.HC_PRED_MEAN
    assert c.nbytes == ref.size
    assert np.array_equal(c.stream[: c.nbytes].cpu().numpy(), ref)
    for st in ("m", "p", "q", "f"):
        got = hc.decompress(c, st).cpu().numpy().reshape(-1)
        want = orc.decode(ref, st).reshape(-1)
        assert np.array_equal(got, want), st
    q = orc.decode(ref, "q").reshape(-1)
    M = orc.decode(ref, "m")
    dp = orc.decode(ref, "p").reshape(-1)
    n = q.size
    s1, s2 = orc.sums_q(q)
    # stage 1 (Eq. mean_m): fused on the stream and on the block-means array
    T = orc.mean_m_sum(M, S, n)
    for r in (hc.parse_scalar(hc.mean(c, level="m")),
              hc.parse_scalar(hc.mean(hc.as_stage(c, "m", hc.decompress(c, "m"))))):
        assert r["s1"] == T and r["exact"] == 0 and r["status"] == 0
        assert r["mean"] == (float(T) / n) * (2 * eps)
    # stage 2: exact mean; the standard deviation about the integer mean
    r = hc.parse_scalar(hc.mean(c, level="p"))
    assert r["s1"] == s1 == orc.mean_p_sum_x(dp, M, S)
    mt, ss, sigma = orc.std_p_x(dp, M, S, eps)
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


@pytest.mark.parametrize("name,x,eb,rel,S", CASES[:6], ids=[c[0] for c in CASES[:6]])
def test_hszx_stencils(env, orc, name, x, eb, rel, S):
    hc, torch, dev = env
    ref, eps = orc.compress(x, eb, rel, S, pred=1)
    c = hc.compress(torch.from_numpy(x).to(dev), eb, rel=rel, S=S, predictor="mean")
    q = orc.decode(ref, "q")
    for ax in range(q.ndim):
        d = hc.derivative(c, ax, out_dtype="int64").cpu().numpy()
        assert np.array_equal(d, orc.deriv_q(q, ax)), ax
    assert np.array_equal(hc.laplacian(c, out_dtype="int64").cpu().numpy(), orc.lap_q(q))
    g = hc.gradmag(c).cpu().numpy()
    val = orc.stencil_q(q, orc.KIND_GRADMAG, eps)
    assert np.all(np.abs(g - val) <= 1e-6 * np.maximum(np.abs(val), eps))
    # one pass and the batched launch on the same stream
    r = hc.multi(c, out_dtype="float64")
    assert torch.equal(r["laplacian"], hc.laplacian(c, out_dtype="float64"))
    assert hc.parse_scalar(r["stats"]) == hc.parse_scalar(hc.variance(c, level="q"))
    b = hc.Batch([(c, "mean|variance|laplacian")], field_dtype="int64")
    b.run()
    (sc, f), = b.results()
    assert np.array_equal(f.cpu().numpy(), orc.lap_q(q))
    assert (sc["s1"], sc["s2"]) == orc.sums_q(q)
    assert hc.workspace_status() == 0


def test_hszx_stage_rules(env, orc):
    """Stage 1 and the stage-2 deviation are HSZx forms: a delta-coded stream
    refuses stage 1, and stencils refuse stages 1 and 2."""
    import synth

    hc, torch, dev = env
    x = torch.from_numpy(synth.grf_field((8, 16, 32), 60)).to(dev)
    cd = hc.compress(x, 1e-3, rel=True, S=32)
    with pytest.raises(hc.HcError) as e:
        hc.mean(cd, level="m")
    assert e.value.status == hc.HC_ERR_UNSUPPORTED
    cx = hc.compress(x, 1e-3, rel=True, S=32, predictor="mean")
    with pytest.raises(hc.HcError) as e:
        hc.variance(cx, level="m")
    assert e.value.status == hc.HC_ERR_UNSUPPORTED
    for lv in ("m", "p"):
        with pytest.raises(hc.HcError) as e:
            hc.laplacian(cx, level=lv)
        assert e.value.status == hc.HC_ERR_UNSUPPORTED
    with pytest.raises(hc.HcError) as e:
        hc.mean(hc.as_stage(cx, "p", hc.decompress(cx, "p")))
    assert e.value.status == hc.HC_ERR_UNSUPPORTED


@pytest.mark.parametrize("fi", [1, 4])
def test_hszx_paper_field_full_size(env, orc, fi):
    """The 512^3 and the 1800x3600 paper-like fields as HSZx streams (block 32):
    bytes, stage-1 and exact sums, sampled stencils."""
    import synth

    hc, torch, dev = env
    shape = synth.PAPER_SHAPES[fi]
    x = synth.grf_field(shape, 1000 + fi)
    ref, eps = orc.compress(x, 1e-3, True, 32, pred=1)
    c = hc.compress(torch.from_numpy(x).to(dev), 1e-3, rel=True, S=32, predictor="mean")
    del x
    assert np.array_equal(c.stream[: c.nbytes].cpu().numpy(), ref)
    q = orc.decode(ref, "q")
    M = orc.decode(ref, "m")
    s1, s2 = orc.sums_q(q)
    assert hc.parse_scalar(hc.mean(c, level="m"))["s1"] == orc.mean_m_sum(M, 32, q.size)
    assert hc.parse_scalar(hc.mean(c, level="p"))["s1"] == s1
    r = hc.parse_scalar(hc.variance(c, level="q"))
    assert (r["s1"], r["s2"]) == (s1, s2)
    rng = np.random.default_rng(fi)
    idx = np.unique(np.concatenate([[0, q.size - 1], rng.integers(0, q.size, 4000)]))
    num, _ = orc.stencil_at(q, orc.KIND_LAPLACIAN, eps, idx)
    lap = hc.laplacian(c, out_dtype="int64").reshape(-1)[torch.from_numpy(idx).to(dev)].cpu().numpy()
    assert np.array_equal(lap, num)
