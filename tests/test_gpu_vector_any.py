"""Divergence and curl on components of any predictor (Section V-C) on the
GPU against the oracle (needs a GPU): HSZp-nd and HSZx-nd components at
stage 2 (each component's stage-2 derivative -- box sums of D_p, or D_p with
the box means at box borders -- then added) and at stage 3, and components of
mixed predictors; the same values as the fused kernel's formula."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

PRED = {"delta": 0, "mean": 1, "lorenzo": 2, "global": 3}


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2603_25206_gb300 import hc

    hc.lib()
    return hc, torch, torch.device("cuda:0")


def _components(orc, hc, torch, dev, shape, preds, rel, seed, block=None):
    import synth

    comps, qs, eps = [], [], []
    for c, pred in enumerate(preds):
        x = synth.grf_field(shape, seed + c)
        eb = 1e-3 if rel else 2e-3
        if pred == "mean-nd":
            ref, e = orc.compress_nd(x, block, eb, rel)
            cc = hc.compress(torch.from_numpy(x).to(dev), eb, rel=rel, predictor="mean-nd", block=block)
        else:
            ref, e = orc.compress(x, eb, rel, 32, pred=PRED[pred])
            cc = hc.compress(torch.from_numpy(x).to(dev), eb, rel=rel, S=32, predictor=pred)
        assert np.array_equal(cc.stream[: cc.nbytes].cpu().numpy(), ref)
        comps.append(cc)
        qs.append(orc.decode(ref, "q"))
        eps.append(e)
    return comps, qs, eps


DIV_CASES = [((40, 70), ("lorenzo", "lorenzo"), False, None),
             ((40, 70), ("mean-nd", "mean-nd"), True, (8, 8)),
             ((10, 20, 30), ("lorenzo", "lorenzo", "lorenzo"), True, None),
             ((9, 17, 33), ("mean-nd", "mean-nd", "mean-nd"), False, (2, 4, 4)),
             ((12, 16, 40), ("lorenzo", "mean-nd", "delta"), False, (4, 4, 4)),
             ((12, 16, 40), ("global", "mean", "delta"), True, None)]


@pytest.mark.parametrize("shape,preds,rel,block", DIV_CASES)
def test_divergence_any_predictor(env, orc, shape, preds, rel, block):
    hc, torch, dev = env
    comps, qs, eps = _components(orc, hc, torch, dev, shape, preds, rel, 2100 + len(shape), block)
    num, val = orc.divergence_q(qs, eps)
    stage2 = all(p in ("lorenzo", "mean-nd") for p in preds)
    for level in ("p", "q"):
        if level == "p" and not stage2:
            with pytest.raises(hc.HcError) as e:
                hc.divergence(comps, out_dtype="float64", level="p")
            assert e.value.status == hc.HC_ERR_UNSUPPORTED
            continue
        d64 = hc.divergence(comps, out_dtype="float64", level=level).cpu().numpy()
        assert np.array_equal(d64, val), level
        d32 = hc.divergence(comps, out_dtype="float32", level=level).cpu().numpy()
        assert np.all(np.abs(d32 - val) <= 1e-6 * np.maximum(np.abs(val), min(eps))), level
        if len(set(eps)) == 1:
            assert np.array_equal(hc.divergence(comps, out_dtype="int64", level=level).cpu().numpy(), num)
    assert hc.workspace_status() == 0


@pytest.mark.parametrize("preds,rel,block", [(("lorenzo", "lorenzo"), False, None), (("mean-nd", "mean-nd"), True, (4, 8)),
                                             (("lorenzo", "mean-nd"), False, (8, 8)), (("delta", "lorenzo"), True, None)])
def test_curl_any_predictor(env, orc, preds, rel, block):
    hc, torch, dev = env
    comps, qs, eps = _components(orc, hc, torch, dev, (50, 36), preds, rel, 2200, block)
    num, val = orc.curl2_q(qs[0], qs[1], eps[0], eps[1])
    for level in ("p", "q"):
        if level == "p" and "delta" in preds:
            continue
        assert np.array_equal(hc.curl(comps, out_dtype="float64", level=level).cpu().numpy(), val), level
        if eps[0] == eps[1]:
            assert np.array_equal(hc.curl(comps, out_dtype="int64", level=level).cpu().numpy(), num), level
    assert hc.workspace_status() == 0
