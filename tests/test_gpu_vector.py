"""Divergence and curl of vector fields stored as compressed components
(Section V-C), fused on the GPU, against the oracle (needs a GPU)."""
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


def _components(orc, hc, torch, dev, shape, S, rel, seed, predictor="delta"):
    import synth

    comps, qs, eps = [], [], []
    pred = 1 if predictor == "mean" else 0
    for c in range(len(shape)):
        x = synth.grf_field(shape, seed + c)
        eb = 1e-3 if rel else 2e-3
        ref, e = orc.compress(x, eb, rel, S, pred=pred)
        cc = hc.compress(torch.from_numpy(x).to(dev), eb, rel=rel, S=S, predictor=predictor)
        assert np.array_equal(cc.stream[: cc.nbytes].cpu().numpy(), ref)
        comps.append(cc)
        qs.append(orc.decode(ref, "q"))
        eps.append(e)
    return comps, qs, eps


@pytest.mark.parametrize("shape,S,rel,pred", [((40, 70), 32, False, "delta"), ((40, 70), 32, True, "delta"),
                                              ((10, 20, 30), 32, True, "delta"), ((9, 17, 33), 16, False, "delta"),
                                              ((33, 64), 64, True, "mean"), ((6, 8, 130), 32, False, "mean")])
def test_divergence_matches_oracle(env, orc, shape, S, rel, pred):
    hc, torch, dev = env
    comps, qs, eps = _components(orc, hc, torch, dev, shape, S, rel, 900 + len(shape) + S, pred)
    num, val = orc.divergence_q(qs, eps)
    d64 = hc.divergence(comps, out_dtype="float64").cpu().numpy()
    assert np.array_equal(d64, val)
    d32 = hc.divergence(comps, out_dtype="float32").cpu().numpy()
    scale = np.maximum(np.abs(val), min(eps))
    assert np.all(np.abs(d32 - val) <= 1e-6 * scale)
    if len(set(eps)) == 1:
        assert np.array_equal(hc.divergence(comps, out_dtype="int64").cpu().numpy(), num)
    else:
        with pytest.raises(hc.HcError) as e:
            hc.divergence(comps, out_dtype="int64")
        assert e.value.status == hc.HC_ERR_UNSUPPORTED
    assert hc.workspace_status() == 0


@pytest.mark.parametrize("shape,S,rel", [((40, 70), 32, False), ((50, 36), 32, True), ((31, 45), 7, False)])
def test_curl_matches_oracle(env, orc, shape, S, rel):
    hc, torch, dev = env
    comps, qs, eps = _components(orc, hc, torch, dev, shape, S, rel, 950 + S)
    num, val = orc.curl2_q(qs[0], qs[1], eps[0], eps[1])
    assert np.array_equal(hc.curl(comps, out_dtype="float64").cpu().numpy(), val)
    c32 = hc.curl(comps).cpu().numpy()
    assert np.all(np.abs(c32 - val) <= 1e-6 * np.maximum(np.abs(val), min(eps)))
    if eps[0] == eps[1]:
        assert np.array_equal(hc.curl(comps, out_dtype="int64").cpu().numpy(), num)


def test_vector_argument_rules(env, orc):
    hc, torch, dev = env
    comps, qs, eps = _components(orc, hc, torch, dev, (6, 8, 16), 32, False, 990)
    with pytest.raises(hc.HcError) as e:
        hc.curl(comps[:2] + [comps[2]])  # 3-D curl is not defined here
    assert e.value.status == hc.HC_ERR_UNSUPPORTED
    with pytest.raises(hc.HcError) as e:
        hc.divergence(comps[:2])  # ncomp != ndim
    assert e.value.status == hc.HC_ERR_INVALID_ARG
