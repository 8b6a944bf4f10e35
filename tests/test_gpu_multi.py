"""All operations of one field from one decode (hc_op_multi) against the
one-operation entry points and the oracle (needs a GPU)."""
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


# (shape, S, out dtype): block 32 with rows of a multiple of 8 / 4 take the
# one-pass kernel; other rows, other block sizes and 1-D fields walk the
# one-operation kernels in turn
CASES = [
    ((40, 33, 64), 32, "float32"),
    ((17, 20, 36), 32, "float32"),
    ((9, 30, 40), 32, "float64"),
    ((300, 256), 32, "float32"),
    ((13, 14, 30), 32, "float32"),
    ((12, 16, 64), 64, "float32"),
    ((4096,), 32, "float32"),
    ((64, 64, 64), 16, "float64"),
    ((1, 24, 40), 32, "float32"),  # first axis of length 1: walked as (24, 1, 40)
]


@pytest.mark.parametrize("shape,S,dt", CASES)
def test_multi_equals_one_operation_calls(env, orc, shape, S, dt):
    import synth

    hc, torch, dev = env
    x = synth.grf_field(shape, 7000 + S + len(shape))
    ref, eps = orc.compress(x, 1e-3, True, S)
    c = hc.compress(torch.from_numpy(x).to(dev), 1e-3, rel=True, S=S)
    r = hc.multi(c, out_dtype=dt)
    torch.cuda.synchronize()
    for a in range(len(shape)):
        assert torch.equal(r["derivative"][a], hc.derivative(c, a, out_dtype=dt)), a
    assert torch.equal(r["gradmag"], hc.gradmag(c, out_dtype=dt))
    assert torch.equal(r["laplacian"], hc.laplacian(c, out_dtype=dt))
    m = hc.parse_scalar(r["stats"])
    v = hc.parse_scalar(hc.variance(c, level="q"))
    assert m == v
    q = orc.decode(ref, "q")
    s1, s2 = orc.sums_q(q)
    assert (m["s1"], m["s2"], m["status"]) == (s1, s2, 0)
    tol = 1e-6 if dt == "float32" else 1e-12
    for a in range(len(shape)):
        val = orc.stencil_q(q, orc.KIND_DERIV, eps, a)
        assert np.all(np.abs(r["derivative"][a].cpu().numpy() - val) <= tol * np.maximum(np.abs(val), eps)), a
    val = orc.stencil_q(q, orc.KIND_LAPLACIAN, eps)
    assert np.all(np.abs(r["laplacian"].cpu().numpy() - val) <= tol * np.maximum(np.abs(val), 2 * eps))
    assert hc.workspace_status() == 0


def test_multi_subsets_and_full_size(env, orc):
    """Any subset of outputs; the 512^3 paper-like field at full size."""
    import synth

    hc, torch, dev = env
    x = synth.grf_field((512, 512, 512), 1001)
    c = hc.compress(torch.from_numpy(x).to(dev), 1e-3, rel=True, S=32)
    del x
    r = hc.multi(c, derivative=False, gradmag=False, laplacian=True, stats=True)
    assert set(r) == {"laplacian", "stats"}
    assert torch.equal(r["laplacian"], hc.laplacian(c))
    full = hc.multi(c)
    for a in range(3):
        assert torch.equal(full["derivative"][a], hc.derivative(c, a))
    assert torch.equal(full["gradmag"], hc.gradmag(c))
    assert torch.equal(full["laplacian"], r["laplacian"])
    assert hc.parse_scalar(full["stats"]) == hc.parse_scalar(hc.variance(c, level="q"))
    # statistics only
    s = hc.multi(c, derivative=False, gradmag=False, laplacian=False)
    assert hc.parse_scalar(s["stats"]) == hc.parse_scalar(full["stats"])
    assert hc.workspace_status() == 0


def test_multi_autotune_keeps_results(env, orc):
    """Tuning the one-pass kernel's tile height changes no output."""
    import synth

    hc, torch, dev = env
    x = synth.grf_field((70, 96, 120), 7100)
    c = hc.compress(torch.from_numpy(x).to(dev), 1e-3, rel=True, S=32)
    before = hc.multi(c)
    ty = hc.autotune(c, "multi")
    assert ty in (1, 2, 4, 8, 16)
    after = hc.multi(c)
    for a in range(3):
        assert torch.equal(before["derivative"][a], after["derivative"][a])
    assert torch.equal(before["gradmag"], after["gradmag"]) and torch.equal(before["laplacian"], after["laplacian"])
    assert hc.parse_scalar(before["stats"]) == hc.parse_scalar(after["stats"])
