"""The allocation-free variance entry point (needs a GPU).

hc_op_variance_noalloc serves callers that cannot allocate device memory:
its scratch is a static array inside libhc.so instead of a caller workspace.
This file is collected last.  It calls the entry point through the C ABI
twice in a row on each stream (the static scratch keeps the previous call's
contents, so the second call checks that the ticket is cleared) and compares
every result with hc_op_variance's on the same stream: exact integer sums
bit for bit, the scaled statistics within the 1e-12 relative bar of the other
GPU tests.
"""
import ctypes

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


def _noalloc(hc, torch, c, level):
    out = torch.empty(hc.SCALAR_BYTES, dtype=torch.uint8, device=c.stream.device)
    st = c.stage(level)
    rc = hc.lib().hc_op_variance_noalloc(ctypes.byref(st), c.eps, len(c.shape), hc._dims(c.shape),
                                         ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == hc.HC_OK, hc.lib().hc_last_error()
    return hc.parse_scalar(out)


def _same(got, ref):
    assert got["status"] == 0 and got["exact"] == 1
    assert (got["n"], got["s1"], got["s2"]) == (ref["n"], ref["s1"], ref["s2"])
    for k in ("mean", "variance", "std"):
        assert abs(got[k] - ref[k]) <= 1e-12 * abs(ref[k])


@pytest.mark.parametrize("shape,S,eb", [((64, 64, 64), 32, 1e-3), ((13, 17, 19), 16, 1e-2), ((5, 6, 70), 64, 1e-4),
                                        ((512, 512), 32, 1e-3)])
def test_noalloc_matches_workspace_variance(env, shape, S, eb):
    hc, torch, dev = env
    import synth

    c = hc.compress(torch.from_numpy(synth.grf_field(shape, 77)).to(dev), eb, S=S)
    for level in ("q", "p"):
        ref = hc.parse_scalar(hc.variance(c, level=level))
        for _ in range(2):
            _same(_noalloc(hc, torch, c, level), ref)


@pytest.mark.parametrize("shape,S,eb", [((64, 64, 64), 32, 1e-3), ((5, 6, 70), 64, 1e-4)])
def test_noalloc_block_mean_streams(env, shape, S, eb):
    """Block-mean (HSZx) streams at level q: the same exact sums as the
    workspace path, twice in a row; through the Python wrapper as well.  Their
    stage-2 deviation needs a workspace and is refused."""
    hc, torch, dev = env
    import synth

    c = hc.compress(torch.from_numpy(synth.grf_field(shape, 78)).to(dev), eb, S=S, predictor="mean")
    ref = hc.parse_scalar(hc.variance(c, level="q"))
    for _ in range(2):
        _same(_noalloc(hc, torch, c, "q"), ref)
        _same(hc.parse_scalar(hc.variance_noalloc(c, level="q")), ref)
    out = torch.empty(hc.SCALAR_BYTES, dtype=torch.uint8, device=dev)
    st = c.stage("p")
    rc = hc.lib().hc_op_variance_noalloc(ctypes.byref(st), c.eps, len(c.shape), hc._dims(c.shape),
                                         ctypes.c_void_p(out.data_ptr()), None)
    assert rc == hc.HC_ERR_UNSUPPORTED


def test_noalloc_rejects_array_inputs(env):
    hc, torch, dev = env
    q = torch.zeros(64, dtype=torch.int32, device=dev)
    st = hc.StageArray("q", q, (64,), 0.5).stage()
    out = torch.empty(hc.SCALAR_BYTES, dtype=torch.uint8, device=dev)
    rc = hc.lib().hc_op_variance_noalloc(ctypes.byref(st), 0.5, 1, hc._dims((64,)), ctypes.c_void_p(out.data_ptr()),
                                         None)
    assert rc == hc.HC_ERR_UNSUPPORTED
