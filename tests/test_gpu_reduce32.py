"""Fused statistics of block-size-32 streams (the warp-autonomous kernel of
hc_reduce32.cu) against the CPU oracle, through the C ABI (needs a GPU).

The streams are encoded by the oracle from drawn codes, so the block widths
and the code range are chosen: every group size of the grouped unpacker
(largest width <= 8, <= 10, <= 16), both accumulator classes (max |q| below
and above 2^12), width-0 blocks, a last chunk with fewer than 128 blocks and
a last block with fewer than 32 codes, streams of one block, and a stream
long enough that every warp of the persistent grid takes several chunks
(both copy buffers reused).  Bars: the exact sums s1 and s2 bit for bit; the
mean, variance and std within 1e-12 relative (the same double arithmetic).
"""
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


def _codes(n, wmax, base_bits, zero_frac, seed):
    """Codes whose in-block deltas stay below 2^(wmax-1) and whose blocks sit
    at offsets up to 2^base_bits; a fraction of blocks constant (width 0)."""
    rng = np.random.default_rng(seed)
    nb = (n + 31) // 32
    base = rng.integers(-(1 << base_bits), (1 << base_bits) + 1, size=nb).astype(np.int64)
    a = (1 << (wmax - 1)) - 1 if wmax > 1 else 0  # |p| <= 2a < 2^wmax
    u = rng.integers(-a, a + 1, size=nb * 32).astype(np.int64) if a > 0 else np.zeros(nb * 32, np.int64)
    const = rng.random(nb) < zero_frac
    u.reshape(nb, 32)[const] = 0
    q = (np.repeat(base, 32) + u)[:n]
    return np.ascontiguousarray(q.astype(np.int32))


CASES = [
    # name, n, wmax bound, base bits, width-0 fraction
    ("g4_narrow", 4096 * 37 + 32 * 5 + 7, 8, 10, 0.1),
    ("g3_narrow", 4096 * 21 + 32 * 127 + 31, 10, 10, 0.0),
    ("g2_narrow", 4096 * 9 + 1, 14, 10, 0.05),
    ("g2_wide_codes", 4096 * 13 + 32 * 3, 16, 24, 0.1),
    ("g4_wide_codes", 4096 * 5 + 17, 7, 25, 0.3),
    ("one_block", 32, 9, 8, 0.0),
    ("one_partial_block", 19, 9, 8, 0.0),
    ("all_constant", 4096 * 3 + 100, 1, 11, 1.0),
]


def _check(hc, torch, dev, orc, q, pred):
    eps = 0.5e-3
    ref = orc.compress_codes(q, eps, 32, pred=pred)
    h = orc.read_header(ref)
    c = hc.from_stream(torch.from_numpy(ref).to(dev))
    assert c.header.wmax <= 16 and c.header.S == 32
    s1, s2 = orc.sums_q(q)
    n = q.size
    m_ref, v_ref, sd_ref = orc.finalize(n, s1, s2, eps)
    for level in ("p", "q"):
        rm = hc.parse_scalar(hc.mean(c, level=level))
        assert rm["status"] == 0 and rm["s1"] == s1, level
        assert abs(rm["mean"] - m_ref) <= 1e-12 * max(abs(m_ref), 2 * eps)
    rv = hc.parse_scalar(hc.variance(c, level="q"))
    assert rv["status"] == 0 and (rv["s1"], rv["s2"], rv["exact"]) == (s1, s2, 1)
    if n >= 2:
        assert abs(rv["variance"] - v_ref) <= 1e-12 * max(v_ref, (2 * eps) ** 2)
        assert abs(rv["std"] - sd_ref) <= 1e-12 * max(sd_ref, 2 * eps)
    if pred == 0:
        rp = hc.parse_scalar(hc.variance(c, level="p"))
        assert (rp["s1"], rp["s2"], rp["exact"], rp["status"]) == (s1, s2, 1, 0)
    else:
        M = orc.decode(ref, "m")
        dp = orc.decode(ref, "p").reshape(-1)
        mt, ss, sigma = orc.std_p_x(dp, M, 32, eps)
        rp = hc.parse_scalar(hc.variance(c, level="p"))
        assert (rp["s1"], rp["s2"], rp["exact"], rp["status"]) == (s1, ss, 0, 0)
        if n >= 2:
            assert abs(rp["std"] - sigma) <= 1e-12 * max(sigma, 2 * eps)
    assert hc.workspace_status() == 0
    return h


@pytest.mark.parametrize("name,n,wmax,bits,zf", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("pred", [0, 1], ids=["delta", "mean"])
def test_reduce32_matches_the_oracle(env, orc, name, n, wmax, bits, zf, pred):
    hc, torch, dev = env
    q = _codes(n, wmax, bits, zf, seed=sum(map(ord, name)) + 17 * pred)
    h = _check(hc, torch, dev, orc, q, pred)
    assert h["wmax"] <= wmax


def test_reduce32_many_chunks_per_warp(env, orc):
    """Far more chunks than warps in the persistent grid (each warp reuses
    both copy buffers many times) and a ragged end."""
    hc, torch, dev = env
    n = 4096 * 12000 + 32 * 77 + 9
    q = _codes(n, 10, 12, 0.05, seed=99)
    _check(hc, torch, dev, orc, q, 0)


def test_reduce32_and_general_kernel_agree(env, orc):
    """A stream the fast kernel takes and the same codes at widths it does
    not (largest width 17): both give the oracle's exact sums."""
    hc, torch, dev = env
    q = _codes(4096 * 30 + 5, 10, 10, 0.0, seed=5)
    q_wide = q.copy()
    q_wide[100] += 1 << 16  # one block of width 17: the general kernel
    for arr in (q, q_wide):
        ref = orc.compress_codes(arr, 1e-3, 32)
        c = hc.from_stream(torch.from_numpy(ref).to(dev))
        s1, s2 = orc.sums_q(arr)
        r = hc.parse_scalar(hc.variance(c, level="q"))
        assert (r["s1"], r["s2"], r["status"]) == (s1, s2, 0)
        assert hc.parse_scalar(hc.mean(c, level="p"))["s1"] == s1
