"""Sharded reductions on the GPU (needs a GPU): every rank's shard (hc.shard,
built on the device) is byte for byte the oracle's compression of its slice
of the codes (but for the two header bounds the shard keeps from the whole
field), the fused statistics on the shards add up to the whole field's exact
sums, and the combined mean and variance (paper_2603_25206_gb300.shard)
equal the one-launch result bit for bit."""
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


@pytest.mark.parametrize("pred,name", [(0, "delta"), (1, "mean")])
def test_shards_reduce_to_the_whole_field(env, orc, pred, name):
    import synth
    from paper_2603_25206_gb300 import shard

    hc, torch, dev = env
    x = synth.grf_field((40, 64, 96), 41)
    c = hc.compress(torch.from_numpy(x).to(dev), 1e-3, rel=True, S=32, predictor=name)
    ref, eps = orc.compress(x, 1e-3, True, 32, pred=pred)
    q = orc.decode(ref, "q").reshape(-1)
    s1, s2 = orc.sums_q(q)
    full = hc.parse_scalar(hc.variance(c, level="q"))
    assert (full["s1"], full["s2"]) == (s1, s2)
    for world in (1, 2, 3, 7):
        tot = [0, 0, 0]
        for rank in range(world):
            sh = hc.shard(c, rank, world)
            if sh is None:
                continue
            got = sh.stream.cpu().numpy()
            m = int(sh.header.N)
            alone = orc.compress_codes(q[tot[2]:tot[2] + m], eps, 32, np.float32, eb=1e-3, rel=True, pred=pred)
            assert got.size == alone.size
            assert set(np.nonzero(got != alone)[0].tolist()) <= set(range(60, 64)) | set(range(136, 140))
            r = hc.parse_scalar(hc.variance(sh, level="q"))
            assert r["status"] == 0 and r["n"] == m
            if pred == 0:
                assert hc.parse_scalar(hc.mean(sh, level="p"))["s1"] == r["s1"]
            tot[0] += r["s1"]
            tot[1] += r["s2"]
            tot[2] += m
        assert tuple(tot) == (s1, s2, q.size)
        mean, var, _ = shard.finalize(tot[2], tot[0], tot[1], eps)
        assert (mean, var) == (full["mean"], full["variance"])
