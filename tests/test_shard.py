"""Sharding a reduction over ranks, on the CPU: the shard plan of the C ABI
(hc_shard_plan, host only), the shard streams it describes (built here with
numpy from oracle streams), and the exact cross-rank combination
(paper_2603_25206_gb300.shard) over world-size-2 gloo ranks.

Pins: a shard is byte for byte the oracle's own compression of the same
slice of codes as a 1-D field (except the header's max |q| and max width,
which the shard keeps from the whole field as upper bounds); the oracle
decodes every shard to exactly its slice; the ranks' exact sums add up to
the whole field's, and the combined mean / variance / std equal the
oracle's bit for bit.
"""
import os
import sys

import numpy as np
import pytest

from test_abi_host import _header_from_oracle_stream

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hc():
    from paper_2603_25206_gb300 import build as b

    b.build()
    from paper_2603_25206_gb300 import hc as mod

    mod.lib()
    return mod


def _chunks(orc, s, h):
    r16 = lambda v: (v + 15) & ~15  # noqa: E731
    off = r16(r16(256 + h.nb) + 4 * h.nb)
    assert off == h.off_chunks
    return np.frombuffer(s[off:off + 8 * (h.nchunks + 1)].tobytes(), np.uint64)


def _build_shard(s, plan, rebased):
    """The shard stream from the plan, with numpy (what hc.shard does on the device)."""
    out = np.zeros(int(plan.hdr.total_bytes), np.uint8)
    out[:256] = np.frombuffer(bytes(plan.header_bytes), np.uint8)
    for k in range(3):
        n, so, do = int(plan.nbytes[k]), int(plan.src_off[k]), int(plan.dst_off[k])
        out[do:do + n] = s[so:so + n]
    co = int(plan.chunks_off)
    out[co:co + 8 * rebased.size] = rebased.view(np.uint8)
    return out


def _field(rng, n, dtype):
    return (np.cumsum(rng.standard_normal(n)) + 5 * (rng.random(n) < 0.02)).astype(dtype)


CASES = [(20000, 32, 0, np.float32), (20000, 32, 1, np.float32), (4096 * 3 + 17, 16, 0, np.float64),
         (50001, 64, 1, np.float64), (9000, 7, 0, np.float32), (100, 32, 0, np.float32)]


@pytest.mark.parametrize("n,S,pred,dtype", CASES)
def test_shards_are_standalone_streams_of_their_slices(hc, orc, rng, n, S, pred, dtype):
    x = _field(rng, n, dtype)
    s, eps = orc.compress(x, 1e-3, True, S, pred=pred)
    h = _header_from_oracle_stream(hc, orc, s)
    q = orc.decode(s, "q").reshape(-1)
    chunks = _chunks(orc, s, h)
    s1_full, s2_full = orc.sums_q(q)
    for world in (1, 2, 3, 5, 8):
        tot1, tot2, cover = 0, 0, 0
        for rank in range(world):
            c0, c1 = hc.shard_range(int(h.nchunks), rank, world)
            if c1 <= c0:
                continue
            plan, rebased = hc.shard_plan(h, chunks, c0, c1)
            sh = _build_shard(s, plan, rebased)
            first, m = int(plan.first), int(plan.hdr.N)
            assert first == cover  # contiguous, in rank order
            cover += m
            qs = orc.decode(sh, "q")
            np.testing.assert_array_equal(qs, q[first:first + m])
            np.testing.assert_array_equal(orc.decode(sh, "m"), orc.decode(s, "m")[c0 * h.G:c0 * h.G + plan.hdr.nb])
            # byte for byte the oracle's compression of the slice, but for the two upper bounds
            alone = orc.compress_codes(q[first:first + m], eps, S, dtype, eb=1e-3, rel=True, pred=pred)
            assert alone.size == sh.size
            diff = np.nonzero(alone != sh)[0]
            assert set(diff.tolist()) <= set(range(60, 64)) | set(range(136, 140))
            g = orc.read_header(sh)
            assert g["qmax"] == h.qmax and g["wmax"] == h.wmax and g["N"] == m
            a, b = orc.sums_q(qs)
            tot1 += a
            tot2 += b
        assert cover == n
        assert (tot1, tot2) == (s1_full, s2_full)


def test_shard_plan_refusals(hc, orc, rng):
    x = _field(rng, 9000, np.float32)
    for pred in (2, 3):
        s, _ = orc.compress(x, 1e-3, True, 32, pred=pred)
        h = _header_from_oracle_stream(hc, orc, s)
        with pytest.raises(hc.HcError) as e:
            hc.shard_plan(h, _chunks(orc, s, h), 0, 1)
        assert e.value.status == hc.HC_ERR_UNSUPPORTED
    s4, _ = orc.compress_nd(x.reshape(90, 100), (4, 4), 1e-3, True)
    h4 = _header_from_oracle_stream(hc, orc, s4)
    with pytest.raises(hc.HcError) as e:
        hc.shard_plan(h4, _chunks(orc, s4, h4), 0, 1)
    assert e.value.status == hc.HC_ERR_UNSUPPORTED
    s, _ = orc.compress(x, 1e-3, True, 32)
    h = _header_from_oracle_stream(hc, orc, s)
    ch = _chunks(orc, s, h)
    for c0, c1 in ((-1, 1), (1, 1), (2, 1), (0, int(h.nchunks) + 1)):
        with pytest.raises(hc.HcError) as e:
            hc.shard_plan(h, ch, c0, c1)
        assert e.value.status == hc.HC_ERR_INVALID_ARG
    bad = ch.copy()
    bad[1], bad[2] = bad[2], bad[1]  # not ascending
    with pytest.raises(hc.HcError) as e:
        hc.shard_plan(h, bad, 0, 1)
    assert e.value.status == hc.HC_ERR_CORRUPT
    bad = ch.copy()
    bad[-1] += 1  # does not end at the payload size
    with pytest.raises(hc.HcError) as e:
        hc.shard_plan(h, bad, 0, 1)
    assert e.value.status == hc.HC_ERR_CORRUPT
    with pytest.raises(ValueError):
        hc.shard_plan(h, ch[:-1], 0, 1)
    with pytest.raises(ValueError):
        hc.shard_range(4, 4, 4)


def test_limbs_round_trip_and_add_exactly():
    """The limb form of (s1, s2, n) adds limb by limb to the exact totals for
    any signs and sizes, including s2 near 2^128 spread over many ranks."""
    from paper_2603_25206_gb300 import shard

    rng = np.random.default_rng(3)
    parts = [(-(1 << 62), (1 << 127) // 64, 5), ((1 << 62) - 1, (1 << 126) // 64, 7), (0, 0, 0), (-1, 1, 1)]
    parts += [(int(rng.integers(-(1 << 60), 1 << 60)), int(rng.integers(0, 1 << 62)) << 60, int(rng.integers(0, 1 << 40)))
              for _ in range(60)]
    for s1, s2, n in parts:
        assert shard.from_limbs(shard.to_limbs(s1, s2, n)) == (s1, s2, n)
    summed = np.sum([shard.to_limbs(*p) for p in parts], axis=0, dtype=np.int64)
    want = (sum(p[0] for p in parts), sum(p[1] for p in parts), sum(p[2] for p in parts))
    assert shard.from_limbs(summed.tolist()) == want
    for bad in ((1 << 63, 0, 0), (0, 1 << 128, 0), (0, -1, 0), (0, 0, -1)):
        with pytest.raises(ValueError):
            shard.to_limbs(*bad)


def test_finalize_matches_the_oracle_bit_for_bit(orc, rng):
    from paper_2603_25206_gb300 import shard

    for _ in range(50):
        n = int(rng.integers(1, 1 << 30))
        q = rng.integers(-(1 << 29), 1 << 29, size=8)
        s1 = int(q.sum()) * (n // 8 + 1)
        s2 = int((q.astype(object) ** 2).sum()) * (n // 8 + 1) + int(rng.integers(0, 1 << 40))
        eps = float(rng.choice([1e-6, 3.3e-3, 0.5, 17.0]))
        if n * s2 < s1 * s1:
            s2 = (s1 * s1) // n + 1
        assert shard.finalize(n, s1, s2, eps)[:2] == orc.finalize(n, s1, s2, eps)[:2] or n < 2


def _rank_worker(rank, world, port, streams, eps, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist

    import oracle
    from paper_2603_25206_gb300 import shard

    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        s1, s2, n = 0, 0, 0
        for sh in streams[rank]:  # this rank's shards (one per field)
            qs = oracle.decode(sh, "q")
            a, b = oracle.sums_q(qs)
            s1, s2, n = s1 + a, s2 + b, n + qs.size
        tot = shard.allreduce_exact(s1, s2, n)
        out.put((rank, tot, shard.finalize(tot[2], tot[0], tot[1], eps)))
    finally:
        dist.destroy_process_group()


def test_gloo_ranks_combine_to_the_whole_field(hc, orc, rng):
    """Two gloo ranks each reduce their shard of one field (through the
    oracle, standing in for each rank's GPU) and combine exactly: both get
    the whole field's s1, s2 and N, and its mean and variance bit for bit."""
    import multiprocessing as mp
    import socket

    x = _field(rng, 30000, np.float32)
    s, eps = orc.compress(x, 1e-3, True, 32)
    h = _header_from_oracle_stream(hc, orc, s)
    chunks = _chunks(orc, s, h)
    world = 2
    streams = []
    for rank in range(world):
        c0, c1 = hc.shard_range(int(h.nchunks), rank, world)
        plan, rebased = hc.shard_plan(h, chunks, c0, c1)
        streams.append([_build_shard(s, plan, rebased)])
    q = orc.decode(s, "q")
    s1, s2 = orc.sums_q(q)
    want_stats = orc.finalize(q.size, s1, s2, eps)
    sock = socket.socket()
    sock.bind(("127.0.0.1", 0))
    port = sock.getsockname()[1]
    sock.close()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    ps = [ctx.Process(target=_rank_worker, args=(r, world, port, streams, eps, out)) for r in range(world)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(out.get(timeout=10) for _ in range(world))
    for rank, tot, stats in got:
        assert tot == (s1, s2, q.size)
        assert stats[:2] == want_stats[:2]


def test_binding_shard_builds_the_planned_streams(hc, orc, rng, monkeypatch):
    """hc.shard, run on CPU tensors (a stand-in replaces torch.cuda's stream
    calls), builds for every rank the stream the plan describes: the oracle
    decodes each to its slice of the codes, the slices tile the field in rank
    order, and a rank without chunks gets None."""
    import contextlib

    import torch

    class _Cuda:
        @staticmethod
        def current_stream(device=None):
            return None

        @staticmethod
        def stream(s):
            return contextlib.nullcontext()

    class _Torch:
        cuda = _Cuda

        def __getattr__(self, name):
            return getattr(torch, name)

    monkeypatch.setattr(hc, "_torch", lambda: _Torch())
    for pred in (0, 1):
        x = _field(rng, 4096 * 5 + 300, np.float32)
        s, eps = orc.compress(x, 1e-3, True, 32, pred=pred)
        h = _header_from_oracle_stream(hc, orc, s)
        c = hc.Compressed(torch.from_numpy(np.concatenate([s, np.zeros(64, np.uint8)])), h, int(s.size))
        q = orc.decode(s, "q").reshape(-1)
        for world in (1, 2, 4, 9):
            pos = 0
            for rank in range(world):
                sh = hc.shard(c, rank, world)
                c0, c1 = hc.shard_range(int(h.nchunks), rank, world)
                if c1 <= c0:
                    assert sh is None
                    continue
                b = sh.stream.numpy()
                assert b.size == sh.nbytes == int(sh.header.total_bytes)
                assert orc.read_header(b)["N"] == int(sh.header.N)
                qs = orc.decode(b, "q")
                np.testing.assert_array_equal(qs, q[pos:pos + qs.size])
                pos += qs.size
            assert pos == q.size
