"""Exact combination of the statistics of a field reduced in parts by
several ranks (hc.shard gives each rank its chunks as a stream of its own).

Section V-A's statistics come from two integer sums, s1 = sum q (int64) and
s2 = sum q^2 (up to 128 bits), and the count N.  Sums over a partition of the
blocks add up exactly, so the ranks' totals need one all-reduce of integers:
s1 is split into a signed high and an unsigned low 32-bit half, s2 into four
unsigned 32-bit limbs, each rank's limbs are summed as int64 (no overflow for
fewer than 2^31 ranks), and the carries are resolved in Python integers.  The
result does not depend on the order of the ranks, the backend or the
partition: every rank gets the whole field's s1 and s2 bit for bit, and
`finalize` has the library scale them (hc_finalize: the arithmetic of its
own last-CTA finish), so the mean, variance and std equal a one-GPU
reduction's.
"""
from __future__ import annotations

LIMB = 32
_MASK = (1 << LIMB) - 1
N_LIMBS = 7  # s1 (2), s2 (4), n (1)


def to_limbs(s1: int, s2: int, n: int) -> list:
    """(s1, s2, n) as seven integers that fit int64 and add limb by limb."""
    if not (-(1 << 63) <= s1 < (1 << 63)) or not (0 <= s2 < (1 << 128)) or not (0 <= n < (1 << 62)):
        raise ValueError("s1 must fit int64, s2 128 bits unsigned, n 62 bits")
    return [s1 & _MASK, s1 >> LIMB] + [(s2 >> (LIMB * k)) & _MASK for k in range(4)] + [n]


def from_limbs(limbs) -> tuple:
    """Inverse of to_limbs after the limbs of several ranks were added."""
    limbs = [int(v) for v in limbs]
    if len(limbs) != N_LIMBS:
        raise ValueError(f"expected {N_LIMBS} limbs")
    s1 = limbs[0] + (limbs[1] << LIMB)
    s2 = sum(v << (LIMB * k) for k, v in enumerate(limbs[2:6]))
    return s1, s2, limbs[6]


def allreduce_exact(s1: int, s2: int, n: int, group=None, device=None) -> tuple:
    """Sum (s1, s2, n) over the ranks of `group` exactly (one all-reduce of
    int64 limbs).  `device`: where the limb tensor lives (the CPU for gloo,
    the rank's GPU for nccl)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor(to_limbs(s1, s2, n), dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return from_limbs(t.cpu().tolist())


def finalize(n: int, s1: int, s2: int, eps: float) -> tuple:
    """(mean, variance, std) from the exact sums (Eq. var_q), scaled by the
    library (hc_finalize, host code with the device finish's arithmetic and
    roundings), so they equal a one-launch reduction's bit for bit.  N < 2
    gives NaN variance and std."""
    from . import hc

    r = hc.finalize(n, s1, s2, eps)
    return r["mean"], r["variance"], r["std"]
