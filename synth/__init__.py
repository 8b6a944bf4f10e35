"""Seeded synthetic scientific fields.

This module only draws inputs: it holds none of the compressor's or the
operations' arithmetic.  The same arrays feed the CPU oracle and the CUDA
library.  They stand in for the paper's datasets (Ocean, Miranda, Hurricane,
NYX, JHTDB; Table 3), which are not available here.

Recipes
-------
* ``sinusoid_field``: a sum of 8 random plane sinusoids (amplitudes U(0.5, 1),
  integer wave vectors in [1, 4]^d, phases U(0, 2 pi)), min-max normalised to
  [0, 1], plus N(0, 0.01^2) noise, normalised again.
* ``grf_field``: a Gaussian random field with power spectrum ~ k^-3 (white
  noise filtered by k^-1.5 in Fourier space, k = 0 removed), standardised,
  plus sparse spikes on 5% of the points (+-U(3, 10) standard deviations),
  min-max normalised to [0, 1].
* ``wide_field``: the k^-3 field times 1e4 plus a linear trend 1e4 * i0/n0
  along the slowest axis, in float64.
* ``grf_field_device``: the ``grf_field`` recipe drawn on a CUDA device with
  torch's seeded CUDA generator (for workloads too large to draw on the host,
  such as the 200-field serving set); the same spectrum and spikes, but not
  the same numbers as the host generator.
* ``wide_field_device``: the ``wide_field`` recipe drawn on a CUDA device
  (float64), for the benchmark's wide-code configuration.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["sinusoid_field", "grf_field", "grf_field_device", "wide_field", "wide_field_device", "log_uniform_shapes",
           "PAPER_SHAPES"]

# Shapes of the paper-like workload: Hurricane-like, NYX-like, Miranda-like,
# a 98 x 1200 x 1200 volume and a 1800 x 3600 (2-D) ocean-like slice.
PAPER_SHAPES = ((100, 500, 500), (512, 512, 512), (256, 384, 384), (98, 1200, 1200), (1800, 3600))


def _minmax(a: np.ndarray) -> np.ndarray:
    lo, hi = a.min(), a.max()
    if hi > lo:
        a = (a - lo) / (hi - lo)
    return a


def sinusoid_field(shape, seed: int = 1, noise_seed: int = 2, waves: int = 8, sigma: float = 0.01,
                   dtype=np.float32) -> np.ndarray:
    rng = np.random.default_rng(seed)
    nd = len(shape)
    grids = np.meshgrid(*[np.arange(n, dtype=np.float64) / n for n in shape], indexing="ij")
    acc = np.zeros(shape, np.float64)
    for _ in range(waves):
        a = rng.uniform(0.5, 1.0)
        f = rng.integers(1, 5, size=nd)
        ph = rng.uniform(0.0, 2 * math.pi)
        arg = sum(2 * math.pi * f[i] * grids[i] for i in range(nd)) + ph
        acc += a * np.sin(arg)
    acc = _minmax(acc)
    acc += np.random.default_rng(noise_seed).normal(0.0, sigma, size=shape)
    return np.ascontiguousarray(_minmax(acc).astype(dtype))


def _grf(shape, seed: int) -> np.ndarray:
    """Standardised k^-3 Gaussian random field in float64."""
    import torch  # CPU FFT only; faster than numpy's complex128 path for large volumes

    rng = np.random.default_rng(seed)
    white = torch.from_numpy(rng.standard_normal(size=shape, dtype=np.float32))
    spec = torch.fft.rfftn(white)
    del white
    k2 = None
    for ax, n in enumerate(shape):
        if ax == len(shape) - 1:
            f = torch.fft.rfftfreq(n, d=1.0 / n)
        else:
            f = torch.fft.fftfreq(n, d=1.0 / n)
        view = [1] * len(shape)
        view[ax] = -1
        f2 = (f.to(torch.float32) ** 2).reshape(view)
        k2 = f2 if k2 is None else k2 + f2
    amp = torch.where(k2 > 0, k2.clamp_min(1e-12) ** -0.75, torch.zeros((), dtype=torch.float32))
    spec *= amp
    del amp, k2
    field = torch.fft.irfftn(spec, s=shape).numpy().astype(np.float64)
    del spec
    field -= field.mean()
    sd = field.std()
    if sd > 0:
        field /= sd
    return field


def grf_field(shape, seed: int, spikes: float = 0.05, dtype=np.float32) -> np.ndarray:
    field = _grf(tuple(int(s) for s in shape), seed)
    if spikes > 0:
        rng = np.random.default_rng(seed + 500000)
        mask = rng.random(field.shape) < spikes
        amp = rng.uniform(3.0, 10.0, size=int(mask.sum())) * rng.choice((-1.0, 1.0), size=int(mask.sum()))
        field[mask] += amp
    return np.ascontiguousarray(_minmax(field).astype(dtype))


def _grf_device(shape, device, g):
    """Standardised k^-3 Gaussian random field in float64 on a CUDA device,
    white noise drawn from the seeded generator g."""
    import torch

    white = torch.randn(shape, generator=g, device=device, dtype=torch.float32)
    spec = torch.fft.rfftn(white)
    del white
    k2 = None
    for ax, n in enumerate(shape):
        f = (torch.fft.rfftfreq(n, d=1.0 / n) if ax == len(shape) - 1 else torch.fft.fftfreq(n, d=1.0 / n))
        view = [1] * len(shape)
        view[ax] = -1
        f2 = (f.to(device=device, dtype=torch.float32) ** 2).reshape(view)
        k2 = f2 if k2 is None else k2 + f2
    spec *= torch.where(k2 > 0, k2.clamp_min(1e-12) ** -0.75, torch.zeros((), device=device))
    del k2
    field = torch.fft.irfftn(spec, s=shape).to(torch.float64)
    del spec
    field -= field.mean()
    sd = field.std()
    if sd > 0:
        field /= sd
    return field


def grf_field_device(shape, seed: int, device, spikes: float = 0.05):
    """k^-3 Gaussian random field (+ spikes) as a float32 CUDA tensor in [0, 1]."""
    import torch

    shape = tuple(int(s) for s in shape)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    field = _grf_device(shape, device, g)
    if spikes > 0:
        mask = torch.rand(shape, generator=g, device=device) < spikes
        amp = torch.rand(shape, generator=g, device=device, dtype=torch.float64) * 7.0 + 3.0
        sign = torch.where(torch.rand(shape, generator=g, device=device) < 0.5, -1.0, 1.0).to(torch.float64)
        field += torch.where(mask, amp * sign, torch.zeros((), device=device, dtype=torch.float64))
        del mask, amp, sign
    lo, hi = field.min(), field.max()
    if hi > lo:
        field = (field - lo) / (hi - lo)
    return field.to(torch.float32).contiguous()


def wide_field(shape, seed: int) -> np.ndarray:
    field = _grf(tuple(int(s) for s in shape), seed) * 1e4
    n0 = shape[0]
    trend = 1e4 * (np.arange(n0, dtype=np.float64) / n0)
    field += trend.reshape((n0,) + (1,) * (len(shape) - 1))
    return np.ascontiguousarray(field)


def wide_field_device(shape, seed: int, device):
    """The ``wide_field`` recipe drawn on a CUDA device (float64 tensor): the
    same spectrum, scale and trend, not the same numbers as the host draw."""
    import torch

    shape = tuple(int(s) for s in shape)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    field = _grf_device(shape, device, g) * 1e4
    n0 = shape[0]
    trend = 1e4 * (torch.arange(n0, device=device, dtype=torch.float64) / n0)
    field += trend.reshape((n0,) + (1,) * (len(shape) - 1))
    return field.contiguous()


def log_uniform_shapes(count: int, lo: int, hi: int, seed: int, ndim: int = 3):
    """Shapes whose every axis is drawn log-uniformly from [lo, hi]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        out.append(tuple(int(round(math.exp(rng.uniform(math.log(lo), math.log(hi))))) for _ in range(ndim)))
    return out
