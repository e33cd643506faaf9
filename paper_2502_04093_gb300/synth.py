"""Seeded synthetic fields shaped like the IPComp paper's workloads.

The paper (Sec. 6.1, Table 3) evaluates on FP64 turbulence, weather, seismic
and combustion fields of 100-1008 points per dimension. Those datasets are not
available here, so these generators stand in for them. This module holds no
part of the compression method: it only draws inputs. Both the CUDA path and
the CPU oracle consume the arrays it returns.

Workloads (one generator each):

* ``gaussians3d``  -- 64^3 f32, sum of 8 random 3-D Gaussians + 1e-3 noise.
* ``grf_k53``      -- Gaussian random field with a k^-5/3 power spectrum
  (amplitude k^-5/6, uniform phases, inverse real FFT), min-max normalised to
  [0, 1]; the 512^3 f32 roofline field and the serving fields.
* ``zonal2d``      -- smooth zonal bands + longitude modulation + noise, the
  uneven 2-D batch (1800x3600, 900x1800, 450x900).
* ``sinusoids3d``  -- sums of 8 integer-wavenumber sinusoids + 1e-4 noise,
  384x384x256 f64 (the paper's turbulence shape).
"""
from __future__ import annotations

import math

import numpy as np


def gaussians3d(shape=(64, 64, 64), n=8, seed=1001, noise=1e-3, dtype=np.float32):
    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in shape)
    centers = rng.uniform(0, 1, size=(n, len(shape))) * np.array(shape)
    sigma = rng.uniform(4.0, 12.0, size=n)
    amp = rng.uniform(-1.0, 1.0, size=n)
    axes = [np.arange(s, dtype=np.float64) for s in shape]
    f = np.zeros(shape, dtype=np.float64)
    for j in range(n):
        g = np.ones(shape, dtype=np.float64)
        for e, ax in enumerate(axes):
            d = ax - centers[j, e]
            sh = [1] * len(shape)
            sh[e] = -1
            g = g * np.exp(-d * d / (2 * sigma[j] ** 2)).reshape(sh)
        f += amp[j] * g
    f += rng.normal(0.0, noise, size=shape)
    return f.astype(dtype)


def grf_k53(shape=(512, 512, 512), seed=1002, dtype=np.float32, device="cpu"):
    """k^-5/3 Gaussian random field via torch's FFT (CPU or CUDA).

    Returns a torch tensor on ``device`` (min-max normalised to [0, 1])."""
    import torch

    shape = tuple(int(s) for s in shape)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    half = shape[:-1] + (shape[-1] // 2 + 1,)
    ks = []
    for e, s in enumerate(shape):
        if e == len(shape) - 1:
            k = torch.arange(s // 2 + 1, device=device, dtype=torch.float32)
        else:
            k = torch.fft.fftfreq(s, d=1.0 / s, device=device).to(torch.float32)
        view = [1] * len(shape)
        view[e] = -1
        ks.append(k.view(view))
    k2 = torch.zeros(half, device=device, dtype=torch.float32)
    for k in ks:
        k2 = k2 + k * k
    kk = torch.sqrt(k2)
    kk[(0,) * len(shape)] = 1.0
    amp = kk.pow(-5.0 / 6.0)
    amp[(0,) * len(shape)] = 0.0
    del k2, kk
    phase = torch.rand(half, generator=gen, device=device, dtype=torch.float32)
    spec = torch.polar(amp, phase * (2 * math.pi))
    del amp, phase
    f = torch.fft.irfftn(spec, s=shape)
    del spec
    lo, hi = f.min(), f.max()
    f = (f - lo) / (hi - lo)
    tdt = torch.float32 if np.dtype(dtype) == np.float32 else torch.float64
    return f.to(tdt).contiguous()


def zonal2d(shape=(450, 900), seed=1300, dtype=np.float32):
    rng = np.random.default_rng(seed)
    H, W = int(shape[0]), int(shape[1])
    lat = np.arange(H, dtype=np.float64)[:, None]
    lon = np.arange(W, dtype=np.float64)[None, :]
    a = rng.uniform(-1.0, 1.0, size=6)
    phi = rng.uniform(0, 2 * math.pi, size=6)
    f = np.zeros((H, W))
    for j in range(6):
        f = f + a[j] * np.cos((j + 1) * math.pi * lat / H + phi[j])
    m = rng.integers(1, 6)
    psi = rng.uniform(0, 2 * math.pi)
    f = f + 0.1 * np.abs(a).max() * np.sin(2 * math.pi * m * lon / W + psi) * np.cos(math.pi * lat / H)
    amp = np.abs(a).sum()
    f = f + rng.normal(0.0, 1e-3 * amp, size=(H, W))
    return f.astype(dtype)


def zonal_batch(seed=1300, scale=1):
    """The 64-field uneven 2-D batch (16 x 1800x3600, 24 x 900x1800,
    24 x 450x900), shuffled. ``scale`` > 1 divides every edge (for tests)."""
    shapes = [(1800, 3600)] * 16 + [(900, 1800)] * 24 + [(450, 900)] * 24
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(shapes))
    shapes = [tuple(max(1, s // scale) for s in shapes[i]) for i in order]
    return shapes, [seed + j for j in range(len(shapes))]


def sinusoids3d(shape=(384, 384, 256), seed=1400, dtype=np.float64, nterms=8, kmax=8):
    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in shape)
    axes = [np.arange(s, dtype=np.float64) / s for s in shape]
    f = np.zeros(shape, dtype=np.float64)
    amps = rng.uniform(-1.0, 1.0, size=nterms)
    for j in range(nterms):
        k = rng.integers(-kmax, kmax + 1, size=len(shape))
        phi = rng.uniform(0, 2 * math.pi)
        arg = phi
        for e, ax in enumerate(axes):
            sh = [1] * len(shape)
            sh[e] = -1
            arg = arg + 2 * math.pi * k[e] * ax.reshape(sh)
        f += amps[j] * np.sin(arg)
    f += rng.normal(0.0, 1e-4 * np.abs(amps).sum(), size=shape)
    return f.astype(dtype)


def serving_edges(nfields=128, seed=1500, lo=128, hi=768, step=32):
    """Edges of the resident serving fields: log-uniform in [lo, hi], rounded
    to a multiple of ``step``."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(math.log(lo), math.log(hi), size=nfields)
    e = np.clip(np.round(np.exp(u) / step) * step, lo, hi).astype(int)
    return [int(v) for v in e]


def random_field(shape, seed, dtype=np.float32, kind="smooth"):
    """Small seeded test fields: 'smooth' (a few low-frequency modes + noise),
    'noise' (white), 'const', 'ramp', 'spiky' (smooth + rare huge spikes)."""
    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in shape)
    if kind == "noise":
        return rng.normal(0, 1, size=shape).astype(dtype)
    if kind == "const":
        return np.full(shape, rng.normal(), dtype=dtype)
    if kind == "ramp":
        idx = np.indices(shape).sum(axis=0).astype(np.float64)
        return (0.37 * idx - 3.0).astype(dtype)
    f = np.zeros(shape, dtype=np.float64)
    grids = np.indices(shape).astype(np.float64)
    for _ in range(4):
        arg = rng.uniform(0, 2 * math.pi)
        for e in range(len(shape)):
            arg = arg + rng.uniform(-0.4, 0.4) * grids[e]
        f += rng.uniform(-1, 1) * np.sin(arg)
    f += rng.normal(0, 1e-3, size=shape)
    if kind == "spiky":
        flat = f.reshape(-1)
        k = max(1, flat.size // 97)
        pos = rng.choice(flat.size, size=k, replace=False)
        flat[pos] = rng.choice([-1.0, 1.0], size=k) * 1e9
    return f.astype(dtype)


def zonal2d_torch(shape, seed, device="cuda"):
    """zonal2d drawn on the device (same recipe, for large batches)."""
    import torch

    rng = np.random.default_rng(seed)
    H, W = int(shape[0]), int(shape[1])
    a = rng.uniform(-1.0, 1.0, size=6)
    phi = rng.uniform(0, 2 * math.pi, size=6)
    m = int(rng.integers(1, 6))
    psi = float(rng.uniform(0, 2 * math.pi))
    lat = torch.arange(H, device=device, dtype=torch.float64)[:, None]
    lon = torch.arange(W, device=device, dtype=torch.float64)[None, :]
    f = torch.zeros((H, W), device=device, dtype=torch.float64)
    for j in range(6):
        f = f + float(a[j]) * torch.cos((j + 1) * math.pi * lat / H + float(phi[j]))
    f = f + 0.1 * float(np.abs(a).max()) * torch.sin(2 * math.pi * m * lon / W + psi) * \
        torch.cos(math.pi * lat / H)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    f = f + torch.randn((H, W), generator=gen, device=device, dtype=torch.float64) * \
        (1e-3 * float(np.abs(a).sum()))
    return f.to(torch.float32).contiguous()


def sinusoids3d_torch(shape=(384, 384, 256), seed=1400, device="cuda", nterms=8, kmax=8):
    """sinusoids3d drawn on the device in float64."""
    import torch

    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in shape)
    axes = [torch.arange(s, device=device, dtype=torch.float64) / s for s in shape]
    f = torch.zeros(shape, device=device, dtype=torch.float64)
    amps = rng.uniform(-1.0, 1.0, size=nterms)
    for j in range(nterms):
        k = rng.integers(-kmax, kmax + 1, size=len(shape))
        arg = torch.full((1,) * len(shape), float(rng.uniform(0, 2 * math.pi)), device=device,
                         dtype=torch.float64)
        for e, ax in enumerate(axes):
            sh = [1] * len(shape)
            sh[e] = -1
            arg = arg + 2 * math.pi * float(k[e]) * ax.reshape(sh)
        f += float(amps[j]) * torch.sin(arg)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    f += torch.randn(shape, generator=gen, device=device, dtype=torch.float64) * \
        (1e-4 * float(np.abs(amps).sum()))
    return f.contiguous()
