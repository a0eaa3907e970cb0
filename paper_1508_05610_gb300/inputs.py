"""Seeded synthetic inputs for the leapfrog lattice-field step.

This module only draws random numbers and lays them out; it holds none of the method's
arithmetic, so that both the CUDA path and the FP64 CPU oracle can be fed the same bytes.

Layout of every field array: ``(nz, ny, nx, ncomp)``, row-major with x fastest and the
components of a site next to each other -- the row-major per-site component lists of
LATfield2's Site and binary I/O (arXiv:1508.05610, Sec. 3.4 and Sec. 3.5).

Random streams:
  * host arrays use numpy's counter-based Philox-4x32-10 bit generator (Salmon et al.,
    SC'11) keyed by the seed, then numpy's standard normal transform in FP64;
  * device arrays (lattices too large for the host path) use torch's seeded CUDA generator.
The two streams differ; a comparison always feeds one array to both sides (for large
lattices the oracle gets cut-out boxes of the device array, copied back to the host).
"""
from __future__ import annotations

import math

import numpy as np

BASE_SEED = 20150820


def rng(seed: int) -> np.random.Generator:
    """numpy Philox-4x32-10 stream keyed by ``seed``."""
    return np.random.Generator(np.random.Philox(key=int(seed)))


def gaussian_field(nx: int, ny: int, nz: int, ncomp: int, sigma: float = 0.1,
                   seed: int = BASE_SEED, mean: float = 0.0) -> np.ndarray:
    """i.i.d. Gaussian components, FP64, shape (nz, ny, nx, ncomp)."""
    g = rng(seed)
    return mean + sigma * g.standard_normal((nz, ny, nx, ncomp))


def integer_field(nx: int, ny: int, nz: int, ncomp: int, lo: int = -8, hi: int = 8,
                  seed: int = BASE_SEED) -> np.ndarray:
    """Integer-valued FP64 field with entries uniform in [lo, hi]; with dx = dt = 1 and no
    potential every operation of a step is exact, in FP64 and in FP32."""
    g = rng(seed)
    return g.integers(lo, hi + 1, size=(nz, ny, nx, ncomp)).astype(np.float64)


def gaussian_field_device(nx: int, ny: int, nz: int, ncomp: int, sigma: float = 0.1,
                          seed: int = BASE_SEED, dtype=None, device="cuda"):
    """i.i.d. Gaussian field generated on the device with torch's seeded generator.

    ``dtype`` defaults to torch.float64; for float32 the FP64 draw is rounded once, so the
    FP32 and FP64 runs of one seed start from the same values up to that rounding."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    out = torch.empty((nz, ny, nx, ncomp), dtype=dtype or torch.float64, device=device)
    plane = (ny, nx, ncomp)
    for z in range(nz):  # plane by plane: bounded FP64 temporaries for float32 output
        t = torch.randn(plane, generator=gen, dtype=torch.float64, device=device)
        out[z].copy_(t.mul_(sigma))
    return out


def grf_field_device(n: int, sigma: float = 0.1, seed: int = BASE_SEED, kcut: float = math.pi / 4,
                     spectral_index: float = -2.0, dtype=None, device="cuda"):
    """Real Gaussian random field on an n^3 lattice with power spectrum P(k) ~ k^index for
    0 < |k| <= kcut and 0 elsewhere, rescaled to real-space standard deviation ``sigma``.

    White noise -> FFT -> multiply by sqrt(P(|k|)) with k_i = 2 pi m_i / n (m_i the signed
    FFT frequency) -> inverse FFT.  Done once, off the timed path, with torch.fft in FP64."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    noise = torch.randn((n, n, n), generator=gen, dtype=torch.float64, device=device)
    spec = torch.fft.rfftn(noise)
    del noise
    kz = 2 * math.pi * torch.fft.fftfreq(n, device=device, dtype=torch.float64)
    kx = 2 * math.pi * torch.fft.rfftfreq(n, device=device, dtype=torch.float64)
    k2 = kz[:, None, None] ** 2 + kz[None, :, None] ** 2 + kx[None, None, :] ** 2
    k = torch.sqrt(k2)
    amp = torch.where((k > 0) & (k <= kcut), k.clamp_min(1e-300) ** (0.5 * spectral_index),
                      torch.zeros_like(k))
    del k2, k
    spec.mul_(amp)
    del amp
    field = torch.fft.irfftn(spec, s=(n, n, n))
    del spec
    field.mul_(sigma / field.std())
    return field.to(dtype or torch.float64).reshape(n, n, n, 1)


def ensemble_members(count: int = 64, sides=(64, 96, 128, 160, 192), lam_range=(0.5, 2.0),
                     seed: int = BASE_SEED + 1000):
    """Sides and couplings of a batched ensemble: each lattice is a cube whose side is drawn
    uniformly from ``sides`` and whose lambda is uniform in ``lam_range``.  Returns a list of
    (side, lambda, field_seed) with per-lattice field seeds BASE_SEED + index."""
    g = rng(seed)
    side = g.choice(np.asarray(sides), size=count)
    lam = g.uniform(lam_range[0], lam_range[1], size=count)
    return [(int(side[i]), float(lam[i]), BASE_SEED + i) for i in range(count)]
