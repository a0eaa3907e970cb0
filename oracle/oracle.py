"""FP64 CPU oracle for the leapfrog lattice-field step -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this module; the
library never imports it.  It wraps ``lf2_oracle.c`` (plain C, FP64) with ctypes and
compiles it with gcc on first use.  See the header of ``lf2_oracle.c`` for the model it
follows (LATfield2's Lattice/Field/Site/updateHalo, Sec. 3.2-3.4 of arXiv:1508.05610) and
the readings it takes where the paper is silent (equation of motion, staggered leapfrog,
energy).

Arrays are numpy float64, shaped ``(nz, ny, nx, ncomp)``: row-major with x fastest and
the components of a site next to each other.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lf2_oracle.c")
_LIB = os.path.join(_HERE, "liblf2_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (-O2, no fast-math, OpenMP if available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-o", _LIB + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            i = ctypes.c_int
            lib.ora_update_halo.argtypes = [i, i, i, i, dp]
            lib.ora_force.argtypes = [i, i, i, i, dp, dp, dp]
            lib.ora_evolve.argtypes = [i, i, i, i, dp, dp, dp, i, i, i]
            lib.ora_energy.argtypes = [i, i, i, i, dp, dp, dp, dp]
            lib.ora_derivative.argtypes = [i, i, i, i, i, ctypes.c_double, dp, dp]
            for f in (lib.ora_update_halo, lib.ora_force, lib.ora_evolve, lib.ora_energy, lib.ora_derivative):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _field(a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if a.ndim == 3:
        a = a[..., None]
    if a.ndim != 4:
        raise ValueError("field arrays are (nz, ny, nx[, ncomp])")
    return a.copy()


def _params(dx, dt, lam, eta, m2) -> np.ndarray:
    return np.array([dx, dt, lam, eta, m2], dtype=np.float64)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def update_halo(padded: np.ndarray) -> np.ndarray:
    """Fills the one-site halo of a padded (nz+2, ny+2, nx+2, ncomp) array (Sec. 3.3.1)."""
    a = _field(padded)
    nz, ny, nx, c = a.shape
    _check(_load().ora_update_halo(nx - 2, ny - 2, nz - 2, c, _ptr(a)), "update_halo")
    return a


def force(phi, dx=1.0, dt=0.0, lam=1.0, eta=1.0, m2=0.0) -> np.ndarray:
    """F_a(x) = lap phi_a - lambda phi_a (|phi|^2 - eta^2) - m2 phi_a at every site."""
    a = _field(phi)
    nz, ny, nx, c = a.shape
    out = np.empty_like(a)
    _check(_load().ora_force(nx, ny, nz, c, _ptr(_params(dx, dt, lam, eta, m2)), _ptr(a), _ptr(out)),
           "force")
    return out


def evolve(phi, pi, nsteps, dx=1.0, dt=0.1, lam=1.0, eta=1.0, m2=0.0, half_kick=False, threads=1):
    """Runs ``nsteps`` staggered-leapfrog steps; returns (phi_n, pi_{n-1/2}).

    With ``half_kick`` the given pi is pi_0 and is first turned into pi_{-1/2}.
    ``threads`` > 1 splits the site loops over z-planes (bitwise-identical results)."""
    a, b = _field(phi), _field(pi)
    if a.shape != b.shape:
        raise ValueError("phi and pi shapes differ")
    nz, ny, nx, c = a.shape
    rc = _load().ora_evolve(nx, ny, nz, c, _ptr(_params(dx, dt, lam, eta, m2)), _ptr(a), _ptr(b),
                            int(nsteps), 1 if half_kick else 0, int(threads))
    _check(rc, "evolve")
    return a, b


def energy(phi, pi, dx=1.0, dt=0.1, lam=1.0, eta=1.0, m2=0.0) -> dict:
    """Energy at integer step n from phi_n and pi_{n-1/2}, plus per-component checksums."""
    a, b = _field(phi), _field(pi)
    nz, ny, nx, c = a.shape
    out = np.zeros(4 + 2 * c, dtype=np.float64)
    _check(_load().ora_energy(nx, ny, nz, c, _ptr(_params(dx, dt, lam, eta, m2)), _ptr(a), _ptr(b),
                              _ptr(out)), "energy")
    return {"kinetic": out[0], "gradient": out[1], "potential": out[2], "total": out[3],
            "sum": out[4:4 + c].copy(), "sum_sq": out[4 + c:4 + 2 * c].copy()}


def derivative(phi, dim, dx=1.0) -> np.ndarray:
    """(phi_a(x + i) - phi_a(x - i)) / (2 dx) along dimension dim (0 = x) for every component."""
    a = _field(phi)
    nz, ny, nx, c = a.shape
    out = np.empty_like(a)
    _check(_load().ora_derivative(nx, ny, nz, c, int(dim), float(dx), _ptr(a), _ptr(out)), "derivative")
    return out


def power_spectrum(phi, comp=0, nbins=32, dx=1.0):
    """Binned power spectrum of one component of a field on a cubic N^3 lattice (the paper's FFT
    is for cubic lattices, Sec. 3.6): P(k) = |phi~(k)|^2 / V with phi~(k) = sum_x phi(x)
    exp(-i k.x), k_i = 2 pi m_i / (N dx) for the signed integer frequency m_i.  comp = -1 sums
    the components' powers, sum_a |phi~_a(k)|^2 / V.  Mode (m_x, m_y, m_z) belongs to bin
    b = floor(sqrt(m_x^2 + m_y^2 + m_z^2)) (an exact integer square root).  Returns (mean power,
    mean |k|, mode count) per bin b < nbins.  numpy's FFT is the transform; the binning is a
    plain loop over the modes of the full spectrum."""
    f = _field(phi)
    comps = range(f.shape[-1]) if comp == -1 else [comp]
    nz, ny, nx = f.shape[:3]
    if not nx == ny == nz:
        raise ValueError("the power spectrum is defined for cubic lattices")
    n = nx
    V = n ** 3
    F2 = sum(np.abs(np.fft.fftn(f[..., a])) ** 2 for a in comps)
    m = [int(v) for v in np.fft.fftfreq(n) * n]
    power = np.zeros(nbins)
    ksum = np.zeros(nbins)
    count = np.zeros(nbins)
    for iz in range(n):
        for iy in range(n):
            for ix in range(n):
                s2 = m[ix] ** 2 + m[iy] ** 2 + m[iz] ** 2
                b = math.isqrt(s2)
                if b < nbins:
                    power[b] += F2[iz, iy, ix] / V
                    ksum[b] += 2 * math.pi / (n * dx) * math.sqrt(s2)
                    count[b] += 1
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(count > 0, power / count, 0.0), np.where(count > 0, ksum / count, 0.0), count


def light_cone_box(field: np.ndarray, center, half: int) -> np.ndarray:
    """Cuts the (2 half + 1)^3 box of a periodic field centred on ``center`` = (x, y, z).

    After n <= half - 1 steps the value at the centre of a periodic evolution of this box equals
    the value at ``center`` of the evolution of the whole lattice: information moves one site
    per step, so the wrap-around seam of the box never reaches its centre in time.  This lets
    the oracle check single sites of lattices far too large for it."""
    nz, ny, nx = field.shape[:3]
    cx, cy, cz = center
    r = np.arange(-half, half + 1)
    zi = (cz + r) % nz
    yi = (cy + r) % ny
    xi = (cx + r) % nx
    return np.ascontiguousarray(field[np.ix_(zi, yi, xi)])
