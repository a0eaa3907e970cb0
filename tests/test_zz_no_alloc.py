"""lf2_energy_noalloc: the energy reduction for callers that cannot allocate device memory.

Callers whose device allocator is owned by someone else (a memory pool or a host framework
that forbids cudaMalloc while it runs) cannot use lf2_energy, which allocates its scratch on
first use.  lf2_energy_noalloc keeps that scratch in a fixed array inside the library.  These
tests call it through the C ABI several times in a row, on lattices and precisions chosen so
that each call runs on top of the previous call's leftovers, and check each result against
lf2_energy: bitwise, since both run the same reduction in the same order, and, once, against
the FP64 oracle's energy with the parity tests' tolerance.  One lattice (64^3 = 262,144 sites)
is large enough for the reduction to use all 608 partial rows of the array.  This file is
collected last.
"""
import numpy as np
import pytest

from paper_1508_05610_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12
FIELDS = ("kinetic", "gradient", "potential", "total", "sum", "sum_sq")


@pytest.fixture(scope="module")
def lf2():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1508_05610_gb300 import build, lf2 as binding
    build.build()
    binding.load()
    return binding


def same_bits(a, b):
    for key in FIELDS:
        assert np.array_equal(np.asarray(a[key]), np.asarray(b[key])), key


def test_energy_noalloc_matches_energy_on_calls_in_a_row(lf2):
    kw = dict(dx=1.0, dt=0.05, lam=1.0, eta=1.0, m2=0.0)
    p = lf2.params(**kw)
    # the 64^3 lattice fills all 608 partial rows; the small ones after it use fewer, so the
    # rows they leave alone still hold the larger call's values
    cases = [((64, 64, 64), 2, "f64", 5), ((64, 48, 40), 2, "f64", 7), ((24, 16, 12), 1, "f32k", 3),
             ((64, 64, 64), 1, "f32k", 4)]
    for (shape, ncomp, prec, steps) in cases:
        nx, ny, nz = shape
        phi0 = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.3, seed=41 + ncomp + nx)
        with lf2.System(shape, ncomp, prec) as s:
            s.upload(phi0, np.zeros_like(phi0))
            lf2.lf2_leapfrog_init(s.phi, s.pi, p)
            lf2.lf2_leapfrog(s.phi, s.pi, p, steps)
            got = lf2.lf2_energy_noalloc(s.phi, s.pi, p, ncomp=ncomp)
            again = lf2.lf2_energy_noalloc(s.phi, s.pi, p, ncomp=ncomp)
            want = lf2.lf2_energy(s.phi, s.pi, p, ncomp=ncomp)
        same_bits(got, want)
        same_bits(again, want)


def test_energy_noalloc_matches_the_oracle(lf2, ora):
    """64^3 complex FP64 after 6 steps: the fixed-array energy within 1e-12 of the oracle's."""
    kw = dict(dx=1.0, dt=0.05, lam=1.0, eta=1.0, m2=0.0)
    p = lf2.params(**kw)
    phi0 = inputs.gaussian_field(64, 64, 64, 2, sigma=0.3, seed=77)
    pi0 = np.zeros_like(phi0)
    with lf2.System((64, 64, 64), 2, "f64") as s:
        s.upload(phi0, pi0)
        lf2.lf2_leapfrog_init(s.phi, s.pi, p)
        lf2.lf2_leapfrog(s.phi, s.pi, p, 6)
        got = lf2.lf2_energy_noalloc(s.phi, s.pi, p, ncomp=2)
    ophi, opi = ora.evolve(phi0, pi0, 6, half_kick=True, **kw)
    want = ora.energy(ophi, opi, **kw)
    for key in ("kinetic", "gradient", "potential", "total"):
        assert abs(got[key] - want[key]) <= TOL * abs(want["total"]), key
    for a in range(2):
        assert abs(got["sum_sq"][a] - want["sum_sq"][a]) <= TOL * want["sum_sq"][a]
