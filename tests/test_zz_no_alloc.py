"""lf2_energy_noalloc: the energy reduction for callers that cannot allocate device memory.

Callers whose device allocator is owned by someone else (a memory pool or a host framework
that forbids cudaMalloc while it runs) cannot use lf2_energy, which allocates its scratch on
first use.  lf2_energy_noalloc keeps that scratch in a fixed array inside the library.  This
test calls it through the C ABI twice in a row, on two different lattices and precisions so
that the second call runs on top of the first call's leftovers, and checks each result
against lf2_energy with the FP64 tolerance of the parity tests.  This file is collected last.
"""
import numpy as np
import pytest

from paper_1508_05610_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def lf2():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1508_05610_gb300 import build, lf2 as binding
    build.build()
    binding.load()
    return binding


def close(a, b):
    for key in ("kinetic", "gradient", "potential", "total"):
        assert abs(a[key] - b[key]) <= TOL * abs(b["total"]), key
    for key in ("sum", "sum_sq"):
        scale = max(float(np.max(np.abs(b["sum_sq"]))), 1.0)
        assert np.all(np.abs(a[key] - b[key]) <= TOL * scale), key


def test_energy_noalloc_matches_energy_on_two_calls_in_a_row(lf2):
    kw = dict(dx=1.0, dt=0.05, lam=1.0, eta=1.0, m2=0.0)
    p = lf2.params(**kw)
    cases = [((64, 48, 40), 2, "f64", 7), ((24, 16, 12), 1, "f32k", 3)]
    for (shape, ncomp, prec, steps) in cases:
        nx, ny, nz = shape
        phi0 = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.3, seed=41 + ncomp)
        with lf2.System(shape, ncomp, prec) as s:
            s.upload(phi0, np.zeros_like(phi0))
            lf2.lf2_leapfrog_init(s.phi, s.pi, p)
            lf2.lf2_leapfrog(s.phi, s.pi, p, steps)
            got = lf2.lf2_energy_noalloc(s.phi, s.pi, p, ncomp=ncomp)
            want = lf2.lf2_energy(s.phi, s.pi, p, ncomp=ncomp)
        close(got, want)
