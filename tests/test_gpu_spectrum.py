"""GPU power spectrum (cuFFT transform, own binning) against the oracle's numpy-FFT spectrum,
and the Gaussian-random-field initial condition checked through it."""
import math

import numpy as np
import pytest

from paper_1508_05610_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lf2():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1508_05610_gb300 import build, lf2 as binding
    build.build()
    binding.load()
    return binding


@pytest.mark.parametrize("prec,n,ncomp,comp,tol", [("f64", 16, 2, 1, 1e-12), ("f32", 20, 1, 0, 1e-5),
                                                   ("f64", 15, 1, 0, 1e-12),
                                                   # comp = -1: the components' powers summed
                                                   ("f64", 16, 2, -1, 1e-12), ("f32k", 12, 3, -1, 1e-5),
                                                   ("f64", 10, 6, -1, 1e-12)])
def test_spectrum_matches_oracle(lf2, ora, prec, n, ncomp, comp, tol):
    phi = inputs.gaussian_field(n, n, n, ncomp, sigma=1.0, seed=141)
    nbins = 20
    with lf2.System((n, n, n), ncomp, prec) as s:
        lf2.lf2_field_upload(s.phi, phi)
        stored = lf2.lf2_field_download(s.phi, s.host_shape)
        P, K, C = lf2.lf2_power_spectrum(s.phi, comp=comp, nbins=nbins, dx=0.8)
    oP, oK, oC = ora.power_spectrum(stored, comp=comp, nbins=nbins, dx=0.8)
    assert np.array_equal(C, oC)
    assert np.max(np.abs(P - oP)) <= tol * np.max(oP)
    assert np.max(np.abs(K - oK)) <= 1e-12 * np.max(oK)


def test_spectrum_rejects_non_cubic(lf2):
    with lf2.System((16, 16, 8), 1, "f64") as s:
        with pytest.raises(lf2.LF2Error) as e:
            lf2.lf2_power_spectrum(s.phi)
        assert e.value.status == lf2.LF2_ERR_UNSUPPORTED
    with lf2.System((8, 8, 8), 2, "f64") as s:
        for comp in (-2, 2):
            with pytest.raises(lf2.LF2Error) as e:
                lf2.lf2_power_spectrum(s.phi, comp=comp)
            assert e.value.status == lf2.LF2_ERR_INVALID, comp


def test_grf_initial_condition_has_the_requested_spectrum(lf2):
    """The Gaussian random field initial condition: P(k) ~ k^-2 for 0 < |k| <= pi/4 and no
    power above the cut (up to rounding), checked on the device at 128^3."""
    import torch
    n = 128
    phi = inputs.grf_field_device(n, sigma=0.1, seed=inputs.BASE_SEED)
    lat = lf2.lf2_lattice_create((n, n, n))
    f = lf2.lf2_field_wrap(lat, 1, lf2.LF2_F64, [phi.data_ptr()])
    try:
        P, K, C = lf2.lf2_power_spectrum(f, nbins=n // 2)
    finally:
        lf2.lf2_field_free(f)
        lf2.lf2_lattice_destroy(lat)
    assert abs(float(phi.std()) - 0.1) < 1e-9
    kcut = math.pi / 4
    inside = (K > 0) & (K < kcut * 0.97) & (C > 0)
    above = (K > kcut * 1.03) & (C > 0)
    slope = np.polyfit(np.log(K[inside]), np.log(P[inside]), 1)[0]
    assert -2.15 < slope < -1.85, slope
    assert np.max(P[above]) < 1e-20 * np.max(P[inside])
    assert P[0] < 1e-20 * np.max(P[inside])  # the k = 0 mode is removed
    del phi
    torch.cuda.empty_cache()
