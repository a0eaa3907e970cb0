"""GPU: lf2_field_compare, the device-side error norms of the FP32-vs-FP64 error measurement.

Checked against numpy on the same arrays: the maxima exactly, the sums of squares to FP64
rounding; NaN propagation; compensation buffers; argument and state errors.
"""
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


def numpy_norms(a, ref):
    d = a.astype(np.float64) - ref.astype(np.float64)
    return np.max(np.abs(d)), np.max(np.abs(ref)), np.sum(d * d), np.sum(ref.astype(np.float64) ** 2)


@pytest.mark.parametrize("shape,ncomp,prec,ref_dtype", [
    ((3, 4, 5), 1, "f64", np.float64),
    ((40, 16, 9), 2, "f32k", np.float64),
    ((64, 24, 33), 3, "f32", np.float32),
    ((96, 96, 96), 1, "f32k", np.float64),   # more elements than threads of the largest grid
    ((80, 64, 48), 2, "f64", np.float32),
])
def test_compare_matches_numpy(lf2, shape, ncomp, prec, ref_dtype):
    import torch
    nx, ny, nz = shape
    phi = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.3, seed=inputs.BASE_SEED + 91)
    ref = phi + inputs.gaussian_field(nx, ny, nz, ncomp, sigma=1e-6, seed=inputs.BASE_SEED + 92)
    ref = ref.astype(ref_dtype)
    ref_dev = torch.from_numpy(np.ascontiguousarray(ref)).cuda()
    ref_prec = lf2.LF2_F64 if ref_dtype == np.float64 else lf2.LF2_F32
    with lf2.System(shape, ncomp, prec) as s:
        s.upload(phi, np.zeros_like(phi))
        got = lf2.lf2_field_compare(s.phi, ref_dev.data_ptr(), ref_prec)
        stored, _ = s.download()  # the values the field holds (rounded to float for FP32 storage)
    want = numpy_norms(stored, ref)
    assert got["max_abs_diff"] == want[0]
    assert got["max_abs_ref"] == want[1]
    assert abs(got["sum_sq_diff"] - want[2]) <= 1e-12 * want[2]
    assert abs(got["sum_sq_ref"] - want[3]) <= 1e-12 * want[3]
    assert got["relmax"] == want[0] / want[1]


def wide_range_f32(shape, seed):
    """FP32 values over the whole finite range below 2^21: exponents -150..20 (subnormals
    included), plus +0 and -0, returned as their exact FP64 images."""
    rng = np.random.default_rng(seed)
    v = np.ldexp(rng.standard_normal(shape), rng.integers(-150, 21, shape)).astype(np.float32)
    v.flat[::17] = 0.0
    v.flat[5::29] = -0.0
    return v.astype(np.float64)


@pytest.mark.parametrize("prec,ref_dtype", [("f32", np.float64), ("f32k", np.float64), ("f64", np.float32),
                                            ("f32", np.float32)])
def test_float_to_double_widening_is_exact(lf2, prec, ref_dtype):
    """The FP32 values the comparison kernel reads are widened to FP64 exactly, over every
    exponent (normal and subnormal) and both signed zeros: against the exact images the
    difference is zero everywhere, and the maximum |ref| is the exact one."""
    import torch
    shape, ncomp = (40, 16, 9), 2
    v = wide_range_f32(shape + (ncomp,), inputs.BASE_SEED + 95)
    f32 = v.astype(np.float32)
    assert np.count_nonzero((f32 != 0) & (np.abs(f32) < np.finfo(np.float32).tiny)) > 100
    assert np.count_nonzero(np.signbit(f32) & (f32 == 0)) > 0
    ref = torch.from_numpy(np.ascontiguousarray(v.astype(ref_dtype))).cuda()
    ref_prec = lf2.LF2_F64 if ref_dtype == np.float64 else lf2.LF2_F32
    with lf2.System(shape, ncomp, prec) as s:
        s.upload(v, np.zeros_like(v))
        stored, _ = s.download()
        got = lf2.lf2_field_compare(s.phi, ref.data_ptr(), ref_prec)
    assert np.array_equal(stored.ravel(), v.ravel())  # upload and download are exact
    assert got["max_abs_diff"] == 0.0 and got["sum_sq_diff"] == 0.0
    assert got["max_abs_ref"] == np.max(np.abs(v))
    assert abs(got["sum_sq_ref"] - np.sum(v * v)) <= 1e-12 * np.sum(v * v)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_widening_of_infinities_and_nan(lf2, prec):
    """FP32 infinities widen to FP64 infinities and a NaN to a NaN: against zeros the largest
    difference is inf, then NaN once a NaN is stored."""
    import torch
    v = np.zeros((8, 8, 8, 1))
    v.flat[100], v.flat[200] = np.inf, -np.inf
    zeros = torch.zeros(512, dtype=torch.float32, device="cuda")
    with lf2.System((8, 8, 8), 1, prec) as s:
        s.upload(v, np.zeros_like(v))
        inf = lf2.lf2_field_compare(s.phi, zeros.data_ptr(), lf2.LF2_F32)
        v.flat[300] = np.nan
        s.upload(v, np.zeros_like(v))
        nan = lf2.lf2_field_compare(s.phi, zeros.data_ptr(), lf2.LF2_F32)
    assert inf["max_abs_diff"] == np.inf and inf["sum_sq_diff"] == np.inf and inf["max_abs_ref"] == 0.0
    assert np.isnan(nan["max_abs_diff"]) and np.isnan(nan["sum_sq_diff"])


def test_compare_identical_is_zero_and_nan_propagates(lf2):
    import torch
    phi = inputs.gaussian_field(16, 8, 6, 2, sigma=0.3, seed=inputs.BASE_SEED + 93)
    ref = torch.from_numpy(phi.copy()).cuda()
    with lf2.System((16, 8, 6), 2, "f64") as s:
        s.upload(phi, np.zeros_like(phi))
        same = lf2.lf2_field_compare(s.phi, ref.data_ptr(), lf2.LF2_F64)
        assert same["max_abs_diff"] == 0.0 and same["sum_sq_diff"] == 0.0
        assert same["sum_sq_ref"] > 0
        ref.view(-1)[777] = float("nan")
        bad = lf2.lf2_field_compare(s.phi, ref.data_ptr(), lf2.LF2_F64)
        assert np.isnan(bad["max_abs_diff"]) and np.isnan(bad["max_abs_ref"])


def test_compare_compensation_buffer_and_errors(lf2):
    import torch
    phi = inputs.gaussian_field(8, 8, 8, 1, sigma=0.3, seed=inputs.BASE_SEED + 94)
    zeros32 = torch.zeros(8 * 8 * 8, dtype=torch.float32, device="cuda")
    p = lf2.params(dx=1.0, dt=0.1, lam=1.0, eta=1.0, m2=0.0)
    with lf2.System((8, 8, 8), 1, "f32k") as s:
        s.upload(phi, np.zeros_like(phi))
        # the compensation and the back buffers are allocated by the first step
        for f, which in ((s.phi, 2), (s.pi, 1)):
            with pytest.raises(lf2.LF2Error) as e:
                lf2.lf2_field_compare(f, zeros32.data_ptr(), lf2.LF2_F32, which=which)
            assert e.value.status == lf2.LF2_ERR_STATE
        lf2.lf2_leapfrog_init(s.phi, s.pi, p)
        lf2.lf2_leapfrog(s.phi, s.pi, p, 3)
        c = lf2.lf2_field_compare(s.phi, zeros32.data_ptr(), lf2.LF2_F32, which=2)
        # against zeros: the norms of the compensation itself
        assert c["max_abs_ref"] == 0.0 and c["sum_sq_ref"] == 0.0
        assert np.isfinite(c["max_abs_diff"]) and c["max_abs_diff"] > 0.0
        assert c["max_abs_diff"] ** 2 <= c["sum_sq_diff"] <= 512 * c["max_abs_diff"] ** 2
        assert c["max_abs_diff"] < 1e-6  # a compensation is below one float ulp of |phi| < 2
        for which in (-1, 4):
            with pytest.raises(lf2.LF2Error) as e:
                lf2.lf2_field_compare(s.phi, zeros32.data_ptr(), lf2.LF2_F32, which=which)
            assert e.value.status == lf2.LF2_ERR_INVALID
        with pytest.raises(lf2.LF2Error) as e:
            lf2.lf2_field_compare(s.phi, None, lf2.LF2_F32)
        assert e.value.status == lf2.LF2_ERR_INVALID
        with pytest.raises(lf2.LF2Error) as e:
            lf2.lf2_field_compare(s.phi, zeros32.data_ptr(), 7)
        assert e.value.status == lf2.LF2_ERR_INVALID
