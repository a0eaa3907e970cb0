"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances:
  * FP64: relative 1e-12 of max|.| after 10 steps for phi and pi, and of |E| for the energy.
    The two sides round differently (the kernels fold dt into the force and use FMA), each
    step adds O(10) ulps of relative error, so 10 steps stay near 1e-15.
  * Integer-valued fields with dx = dt = 1 and no potential: every operation is exact in FP64
    and FP32 (values stay below 2^24), so all precisions must match bitwise.
  * FP32 (Kahan or plain) vs the FP64 oracle: relative max error <= 1e-5 after 10 steps
    (float32 rounding of the initial data is ~6e-8 relative, and the per-step force error
    ~1e-7; 10 steps of the phi^4 dynamics amplify that by well under 100).
"""
import numpy as np
import pytest

from paper_1508_05610_gb300 import inputs

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12


@pytest.fixture(scope="module")
def lf2():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1508_05610_gb300 import build, lf2 as binding
    build.build()
    binding.load()
    return binding


def relmax(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def run_gpu(lf2, phi0, pi0, steps, prec, kw, half_kick=True, kernel=None, tile_y=0, zchunk=0, **tb):
    nz, ny, nx, c = phi0.shape
    p = lf2.params(**kw)
    with lf2.System((nx, ny, nz), c, prec) as s:
        s.upload(phi0, pi0)
        if half_kick:
            lf2.lf2_leapfrog_init(s.phi, s.pi, p)
        if kernel is None:
            lf2.lf2_leapfrog(s.phi, s.pi, p, steps)
        else:
            lf2.lf2_leapfrog_ex(s.phi, s.pi, p, steps, kernel=kernel, tile_y=tile_y, zchunk=zchunk, **tb)
        e = lf2.lf2_energy(s.phi, s.pi, p, ncomp=c)
        phi, pi = s.download()
    return phi, pi, e


# ---------------------------------------------------------------- 32^3 real, FP64
def test_cfg_32cube_fp64_every_step(lf2, ora):
    """32^3 real phi^4, FP64, dx=1, dt=0.1, lambda=eta=1, phi0 ~ N(0, 0.1^2), pi0 = 0, 100 steps:
    energy and checksums every step, fields after 10 and 100 steps."""
    kw = dict(dx=1.0, dt=0.1, lam=1.0, eta=1.0, m2=0.0)
    phi0 = inputs.gaussian_field(32, 32, 32, 1, sigma=0.1, seed=inputs.BASE_SEED)
    pi0 = np.zeros_like(phi0)
    p = lf2.params(**kw)
    ophi, opi = ora.evolve(phi0, pi0, 0, half_kick=True, **kw)
    with lf2.System((32, 32, 32), 1, "f64") as s:
        s.upload(phi0, pi0)
        lf2.lf2_leapfrog_init(s.phi, s.pi, p)
        for n in range(101):
            if n > 0:
                lf2.lf2_leapfrog(s.phi, s.pi, p, 1)
                ophi, opi = ora.evolve(ophi, opi, 1, **kw)
            e = lf2.lf2_energy(s.phi, s.pi, p, ncomp=1)
            oe = ora.energy(ophi, opi, **kw)
            assert abs(e["total"] - oe["total"]) <= F64_TOL * abs(oe["total"]), n
            for key in ("kinetic", "gradient", "potential"):
                assert abs(e[key] - oe[key]) <= F64_TOL * abs(oe["total"]), (n, key)
            scale = float(np.sum(np.abs(ophi)))
            assert abs(e["sum"][0] - oe["sum"][0]) <= F64_TOL * scale, n
            assert abs(e["sum_sq"][0] - oe["sum_sq"][0]) <= F64_TOL * oe["sum_sq"][0], n
            if n in (10, 100):
                phi, pi = s.download()
                assert relmax(phi, ophi) <= F64_TOL * (1 if n == 10 else 100), n
                assert relmax(pi, opi) <= F64_TOL * (1 if n == 10 else 100), n


# ----------------------------------------------------- shapes x kernels, FP64 parity
SHAPES = [
    ((3, 4, 5), 1), ((3, 4, 5), 2), ((6, 10, 14), 1), ((6, 10, 14), 2),
    ((40, 16, 9), 1),    # streaming: ragged warp (20 of 32 lanes)
    ((34, 8, 6), 2),     # streaming complex FP64: two x tiles, second has 2 lanes
    ((160, 8, 7), 1),    # streaming FP64 real: 64-site tiles, 3 tiles, last ragged
    ((64, 24, 33), 2),   # z chunks with a ragged last chunk
]


@pytest.mark.parametrize("shape,ncomp", SHAPES)
def test_fp64_parity_10_steps(lf2, ora, shape, ncomp):
    nx, ny, nz = shape
    kw = dict(dx=0.9, dt=0.07, lam=1.3, eta=0.8, m2=0.05)
    phi0 = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.3, seed=101)
    pi0 = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.1, seed=102)
    ophi, opi = ora.evolve(phi0, pi0, 10, half_kick=True, **kw)
    oe = ora.energy(ophi, opi, **kw)
    phi, pi, e = run_gpu(lf2, phi0, pi0, 10, "f64", kw)
    assert relmax(phi, ophi) <= F64_TOL
    assert relmax(pi, opi) <= F64_TOL
    assert abs(e["total"] - oe["total"]) <= F64_TOL * abs(oe["total"])


# ---------------------------------------------------- integer data: bitwise, every path
@pytest.mark.parametrize("prec", ["f64", "f32k", "f32"])
@pytest.mark.parametrize("shape,ncomp", [((5, 4, 3), 1), ((8, 8, 6), 2), ((40, 16, 9), 1), ((96, 8, 5), 1),
                                         ((34, 8, 6), 2)])
def test_integer_fields_bitwise_all_precisions(lf2, ora, prec, shape, ncomp):
    nx, ny, nz = shape
    kw = dict(dx=1.0, dt=1.0, lam=0.0, eta=0.0, m2=0.0)
    phi0 = inputs.integer_field(nx, ny, nz, ncomp, lo=-4, hi=4, seed=5)
    pi0 = inputs.integer_field(nx, ny, nz, ncomp, lo=-4, hi=4, seed=6)
    steps = 4
    ophi, opi = ora.evolve(phi0, pi0, steps, half_kick=False, **kw)
    assert np.max(np.abs(ophi)) < 2 ** 24 and np.max(np.abs(opi)) < 2 ** 24
    for kernel in (lf2.LF2_KERNEL_SITE, lf2.LF2_KERNEL_AUTO):
        phi, pi, _ = run_gpu(lf2, phi0, pi0, steps, prec, kw, half_kick=False, kernel=kernel)
        assert np.array_equal(phi, ophi) and np.array_equal(pi, opi), (prec, kernel)


# ------------------------------------------- every kernel variant gives the same bits
@pytest.mark.parametrize("prec", ["f64", "f32k", "f32"])
@pytest.mark.parametrize("shape,ncomp", [((64, 16, 12), 1), ((32, 16, 10), 2), ((96, 8, 9), 1), ((24, 16, 10), 3),
                                         ((16, 8, 6), 6), ((12, 8, 5), 4), ((136, 8, 5), 3)])
def test_kernel_variants_bitwise_identical(lf2, prec, shape, ncomp):
    nx, ny, nz = shape
    kw = dict(dx=1.0, dt=0.05, lam=1.0, eta=1.0, m2=0.0)
    phi0 = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.5, seed=7)
    pi0 = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.1, seed=8)
    ref = run_gpu(lf2, phi0, pi0, 6, prec, kw, kernel=lf2.LF2_KERNEL_SITE)
    for tile_y in (2, 4, 8, 16 if ny % 16 == 0 else 8):
        for zchunk in (0, 1, 3, nz):
            got = run_gpu(lf2, phi0, pi0, 6, prec, kw, kernel=lf2.LF2_KERNEL_STREAM, tile_y=tile_y, zchunk=zchunk)
            assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), (tile_y, zchunk)
            assert got[2]["total"] == ref[2]["total"]


# ------------------------------------------------------- FP32 against the FP64 oracle
@pytest.mark.parametrize("prec", ["f32k", "f32"])
@pytest.mark.parametrize("ncomp", [1, 2])
def test_fp32_within_stated_error_of_fp64_oracle(lf2, ora, prec, ncomp):
    nx, ny, nz = 32, 24, 20
    kw = dict(dx=1.0, dt=0.05, lam=1.0, eta=1.0, m2=0.0)
    phi0 = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.1, seed=inputs.BASE_SEED)
    pi0 = np.zeros_like(phi0)
    ophi, opi = ora.evolve(phi0, pi0, 10, half_kick=True, **kw)
    oe = ora.energy(ophi, opi, **kw)
    phi, pi, e = run_gpu(lf2, phi0, pi0, 10, prec, kw)
    assert relmax(phi, ophi) <= 1e-5
    assert relmax(pi, opi) <= 1e-5
    assert abs(e["total"] - oe["total"]) <= 1e-5 * abs(oe["total"])


def test_fp32_kahan_beats_plain_over_many_small_steps(lf2, ora):
    """The compensated drift keeps phi's rounding error from growing with the step count.
    A homogeneous field with no potential has F = 0 exactly, so pi stays constant and
    phi_n = 1 + n dt pi.  pi = float32(0.3) and dt = 2^-9 are exact in float32 (the oracle gets the
    same values), but dt * pi has bits far below the ulp of phi, so every FP32 drift rounds:
    plain FP32 accumulates that rounding over 4000 steps, the compensated drift does not."""
    nx, ny, nz = 8, 8, 8
    kw = dict(dx=1.0, dt=2.0 ** -9, lam=0.0, eta=0.0, m2=0.0)
    phi0 = np.full((nz, ny, nx, 1), 1.0)
    pi0 = np.full_like(phi0, float(np.float32(0.3)))
    steps = 4000
    ophi, _ = ora.evolve(phi0, pi0, steps, half_kick=True, **kw)
    ek = relmax(run_gpu(lf2, phi0, pi0, steps, "f32k", kw)[0], ophi)
    ep = relmax(run_gpu(lf2, phi0, pi0, steps, "f32", kw)[0], ophi)
    assert ek <= 2.4e-7 and ek < ep / 10, (ek, ep)


# ------------------------------------------------ temporal blocking: same bits as one step
TB_SHAPES = [((64, 16, 12), 1), ((32, 16, 10), 2), ((96, 8, 9), 1), ((40, 24, 7), 2), ((20, 6, 5), 1)]


TB_PARAMS = [dict(dx=1.0, dt=0.05, lam=1.0, eta=1.0, m2=0.01), dict(dx=0.7, dt=0.03, lam=0.6, eta=1.3, m2=0.0)]


@pytest.mark.parametrize("prec", ["f64", "f32k", "f32"])
@pytest.mark.parametrize("shape,ncomp", TB_SHAPES)
@pytest.mark.parametrize("pset", [0, 1])
def test_tblock_bitwise_identical_to_single_steps(lf2, prec, shape, ncomp, pset):
    """Every depth, column width, tile and z-chunk (ragged tiles and chunks, lattices smaller
    than the halo, step counts that leave a remainder) reproduces the one-step kernel bit for bit."""
    nx, ny, nz = shape
    kw = TB_PARAMS[pset]
    phi0 = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.5, seed=17)
    pi0 = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.1, seed=18)
    steps = 11
    ref = run_gpu(lf2, phi0, pi0, steps, prec, kw, kernel=lf2.LF2_KERNEL_SITE)
    ran = 0
    for depth in (2, 3, 4, 6, 8):
        for cx in (1, 2):
            for tile_x, tile_y in ((8, 4), (16, 8), (32, 16), (12, 6), (24, 8), (56, 8)):
                for zchunk in (0, 5):
                    try:
                        got = run_gpu(lf2, phi0, pi0, steps, prec, kw, kernel=lf2.LF2_KERNEL_TBLOCK, depth=depth, cx=cx,
                                      tile_x=tile_x, tile_y=tile_y, zchunk=zchunk)
                    except lf2.LF2Error as e:
                        assert e.status == lf2.LF2_ERR_UNSUPPORTED, e
                        continue
                    ran += 1
                    cfg = (depth, cx, tile_x, tile_y, zchunk)
                    assert np.array_equal(got[0], ref[0]), cfg
                    assert np.array_equal(got[1], ref[1]), cfg
                    assert got[2]["total"] == ref[2]["total"], cfg
    assert ran >= 20


CLUSTER_SHAPES = [((64, 40, 12), 1), ((60, 36, 10), 2), ((128, 20, 9), 1), ((36, 70, 7), 2)]


@pytest.mark.parametrize("prec", ["f32k", "f32"])
@pytest.mark.parametrize("shape,ncomp", CLUSTER_SHAPES)
def test_tblock_cluster_bitwise_identical_to_single_steps(lf2, prec, shape, ncomp):
    """Temporal blocking with thread-block clusters (2, 4 or 8 CTAs per tile, each holding a band
    of the tile's region rows and passing its edge rows to the neighbouring bands through
    distributed shared memory): every depth, column width and cluster size, with ragged tiles,
    bands of one to many warps and z-chunks, reproduces the one-step kernel bit for bit."""
    nx, ny, nz = shape
    kw = TB_PARAMS[0]
    phi0 = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.5, seed=27)
    pi0 = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.1, seed=28)
    steps = 11
    ref = run_gpu(lf2, phi0, pi0, steps, prec, kw, kernel=lf2.LF2_KERNEL_SITE)
    ran = 0
    for depth in (3, 4):
        for cx in (1, 2, 4):
            tp = -(-depth // cx) * cx
            for cl in (2, 4, 8):
                for band in (2, 16):
                    tile_y = cl * band - 2 * depth
                    for tile_x in (32 * cx - 2 * tp, 16 * cx - 2 * tp):
                        if tile_y < 1 or tile_x < cx:
                            continue
                        for zchunk in (0, 4):
                            try:
                                got = run_gpu(lf2, phi0, pi0, steps, prec, kw, kernel=lf2.LF2_KERNEL_TBLOCK,
                                              depth=depth, cx=cx, tile_x=tile_x, tile_y=tile_y, zchunk=zchunk,
                                              cluster=cl)
                            except lf2.LF2Error as e:
                                assert e.status == lf2.LF2_ERR_UNSUPPORTED, e
                                continue
                            ran += 1
                            cfg = (depth, cx, cl, tile_x, tile_y, zchunk)
                            assert np.array_equal(got[0], ref[0]), cfg
                            assert np.array_equal(got[1], ref[1]), cfg
    assert ran >= 30


def test_tblock_cluster_parity_with_oracle(lf2, ora):
    """A clustered pass (depth 4, 4 CTAs per tile) on a ragged complex lattice: FP32 with the
    compensated drift within a relative 1e-5 of the FP64 oracle after 10 steps, and integer data
    (every operation exact) equal to the oracle bit for bit."""
    nx, ny, nz = 72, 60, 11
    kw = dict(dx=0.9, dt=0.07, lam=1.3, eta=0.8, m2=0.05)
    phi0 = inputs.gaussian_field(nx, ny, nz, 2, sigma=0.5, seed=29)
    pi0 = inputs.gaussian_field(nx, ny, nz, 2, sigma=0.1, seed=30)
    ophi, opi = ora.evolve(phi0, pi0, 10, half_kick=True, **kw)
    cfg = dict(kernel=lf2.LF2_KERNEL_TBLOCK, depth=4, cx=2, tile_x=56, tile_y=56, cluster=4)
    phi, pi, _ = run_gpu(lf2, phi0, pi0, 10, "f32k", kw, **cfg)
    assert relmax(phi, ophi) <= 1e-5 and relmax(pi, opi) <= 1e-5
    ikw = dict(dx=1.0, dt=1.0, lam=0.0, eta=0.0, m2=0.0)
    i0 = inputs.integer_field(nx, ny, nz, 2, lo=-4, hi=4, seed=31)
    j0 = inputs.integer_field(nx, ny, nz, 2, lo=-4, hi=4, seed=32)
    ophi, opi = ora.evolve(i0, j0, 4, **ikw)
    phi, pi, _ = run_gpu(lf2, i0, j0, 4, "f32", ikw, half_kick=False, **cfg)
    assert np.array_equal(phi, ophi) and np.array_equal(pi, opi)


def test_tblock_fp64_parity_with_oracle(lf2, ora):
    nx, ny, nz = 48, 20, 13
    kw = dict(dx=0.9, dt=0.07, lam=1.3, eta=0.8, m2=0.05)
    phi0 = inputs.gaussian_field(nx, ny, nz, 2, sigma=0.3, seed=201)
    pi0 = inputs.gaussian_field(nx, ny, nz, 2, sigma=0.1, seed=202)
    ophi, opi = ora.evolve(phi0, pi0, 10, half_kick=True, **kw)
    phi, pi, _ = run_gpu(lf2, phi0, pi0, 10, "f64", kw, kernel=lf2.LF2_KERNEL_TBLOCK, depth=4, cx=1, tile_x=16,
                         tile_y=8)
    assert relmax(phi, ophi) <= F64_TOL and relmax(pi, opi) <= F64_TOL


# ------------------------------------------------ O(N) fields with 3 to 6 components
@pytest.mark.parametrize("ncomp", [3, 4, 6])
def test_n_component_fields_fp64_parity(lf2, ora, ncomp):
    nx, ny, nz = 12, 10, 8
    kw = dict(dx=0.9, dt=0.07, lam=1.3, eta=0.8, m2=0.05)
    phi0 = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.3, seed=111)
    pi0 = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.1, seed=112)
    ophi, opi = ora.evolve(phi0, pi0, 10, half_kick=True, **kw)
    oe = ora.energy(ophi, opi, **kw)
    phi, pi, e = run_gpu(lf2, phi0, pi0, 10, "f64", kw)
    assert relmax(phi, ophi) <= F64_TOL and relmax(pi, opi) <= F64_TOL
    assert abs(e["total"] - oe["total"]) <= F64_TOL * abs(oe["total"])
    assert np.allclose(e["sum_sq"], oe["sum_sq"], rtol=F64_TOL, atol=0)
    scale = float(np.sum(np.abs(ophi)))
    assert np.all(np.abs(e["sum"] - oe["sum"]) <= F64_TOL * scale)


@pytest.mark.parametrize("prec", ["f32k", "f32"])
def test_n_component_fields_fp32_and_integer_bitwise(lf2, ora, prec):
    nx, ny, nz, ncomp = 12, 10, 8, 3
    kw = dict(dx=1.0, dt=0.05, lam=1.0, eta=1.0, m2=0.0)
    phi0 = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.2, seed=113)
    ophi, opi = ora.evolve(phi0, np.zeros_like(phi0), 10, half_kick=True, **kw)
    phi, pi, _ = run_gpu(lf2, phi0, np.zeros_like(phi0), 10, prec, kw)
    assert relmax(phi, ophi) <= 1e-5 and relmax(pi, opi) <= 1e-5
    ikw = dict(dx=1.0, dt=1.0, lam=0.0, eta=0.0, m2=0.0)
    i0 = inputs.integer_field(nx, ny, nz, 6, lo=-4, hi=4, seed=114)
    j0 = inputs.integer_field(nx, ny, nz, 6, lo=-4, hi=4, seed=115)
    ophi, opi = ora.evolve(i0, j0, 4, **ikw)
    phi, pi, _ = run_gpu(lf2, i0, j0, 4, prec, ikw, half_kick=False)
    assert np.array_equal(phi, ophi) and np.array_equal(pi, opi)


@pytest.mark.parametrize("prec", ["f32k", "f32"])
@pytest.mark.parametrize("shape,ncomp", [((40, 16, 9), 3), ((24, 12, 7), 4), ((33, 10, 6), 6), ((20, 6, 5), 3)])
def test_n_component_tblock_bitwise_identical_to_single_steps(lf2, prec, shape, ncomp):
    """Temporal blocking of 3, 4 and 6 components (packed component pairs, 12- and 24-byte
    sites in chunked accesses): every depth it runs, ragged tiles and z-chunks, odd x extents,
    bit for bit the one-thread-per-site kernel."""
    nx, ny, nz = shape
    kw = TB_PARAMS[0]
    phi0 = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.5, seed=19)
    pi0 = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.1, seed=20)
    steps = 9
    ref = run_gpu(lf2, phi0, pi0, steps, prec, kw, kernel=lf2.LF2_KERNEL_SITE)
    ran = 0
    for depth in (2, 3, 4, 6):
        for tile_x, tile_y in ((8, 4), (16, 8), (24, 8), (12, 6), (28, 12)):
            # built: depth 2-4 (2 for 6 components), at most 512 threads (tile plus halo)
            built = depth in ((2,) if ncomp == 6 else (2, 3, 4)) and \
                (tile_x + 2 * depth) * (tile_y + 2 * depth) <= 512
            for zchunk in (0, 4):
                cfg = (depth, tile_x, tile_y, zchunk)
                try:
                    got = run_gpu(lf2, phi0, pi0, steps, prec, kw, kernel=lf2.LF2_KERNEL_TBLOCK, depth=depth, cx=1,
                                  tile_x=tile_x, tile_y=tile_y, zchunk=zchunk)
                except lf2.LF2Error as e:
                    assert e.status == lf2.LF2_ERR_UNSUPPORTED and not built, (e, cfg)
                    continue
                assert built, cfg
                ran += 1
                assert np.array_equal(got[0], ref[0]), cfg
                assert np.array_equal(got[1], ref[1]), cfg
                assert got[2]["total"] == ref[2]["total"], cfg
    assert ran == (10 if ncomp == 6 else 26)
    # two columns per thread are not built for 3+ components
    with pytest.raises(lf2.LF2Error) as e:
        run_gpu(lf2, phi0, pi0, steps, prec, kw, kernel=lf2.LF2_KERNEL_TBLOCK, depth=2, cx=2, tile_x=16, tile_y=8)
    assert e.value.status == lf2.LF2_ERR_UNSUPPORTED


@pytest.mark.parametrize("ncomp", [3, 4, 6])
def test_n_component_tblock_parity_with_oracle_and_integer_exact(lf2, ora, ncomp):
    nx, ny, nz = 36, 14, 11
    kw = dict(dx=0.9, dt=0.07, lam=1.3, eta=0.8, m2=0.05)
    phi0 = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.3, seed=211)
    pi0 = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.1, seed=212)
    ophi, opi = ora.evolve(phi0, pi0, 10, half_kick=True, **kw)
    depth = 2 if ncomp == 6 else 4
    phi, pi, _ = run_gpu(lf2, phi0, pi0, 10, "f32k", kw, kernel=lf2.LF2_KERNEL_TBLOCK, depth=depth, cx=1,
                         tile_x=24, tile_y=8)
    assert relmax(phi, ophi) <= 1e-5 and relmax(pi, opi) <= 1e-5
    ikw = dict(dx=1.0, dt=1.0, lam=0.0, eta=0.0, m2=0.0)
    i0 = inputs.integer_field(nx, ny, nz, ncomp, lo=-4, hi=4, seed=213)
    j0 = inputs.integer_field(nx, ny, nz, ncomp, lo=-4, hi=4, seed=214)
    ophi, opi = ora.evolve(i0, j0, 4, **ikw)
    phi, pi, _ = run_gpu(lf2, i0, j0, 4, "f32", ikw, half_kick=False, kernel=lf2.LF2_KERNEL_TBLOCK, depth=2, cx=1,
                         tile_x=16, tile_y=8)
    assert np.array_equal(phi, ophi) and np.array_equal(pi, opi)


# ------------------------------------------------ symmetries of the evolution on the GPU
@pytest.mark.parametrize("prec,cfg", [("f64", {}), ("f32k", {}),
                                      ("f32k", dict(kernel=2)),  # streaming
                                      ("f32k", dict(kernel=3, depth=4, cx=2, tile_x=8, tile_y=8)),
                                      ("f64", dict(kernel=3, depth=2, cx=1, tile_x=8, tile_y=4))])
def test_symmetries_translation_and_z2_bitwise_u1_to_rounding(lf2, prec, cfg):
    """Translation by a lattice vector and phi -> -phi commute with the step exactly (every site
    runs the same round-to-nearest arithmetic, and RN is odd), so the fields must match bit for
    bit.  The U(1) quarter turn (phi_0, phi_1) -> (-phi_1, phi_0) changes the order in which
    |phi|^2 is accumulated, so it holds to rounding only."""
    shape = (24, 16, 12)
    kw = dict(dx=0.9, dt=0.07, lam=1.3, eta=0.8, m2=0.05)
    phi0 = inputs.gaussian_field(*shape, 2, sigma=0.5, seed=231)
    pi0 = inputs.gaussian_field(*shape, 2, sigma=0.2, seed=232)
    if cfg:
        cfg = dict(cfg)
        cfg["kernel"] = {2: lf2.LF2_KERNEL_STREAM, 3: lf2.LF2_KERNEL_TBLOCK}[cfg["kernel"]]

    def run(phi, pi):
        return run_gpu(lf2, phi, pi, 9, prec, kw, **cfg)
    base = run(phi0, pi0)
    shift = lambda a: np.roll(a, (5, 3, 7), axis=(0, 1, 2))  # (z, y, x)
    t = run(shift(phi0), shift(pi0))
    assert np.array_equal(t[0], shift(base[0])) and np.array_equal(t[1], shift(base[1]))
    assert abs(t[2]["total"] - base[2]["total"]) <= 1e-12 * abs(base[2]["total"])
    z = run(-phi0, -pi0)
    assert np.array_equal(z[0], -base[0]) and np.array_equal(z[1], -base[1])
    assert z[2]["total"] == base[2]["total"]
    rot = lambda a: np.stack([-a[..., 1], a[..., 0]], axis=-1)
    u = run(rot(phi0), rot(pi0))
    tol = 1e-13 if prec == "f64" else 1e-5
    assert relmax(u[0], rot(base[0])) <= tol and relmax(u[1], rot(base[1])) <= tol


KERNEL_IDS = {1: "LF2_KERNEL_SITE", 2: "LF2_KERNEL_STREAM", 3: "LF2_KERNEL_TBLOCK"}


def kernel_cfg(lf2, cfg):
    cfg = dict(cfg)
    if "kernel" in cfg:
        cfg["kernel"] = getattr(lf2, KERNEL_IDS[cfg["kernel"]])
    return cfg


HOMOGENEOUS_CFGS = [("f64", {}), ("f64", dict(kernel=1)), ("f64", dict(kernel=2)),
                    ("f64", dict(kernel=3, depth=3, cx=1, tile_x=8, tile_y=4)),
                    ("f32k", {}), ("f32k", dict(kernel=1)), ("f32k", dict(kernel=2)),
                    ("f32k", dict(kernel=3, depth=4, cx=2, tile_x=12, tile_y=6)),
                    ("f32", dict(kernel=3, depth=2, cx=1, tile_x=16, tile_y=8))]


@pytest.mark.parametrize("prec,cfg", HOMOGENEOUS_CFGS)
@pytest.mark.parametrize("ncomp", [1, 2])
def test_homogeneous_field_stays_homogeneous_and_follows_the_oscillator(lf2, ora, prec, cfg, ncomp):
    """A spatially constant field has a vanishing lattice Laplacian, and every site runs the same
    arithmetic on the same values: after any number of steps all sites hold bitwise the same phi
    and pi (an indexing slip at a tile, chunk or periodic edge would break this).  The common
    value follows the single-site anharmonic oscillator, which the oracle runs on a 1^3 lattice."""
    nx, ny, nz = 40, 12, 9
    kw = dict(dx=0.9, dt=0.07, lam=1.3, eta=0.8, m2=0.05)
    phi_site = np.array([0.7, -0.45][:ncomp])
    pi_site = np.array([0.2, 0.3][:ncomp])
    phi0 = np.broadcast_to(phi_site, (nz, ny, nx, ncomp)).copy()
    pi0 = np.broadcast_to(pi_site, (nz, ny, nx, ncomp)).copy()
    phi, pi, _ = run_gpu(lf2, phi0, pi0, 13, prec, kw, **kernel_cfg(lf2, cfg))
    assert np.array_equal(phi, np.broadcast_to(phi[0, 0, 0], phi.shape))
    assert np.array_equal(pi, np.broadcast_to(pi[0, 0, 0], pi.shape))
    ophi, opi = ora.evolve(phi0[:1, :1, :1], pi0[:1, :1, :1], 13, half_kick=True, **kw)
    tol = F64_TOL if prec == "f64" else 1e-5
    assert relmax(phi[:1, :1, :1], ophi) <= tol and relmax(pi[:1, :1, :1], opi) <= tol


@pytest.mark.parametrize("prec,cfg", [("f64", {}), ("f32k", {}), ("f32", dict(kernel=2)),
                                      ("f64", dict(kernel=3, depth=2, cx=1, tile_x=8, tile_y=4)),
                                      ("f32k", dict(kernel=3, depth=4, cx=2, tile_x=12, tile_y=6))])
def test_fixed_points_zero_and_vacuum(lf2, prec, cfg):
    """phi = pi = 0 is a fixed point of every kernel exactly.  So is the vacuum |phi| = eta = 1
    with pi = 0 and m2 = 0 in FP32 storage, whose force is the difference form (every neighbour
    difference and |phi|^2 - eta^2 are exact zeros).  The FP64 update folds -6 phi/dx^2 into the
    site's own coefficient (dt F = a nb - (dl |phi|^2 + b0) phi), whose two rounded products
    cancel only to rounding: there the vacuum holds to a few units of 1e-17 per step (an exact
    simulation of the folded update gives pi = 8.3e-17 after the half kick and 11 steps)."""
    nx, ny, nz = 40, 12, 9
    kw = dict(dx=1.0, dt=0.05, lam=1.0, eta=1.0, m2=0.0)
    zero = np.zeros((nz, ny, nx, 2))
    phi, pi, e = run_gpu(lf2, zero, zero, 11, prec, kw, **kernel_cfg(lf2, cfg))
    assert np.all(phi == 0) and np.all(pi == 0)
    assert e["total"] == 0.25 * nx * ny * nz  # lambda/4 eta^4 per site, exact
    vac = np.zeros((nz, ny, nx, 2))
    vac[..., 0] = 1.0
    phi, pi, e = run_gpu(lf2, vac, zero, 11, prec, kw, **kernel_cfg(lf2, cfg))
    if prec == "f64":
        assert np.max(np.abs(phi - vac)) <= 1e-15 and np.max(np.abs(pi)) <= 1e-15
    else:
        assert np.array_equal(phi, vac) and np.all(pi == 0)
    # the energy's synchronising half kick is FP64 arithmetic in the folded form for every
    # storage precision: its pi_n is a rounding residual of about 1e-17 per site
    assert abs(e["total"]) <= 1e-25


@pytest.mark.parametrize("prec,cfg", [("f64", {}), ("f32k", {}), ("f64", dict(kernel=2)),
                                      ("f64", dict(kernel=3, depth=2, cx=1, tile_x=8, tile_y=4)),
                                      ("f32k", dict(kernel=3, depth=4, cx=2, tile_x=8, tile_y=8))])
@pytest.mark.parametrize("perm", [(1, 0, 2), (2, 1, 0)])
def test_axis_permutation_commutes_with_the_step_to_rounding(lf2, prec, cfg, perm):
    """Relabelling two axes maps the lattice and the 7-point stencil onto themselves but changes
    the order in which the directions' terms are added: the evolved fields equal the relabelled
    ones to rounding, not bit for bit."""
    shape = (16, 24, 12)  # (nx, ny, nz); arrays are (z, y, x, comp)
    kw = dict(dx=0.9, dt=0.07, lam=1.3, eta=0.8, m2=0.05)
    phi0 = inputs.gaussian_field(*shape, 2, sigma=0.5, seed=241)
    pi0 = inputs.gaussian_field(*shape, 2, sigma=0.2, seed=242)
    relabel = lambda a: np.ascontiguousarray(np.transpose(a, perm + (3,)))
    base = run_gpu(lf2, phi0, pi0, 9, prec, kw, **kernel_cfg(lf2, cfg))
    swapped = run_gpu(lf2, relabel(phi0), relabel(pi0), 9, prec, kw, **kernel_cfg(lf2, cfg))
    tol = 1e-13 if prec == "f64" else 1e-5
    assert relmax(swapped[0], relabel(base[0])) <= tol and relmax(swapped[1], relabel(base[1])) <= tol
    assert abs(swapped[2]["total"] - base[2]["total"]) <= tol * abs(base[2]["total"])


# ------------------------------------------------ the paper's field operation: derivative
@pytest.mark.parametrize("prec,ncomp", [("f64", 1), ("f64", 3), ("f32", 2), ("f32k", 6)])
@pytest.mark.parametrize("dim", [0, 1, 2])
def test_derivative_matches_oracle(lf2, ora, prec, ncomp, dim):
    nx, ny, nz = 20, 12, 9
    phi0 = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=1.0, seed=120 + dim)
    # integer data with dx = 0.5 (1/(2 dx) = 1): exact in every precision
    i0 = inputs.integer_field(nx, ny, nz, ncomp, seed=130 + dim)
    for data, dx, exact in ((i0, 0.5, True), (phi0, 0.7, False)):
        with lf2.System((nx, ny, nz), ncomp, prec) as src:
            dst = lf2.lf2_field_alloc(src.lat, ncomp, src.prec)  # a second field on the same Lattice
            try:
                lf2.lf2_field_upload(src.phi, data)
                stored = lf2.lf2_field_download(src.phi, src.host_shape)  # the values the GPU holds
                lf2.lf2_field_derivative(src.phi, dst, dim, dx)
                got = lf2.lf2_field_download(dst, src.host_shape)
            finally:
                lf2.lf2_field_free(dst)
        want = ora.derivative(stored, dim, dx=dx)
        if exact:
            assert np.array_equal(got, want)
        else:
            tol = 1e-15 if prec == "f64" else 2e-7
            assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))


# ------------------------------------------------------------- degenerate and edge cases
@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 5), (2, 1, 3), (1, 7, 1), (4, 1, 1)])
@pytest.mark.parametrize("prec", ["f64", "f32k"])
def test_degenerate_lattices(lf2, ora, shape, prec):
    """Lattices one site thick in some dimension: a site is its own neighbour there, so that
    dimension's Laplacian term vanishes; the one-site lattice is a single anharmonic oscillator."""
    nx, ny, nz = shape
    kw = dict(dx=1.0, dt=0.1, lam=1.0, eta=1.0, m2=0.0)
    phi0 = inputs.gaussian_field(nx, ny, nz, 2, sigma=0.5, seed=151)
    ophi, opi = ora.evolve(phi0, np.zeros_like(phi0), 10, half_kick=True, **kw)
    oe = ora.energy(ophi, opi, **kw)
    phi, pi, e = run_gpu(lf2, phi0, np.zeros_like(phi0), 10, prec, kw)
    tol = F64_TOL if prec == "f64" else 1e-5
    assert relmax(phi, ophi) <= tol and relmax(pi, opi) <= tol
    assert abs(e["total"] - oe["total"]) <= tol * abs(oe["total"])


def test_zero_steps_is_identity_and_time_reversal(lf2):
    nx, ny, nz = 24, 16, 12
    kw = dict(dx=1.0, dt=0.05, lam=1.0, eta=1.0, m2=0.0)
    phi0 = inputs.gaussian_field(nx, ny, nz, 1, sigma=0.3, seed=161)
    pi_h = inputs.gaussian_field(nx, ny, nz, 1, sigma=0.1, seed=162)
    p = lf2.params(**kw)
    back = lf2.params(**dict(kw, dt=-kw["dt"]))
    with lf2.System((nx, ny, nz), 1, "f64") as s:
        s.upload(phi0, pi_h)
        lf2.lf2_leapfrog(s.phi, s.pi, p, 0)
        a = s.download()
        assert np.array_equal(a[0], phi0) and np.array_equal(a[1], pi_h)
        lf2.lf2_leapfrog(s.phi, s.pi, p, 30)
        # one more kick turns pi_{n-1/2} into pi_{n+1/2}: the start-up half-kick with dt' = -2 dt
        # is pi - (dt'/2) F = pi + dt F; then 30 steps with -dt retrace the path
        lf2.lf2_leapfrog_init(s.phi, s.pi, lf2.params(**dict(kw, dt=-2 * kw["dt"])))
        lf2.lf2_leapfrog(s.phi, s.pi, back, 30)
        rec = s.download()[0]
    assert np.max(np.abs(rec - phi0)) <= 1e-12
