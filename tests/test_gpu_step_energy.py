"""GPU: leapfrog steps with the energy of every step fused into the step kernel.

lf2_leapfrog_energy must give (1) bitwise the fields of lf2_leapfrog, (2) records bitwise equal
to lf2_energy_device called before each step (same site order and reduction), and (3) records
within 1e-12 of the FP64 oracle's energy and checksums at every step of the 32^3 workload.
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


CASES = [
    ((3, 4, 5), 1, "f64"),
    ((6, 10, 14), 2, "f64"),
    ((5, 7, 9), 6, "f64"),
    ((40, 16, 9), 1, "f32k"),
    ((34, 8, 6), 2, "f32k"),
    ((64, 24, 33), 3, "f32"),
    ((32, 32, 32), 1, "f64"),
    ((96, 96, 96), 1, "f32k"),   # more sites than threads of the largest grid: several per thread
    ((80, 64, 48), 2, "f64"),
]


@pytest.mark.parametrize("shape,ncomp,prec", CASES)
def test_fused_records_and_fields_bitwise_equal_separate_calls(lf2, shape, ncomp, prec):
    import torch
    nx, ny, nz = shape
    kw = dict(dx=0.9, dt=0.07, lam=1.3, eta=0.8, m2=0.2)
    p = lf2.params(**kw)
    phi0 = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.4, seed=inputs.BASE_SEED + 71)
    pi0 = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.2, seed=inputs.BASE_SEED + 72)
    steps = 7
    fused = torch.zeros((steps, 16), dtype=torch.float64, device="cuda")
    separate = torch.zeros((steps, 16), dtype=torch.float64, device="cuda")
    with lf2.System(shape, ncomp, prec) as a, lf2.System(shape, ncomp, prec) as b:
        a.upload(phi0, pi0)
        b.upload(phi0, pi0)
        lf2.lf2_leapfrog_init(a.phi, a.pi, p)
        lf2.lf2_leapfrog_init(b.phi, b.pi, p)
        lf2.lf2_leapfrog_energy(a.phi, a.pi, p, steps, fused.data_ptr())
        for k in range(steps):
            lf2.lf2_energy_device(b.phi, b.pi, p, separate[k].data_ptr())
            lf2.lf2_leapfrog(b.phi, b.pi, p, 1)
        torch.cuda.synchronize()
        fa, pa = a.download()
        fb, pb = b.download()
        ea = lf2.lf2_energy(a.phi, a.pi, p, ncomp=ncomp)
        eb = lf2.lf2_energy(b.phi, b.pi, p, ncomp=ncomp)
    assert np.array_equal(fa, fb) and np.array_equal(pa, pb)
    assert torch.equal(fused, separate)
    assert ea.keys() == eb.keys()
    assert all(np.array_equal(np.asarray(ea[key]), np.asarray(eb[key])) for key in ea)
    # the records are real diagnostics: energy changes little over 7 steps, sums are nonzero
    rec = fused.cpu().numpy()
    assert np.all(np.isfinite(rec))
    assert np.all(np.abs(rec[:, 3] - rec[0, 3]) <= 1e-2 * abs(rec[0, 3]))
    assert np.all(rec[:, 4 + 6: 4 + 6 + ncomp] > 0)
    assert np.all(rec[:, 4 + ncomp: 4 + 6] == 0) and np.all(rec[:, 4 + 6 + ncomp:] == 0)


@pytest.mark.parametrize("shape,ncomp,prec", [((40, 16, 9), 2, "f32k"), ((64, 24, 33), 3, "f32"),
                                               ((96, 96, 96), 1, "f32k")])
def test_energy_of_float_storage_equals_double_storage_of_the_same_values(lf2, shape, ncomp, prec):
    """The FP64 energy of FP32 storage widens each stored value exactly: fields that hold the
    same values (FP32 values over exponents -150..20, subnormals and signed zeros included)
    in FP32 and in FP64 storage give bitwise the same record, from the stand-alone reduction
    and from the fused step kernel's record of its input state."""
    import torch
    rng = np.random.default_rng(inputs.BASE_SEED + 73)

    def values():
        v = np.ldexp(rng.standard_normal(shape + (ncomp,)), rng.integers(-150, 21, shape + (ncomp,)))
        v = v.astype(np.float32)
        v.flat[::13] = 0.0
        v.flat[3::31] = -0.0
        return v.astype(np.float64)

    phi0, pi0 = values(), values()
    p = lf2.params(dx=0.9, dt=0.07, lam=1.3, eta=0.8, m2=0.2)
    fused = torch.zeros((1, 16), dtype=torch.float64, device="cuda")
    with lf2.System(shape, ncomp, prec) as a, lf2.System(shape, ncomp, "f64") as b:
        a.upload(phi0, pi0)
        b.upload(phi0, pi0)
        ea = lf2.lf2_energy(a.phi, a.pi, p, ncomp=ncomp)
        eb = lf2.lf2_energy(b.phi, b.pi, p, ncomp=ncomp)
        lf2.lf2_leapfrog_energy(a.phi, a.pi, p, 1, fused.data_ptr())
        torch.cuda.synchronize()
    assert all(np.array_equal(np.asarray(ea[key]), np.asarray(eb[key])) for key in ea)
    rec = fused[0].cpu().numpy()
    assert rec[3] == eb["total"] and rec[0] == eb["kinetic"] and rec[1] == eb["gradient"]
    assert np.array_equal(rec[4:4 + ncomp], np.asarray(eb["sum"])[:ncomp])
    assert np.isfinite(eb["total"]) and eb["total"] > 0


def test_32cube_fused_energy_every_step_vs_oracle(lf2, ora):
    """The 32^3 real FP64 workload (dt = 0.1, lambda = eta = 1, sigma = 0.1, 100 steps) with
    the energy and checksums of every step from the fused kernel, against the oracle."""
    import torch
    kw = dict(dx=1.0, dt=0.1, lam=1.0, eta=1.0, m2=0.0)
    p = lf2.params(**kw)
    phi0 = inputs.gaussian_field(32, 32, 32, 1, sigma=0.1, seed=inputs.BASE_SEED)
    pi0 = np.zeros_like(phi0)
    steps = 100
    records = torch.zeros((steps, 16), dtype=torch.float64, device="cuda")
    with lf2.System((32, 32, 32), 1, "f64") as s:
        s.upload(phi0, pi0)
        lf2.lf2_leapfrog_init(s.phi, s.pi, p)
        lf2.lf2_leapfrog_energy(s.phi, s.pi, p, steps, records.data_ptr())
        last = lf2.lf2_energy(s.phi, s.pi, p, ncomp=1)
        phi, pi = s.download()
    rec = records.cpu().numpy()
    ophi, opi = ora.evolve(phi0, pi0, 0, half_kick=True, **kw)
    for n in range(steps + 1):
        oe = ora.energy(ophi, opi, **kw)
        got = rec[n] if n < steps else np.array([last["kinetic"], last["gradient"], last["potential"], last["total"]]
                                                + [last["sum"][0]] + [0.0] * 5 + [last["sum_sq"][0]] + [0.0] * 5)
        assert abs(got[3] - oe["total"]) <= F64_TOL * abs(oe["total"]), n
        for j, key in enumerate(("kinetic", "gradient", "potential")):
            assert abs(got[j] - oe[key]) <= F64_TOL * abs(oe["total"]), (n, key)
        scale = float(np.sum(np.abs(ophi)))
        assert abs(got[4] - oe["sum"][0]) <= F64_TOL * scale, n
        assert abs(got[10] - oe["sum_sq"][0]) <= F64_TOL * oe["sum_sq"][0], n
        if n < steps:
            ophi, opi = ora.evolve(ophi, opi, 1, **kw)
    assert float(np.max(np.abs(phi - ophi)) / np.max(np.abs(ophi))) <= 100 * F64_TOL
    assert float(np.max(np.abs(pi - opi)) / np.max(np.abs(opi))) <= 100 * F64_TOL


def test_32cube_fused_energy_in_one_cuda_graph(lf2, ora):
    """100 fused steps captured into one CUDA graph: replay gives the oracle's energies; the
    per-step time of a replay is printed (one kernel launch per step)."""
    import torch
    kw = dict(dx=1.0, dt=0.1, lam=1.0, eta=1.0, m2=0.0)
    p = lf2.params(**kw)
    phi0 = inputs.gaussian_field(32, 32, 32, 1, sigma=0.1, seed=inputs.BASE_SEED)
    steps = 100
    records = torch.zeros((steps, 16), dtype=torch.float64, device="cuda")
    with lf2.System((32, 32, 32), 1, "f64") as s:
        s.upload(phi0, np.zeros_like(phi0))
        lf2.lf2_leapfrog_init(s.phi, s.pi, p)
        lf2.lf2_leapfrog_energy(s.phi, s.pi, p, 2, records.data_ptr())  # first call: allocations
        s.upload(phi0, np.zeros_like(phi0))
        lf2.lf2_leapfrog_init(s.phi, s.pi, p)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            lf2.lf2_leapfrog_energy(s.phi, s.pi, p, steps, records.data_ptr(), torch.cuda.current_stream())
        g.replay()
        torch.cuda.synchronize()
        rec = records.cpu().numpy()
        times = []
        for _ in range(3):  # the state moves on; only the timing of these replays is used
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            g.replay()
            b.record()
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b) * 1e3 / steps)
    ophi, opi = ora.evolve(phi0, np.zeros_like(phi0), 0, half_kick=True, **kw)
    for n in range(steps):
        oe = ora.energy(ophi, opi, **kw)
        assert abs(rec[n, 3] - oe["total"]) <= F64_TOL * abs(oe["total"]), n
        assert abs(rec[n, 10] - oe["sum_sq"][0]) <= F64_TOL * oe["sum_sq"][0], n
        ophi, opi = ora.evolve(ophi, opi, 1, **kw)
    print(f"32^3 fused step + energy, one graph: {min(times):.2f} us per step")
    assert min(times) < 1000


def test_fused_energy_argument_errors(lf2):
    import torch
    p = lf2.params(dx=1.0, dt=0.1, lam=1.0, eta=1.0, m2=0.0)
    with lf2.System((8, 8, 8), 1, "f64") as s:
        s.upload(np.zeros((8, 8, 8, 1)), np.zeros((8, 8, 8, 1)))
        with pytest.raises(lf2.LF2Error) as e:
            lf2.lf2_leapfrog_energy(s.phi, s.pi, p, -1, 0)
        assert e.value.status == lf2.LF2_ERR_INVALID
        with pytest.raises(lf2.LF2Error) as e:
            lf2.lf2_leapfrog_energy(s.phi, s.pi, p, 3, None)
        assert e.value.status == lf2.LF2_ERR_INVALID
        lf2.lf2_leapfrog_energy(s.phi, s.pi, p, 0, None)  # nothing to do, nothing written
        rec = torch.zeros((1, 16), dtype=torch.float64, device="cuda")
        lf2.lf2_leapfrog_energy(s.phi, s.pi, p, 1, rec.data_ptr())
        torch.cuda.synchronize()
        # phi = pi = 0: only the potential lambda/4 eta^4 per site is left (exact in FP64)
        r = rec[0].cpu().numpy()
        assert r[0] == 0.0 and r[1] == 0.0 and r[2] == 0.25 * 512 and r[3] == 0.25 * 512
        assert np.all(r[4:] == 0.0)


def test_barrier_timeout_is_reported_and_the_context_stays_usable(lf2, ora, monkeypatch):
    """Failure detection without a GPU fault: LF2_FAULT=timeout makes every grid-barrier wait of
    the multi-step kernel give up at once.  The run ends by itself, its last records are NaN,
    lf2_field_check reports LF2_ERR_TIMEOUT once, and a normal run right after on the same
    field gives the oracle's energies."""
    import torch
    kw = dict(dx=1.0, dt=0.1, lam=1.0, eta=1.0, m2=0.0)
    p = lf2.params(**kw)
    phi0 = inputs.gaussian_field(16, 16, 16, 1, sigma=0.1, seed=inputs.BASE_SEED + 5)
    steps = 6
    rec = torch.zeros((steps, 16), dtype=torch.float64, device="cuda")
    with lf2.System((16, 16, 16), 1, "f64") as s:
        s.upload(phi0, np.zeros_like(phi0))
        lf2.lf2_leapfrog_init(s.phi, s.pi, p)
        monkeypatch.setenv("LF2_FAULT", "timeout")
        lf2.lf2_leapfrog_energy(s.phi, s.pi, p, steps, rec.data_ptr())
        monkeypatch.delenv("LF2_FAULT")
        with pytest.raises(lf2.LF2Error) as e:
            lf2.lf2_field_check(s.phi)
        assert e.value.status == lf2.LF2_ERR_TIMEOUT
        lf2.lf2_field_check(s.phi)  # reported once
        assert torch.isnan(rec[-1]).all()
        # the same field and context, a clean run
        s.upload(phi0, np.zeros_like(phi0))
        lf2.lf2_leapfrog_init(s.phi, s.pi, p)
        lf2.lf2_leapfrog_energy(s.phi, s.pi, p, steps, rec.data_ptr())
        lf2.lf2_field_check(s.phi)
        got = rec.cpu().numpy()
    ophi, opi = ora.evolve(phi0, np.zeros_like(phi0), 0, half_kick=True, **kw)
    for n in range(steps):
        oe = ora.energy(ophi, opi, **kw)
        assert abs(got[n, 3] - oe["total"]) <= F64_TOL * abs(oe["total"]), n
        ophi, opi = ora.evolve(ophi, opi, 1, **kw)
