"""GPU tests of the autotuner and of batched ensembles.

Both rest on one invariant: every kernel configuration computes bitwise the same result, so
a tuned plan or a batched run must reproduce the one-thread-per-site kernel exactly."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1508_05610_gb300 import inputs

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lf2():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1508_05610_gb300 import build, lf2 as binding
    build.build()
    binding.load()
    return binding


def run_site(lf2, shape, ncomp, prec, phi0, pi0, kw, steps):
    p = lf2.params(**kw)
    with lf2.System(shape, ncomp, prec) as s:
        s.upload(phi0, pi0)
        lf2.lf2_leapfrog_ex(s.phi, s.pi, p, steps, kernel=lf2.LF2_KERNEL_SITE)
        return s.download()


@pytest.mark.parametrize("prec,ncomp", [("f32k", 1), ("f32", 2), ("f64", 1), ("f32k", 3), ("f32", 4), ("f32k", 6)])
def test_tune_leaves_fields_untouched_and_plan_is_bitwise(lf2, prec, ncomp):
    shape = (64, 48, 40)
    kw = dict(dx=1.0, dt=0.05, lam=1.0, eta=1.0, m2=0.0)
    phi0 = inputs.gaussian_field(*shape, ncomp, sigma=0.4, seed=61)
    pi0 = inputs.gaussian_field(*shape, ncomp, sigma=0.1, seed=62)
    p = lf2.params(**kw)
    ref = run_site(lf2, shape, ncomp, prec, phi0, pi0, kw, 13)
    with lf2.System(shape, ncomp, prec) as s:
        s.upload(phi0, pi0)
        before = s.download()
        plan = lf2.lf2_tune(s.phi, s.pi, p, flags=lf2.LF2_TUNE_FORCE)
        after = s.download()
        assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
        assert plan == lf2.lf2_tune_lookup(shape, ncomp, lf2.PRECISIONS[prec])
        lf2.lf2_leapfrog(s.phi, s.pi, p, 13)  # uses the tuned plan
        got = s.download()
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), plan


def test_tune_env_force_tunes_on_first_use_and_off_ignores_plans(lf2, monkeypatch):
    """LF2_TUNE=force: lf2_leapfrog on a shape without a plan tunes it first (a plan exists
    afterwards); LF2_TUNE=off: the default kernel runs; both step bitwise like the site kernel."""
    shape, ncomp, prec = (42, 22, 18), 1, "f32k"  # a shape no other test tunes
    kw = dict(dx=1.0, dt=0.05, lam=1.0, eta=1.0, m2=0.0)
    p = lf2.params(**kw)
    phi0 = inputs.gaussian_field(*shape, ncomp, sigma=0.4, seed=63)
    ref = run_site(lf2, shape, ncomp, prec, phi0, np.zeros_like(phi0), kw, 9)

    def plan():
        try:
            return lf2.lf2_tune_lookup(shape, ncomp, lf2.PRECISIONS[prec])
        except lf2.LF2Error as e:
            assert e.status == lf2.LF2_ERR_STATE
            return None
    assert plan() is None
    for mode in ("off", "force"):
        monkeypatch.setenv("LF2_TUNE", mode)
        with lf2.System(shape, ncomp, prec) as s:
            s.upload(phi0, np.zeros_like(phi0))
            lf2.lf2_leapfrog(s.phi, s.pi, p, 9)  # as run_site: no half-kick
            got = s.download()
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), mode
        planned = plan()
        assert (planned is None) == (mode == "off"), (mode, planned)


def test_tune_cache_file_is_read_by_a_fresh_process(lf2, tmp_path):
    cache = tmp_path / "plans.txt"
    code = r"""
import sys, json
sys.path.insert(0, %r)
from paper_1508_05610_gb300 import lf2
lf2.load()
shape = (32, 32, 16)
if sys.argv[1] == "tune":
    s = lf2.System(shape, 1, "f32k")
    print(json.dumps(lf2.lf2_tune(s.phi, s.pi, lf2.params(dt=0.05))))
    s.close()
else:
    print(json.dumps(lf2.lf2_tune_lookup(shape, 1, lf2.LF2_F32_KAHAN)))
""" % ROOT
    env = dict(os.environ, LF2_TUNE_CACHE=str(cache))
    a = subprocess.run([sys.executable, "-c", code, "tune"], env=env, capture_output=True, text=True, check=True)
    b = subprocess.run([sys.executable, "-c", code, "lookup"], env=env, capture_output=True, text=True, check=True)
    assert a.stdout.strip() == b.stdout.strip() and cache.exists()


ENSEMBLE = [((24, 16, 12), 0.7), ((32, 32, 32), 1.3), ((40, 24, 20), 0.55), ((16, 16, 16), 1.9), ((64, 8, 28), 1.0)]


@pytest.mark.parametrize("prec,ncomp", [("f32k", 1), ("f32k", 2), ("f64", 1)])
def test_ensemble_members_equal_standalone_runs(lf2, prec, ncomp):
    systems, refs, plist = [], [], []
    try:
        for i, (shape, lam) in enumerate(ENSEMBLE):
            kw = dict(dx=1.0, dt=0.05, lam=lam, eta=1.0, m2=0.0)
            phi0 = inputs.gaussian_field(*shape, ncomp, sigma=0.3, seed=100 + i)
            pi0 = inputs.gaussian_field(*shape, ncomp, sigma=0.1, seed=200 + i)
            refs.append((run_site(lf2, shape, ncomp, prec, phi0, pi0, kw, 11),
                         run_site(lf2, shape, ncomp, prec, phi0, pi0, kw, 22)))
            s = lf2.System(shape, ncomp, prec)
            s.upload(phi0, pi0)
            systems.append(s)
            plist.append(lf2.params(**kw))
        e = lf2.lf2_ensemble_create([s.phi for s in systems], [s.pi for s in systems], plist)
        try:
            lf2.lf2_ensemble_run(e, 11)  # 2 passes of depth 4 + 3 single steps
            for s, (r11, _) in zip(systems, refs):
                got = s.download()
                assert np.array_equal(got[0], r11[0]) and np.array_equal(got[1], r11[1])
            lf2.lf2_ensemble_run(e, 11)  # other buffer parity: a second captured graph
            for s, (_, r22) in zip(systems, refs):
                got = s.download()
                assert np.array_equal(got[0], r22[0]) and np.array_equal(got[1], r22[1])
        finally:
            lf2.lf2_ensemble_destroy(e)
    finally:
        for s in systems:
            s.close()


@pytest.mark.parametrize("prec,ncomp,depth", [("f32k", 3, 3), ("f32", 4, 4), ("f32k", 4, 2), ("f32k", 6, 2)])
def test_ensemble_of_many_component_fields_runs_temporal_blocking(lf2, ora, prec, ncomp, depth):
    """Ensembles of 3-, 4- and 6-component O(N) fields on temporal-blocking passes (one column
    per thread): every member bitwise equal to the same lattice on the one-thread-per-site
    kernel, and within a relative 1e-5 of the FP64 oracle, for 11 steps (whole passes plus
    single steps) and again for 11 more (the other buffer parity)."""
    systems, plist, starts = [], [], []
    try:
        for i, (shape, lam) in enumerate(ENSEMBLE):
            kw = dict(dx=1.0, dt=0.05, lam=lam, eta=1.0, m2=0.0)
            phi0 = inputs.gaussian_field(*shape, ncomp, sigma=0.3, seed=700 + i)
            s = lf2.System(shape, ncomp, prec)
            s.upload(phi0, np.zeros_like(phi0))
            systems.append(s)
            plist.append(lf2.params(**kw))
            starts.append((phi0, kw))
        e = lf2.lf2_ensemble_create([s.phi for s in systems], [s.pi for s in systems], plist)
        try:
            # raises LF2_ERR_UNSUPPORTED unless every member runs this temporal-blocking pass
            lf2.lf2_ensemble_set_config(e, depth=depth, cx=1, tile_x=16 - 2 * depth, tile_y=8)
            done = 0
            for steps in (11, 11):
                lf2.lf2_ensemble_run(e, steps)
                done += steps
                for s, (phi0, kw) in zip(systems, starts):
                    got = s.download()
                    ref = run_site(lf2, s.shape, ncomp, prec, phi0, np.zeros_like(phi0), kw, done)
                    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), (s.shape, done)
                    ophi, opi = ora.evolve(phi0, np.zeros_like(phi0), done, **kw)
                    assert np.max(np.abs(got[0] - ophi)) <= 1e-5 * np.max(np.abs(ophi)), (s.shape, done)
                    assert np.max(np.abs(got[1] - opi)) <= 1e-5 * np.max(np.abs(opi)), (s.shape, done)
        finally:
            lf2.lf2_ensemble_destroy(e)
    finally:
        for s in systems:
            s.close()


def test_ensemble_tune_and_configs_bitwise(lf2):
    prec, ncomp = "f32k", 1
    systems, refs, plist = [], [], []
    try:
        for i, (shape, lam) in enumerate(ENSEMBLE):
            kw = dict(dx=1.0, dt=0.05, lam=lam, eta=1.0, m2=0.0)
            phi0 = inputs.gaussian_field(*shape, ncomp, sigma=0.3, seed=300 + i)
            refs.append((phi0, run_site(lf2, shape, ncomp, prec, phi0, np.zeros_like(phi0), kw, 12)))
            s = lf2.System(shape, ncomp, prec)
            systems.append(s)
            plist.append(lf2.params(**kw))
        e = lf2.lf2_ensemble_create([s.phi for s in systems], [s.pi for s in systems], plist)
        try:
            chosen = lf2.lf2_ensemble_tune(e)
            for cfg in (None, dict(depth=2, cx=1, tile_x=12, tile_y=8), dict(depth=3, cx=2, tile_x=24, tile_y=16),
                        dict(kernel=lf2.LF2_KERNEL_STREAM)):
                if cfg is not None:
                    lf2.lf2_ensemble_set_config(e, **cfg)
                for s, (phi0, _) in zip(systems, refs):
                    s.upload(phi0, np.zeros_like(phi0))
                lf2.lf2_ensemble_run(e, 12)
                for s, (_, r) in zip(systems, refs):
                    got = s.download()
                    assert np.array_equal(got[0], r[0]) and np.array_equal(got[1], r[1]), (chosen, cfg)
        finally:
            lf2.lf2_ensemble_destroy(e)
    finally:
        for s in systems:
            s.close()


def test_ensemble_membership_is_enforced(lf2):
    """A member field cannot be freed or join a second ensemble until the ensemble is gone."""
    p = lf2.params(dx=1.0, dt=0.05, lam=1.0, eta=1.0, m2=0.0)
    a, b = lf2.System((16, 8, 8), 1, "f32k"), lf2.System((24, 8, 8), 1, "f32k")
    try:
        e = lf2.lf2_ensemble_create([a.phi, b.phi], [a.pi, b.pi], [p, p])
        try:
            for f in (a.phi, b.pi):
                with pytest.raises(lf2.LF2Error) as err:
                    lf2.lf2_field_free(f)
                assert err.value.status == lf2.LF2_ERR_STATE
            with pytest.raises(lf2.LF2Error) as err:
                lf2.lf2_ensemble_create([a.phi], [a.pi], [p])
            assert err.value.status == lf2.LF2_ERR_STATE
            with pytest.raises(lf2.LF2Error) as err:
                lf2.lf2_lattice_destroy(a.lat)
            assert err.value.status == lf2.LF2_ERR_STATE
            bad = lf2.params(dx=1.0, dt=float("nan"), lam=1.0, eta=1.0, m2=0.0)
            c = lf2.System((16, 8, 8), 1, "f32k")
            try:
                with pytest.raises(lf2.LF2Error) as err:
                    lf2.lf2_ensemble_create([c.phi], [c.pi], [bad])
                assert err.value.status == lf2.LF2_ERR_INVALID
            finally:
                c.close()
            lf2.lf2_ensemble_run(e, 3)  # the ensemble still works
        finally:
            lf2.lf2_ensemble_destroy(e)
        e2 = lf2.lf2_ensemble_create([a.phi], [a.pi], [p])  # free again after destroy
        lf2.lf2_ensemble_destroy(e2)
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("prec,ncomp", [("f64", 2), ("f32k", 1), ("f32", 2)])
def test_snapshot_format_and_exact_restart(lf2, tmp_path, prec, ncomp):
    """Snapshots are the paper's header-less row-major per-site component lists in the storage
    type; writing phi, pi (and the compensation) and reading them into fresh fields continues
    the run bit for bit."""
    shape = (24, 20, 16)
    nx, ny, nz = shape
    kw = dict(dx=1.0, dt=0.05, lam=1.0, eta=1.0, m2=0.0)
    phi0 = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.4, seed=71)
    p = lf2.params(**kw)
    dtype = np.float64 if prec == "f64" else np.float32
    straight = run_site(lf2, shape, ncomp, prec, phi0, np.zeros_like(phi0), kw, 20)
    with lf2.System(shape, ncomp, prec) as s:
        s.upload(phi0, np.zeros_like(phi0))
        lf2.lf2_leapfrog_ex(s.phi, s.pi, p, 10, kernel=lf2.LF2_KERNEL_SITE)
        lf2.lf2_field_write(s.phi, tmp_path / "phi.bin")
        lf2.lf2_field_write(s.pi, tmp_path / "pi.bin")
        if prec == "f32k":
            lf2.lf2_field_write(s.phi, tmp_path / "comp.bin", which=2)
        # the file is the row-major per-site component list in the storage type
        raw = np.fromfile(tmp_path / "phi.bin", dtype=dtype).reshape(nz, ny, nx, ncomp)
        assert np.array_equal(raw.astype(np.float64), s.download()[0])
    with lf2.System(shape, ncomp, prec) as s:
        lf2.lf2_field_read(s.phi, tmp_path / "phi.bin")
        lf2.lf2_field_read(s.pi, tmp_path / "pi.bin")
        if prec == "f32k":
            lf2.lf2_field_read(s.phi, tmp_path / "comp.bin", which=2)
        lf2.lf2_leapfrog_ex(s.phi, s.pi, p, 10, kernel=lf2.LF2_KERNEL_SITE)
        got = s.download()
    assert np.array_equal(got[0], straight[0]) and np.array_equal(got[1], straight[1])
    # a file of the wrong size is rejected
    (tmp_path / "short.bin").write_bytes(b"\0" * 8)
    with lf2.System(shape, ncomp, prec) as s:
        with pytest.raises(lf2.LF2Error) as e:
            lf2.lf2_field_read(s.phi, tmp_path / "short.bin")
        assert e.value.status == lf2.LF2_ERR_INVALID


def test_32cube_run_with_energy_every_step_in_one_cuda_graph(lf2, ora):
    """The 32^3 real FP64 workload (dt = 0.1, lambda = eta = 1, sigma = 0.1) with energy and
    checksum after every one of 100 steps, captured into one CUDA graph (lf2_leapfrog +
    lf2_energy_device per step) and replayed: every record within 1e-12 of the oracle."""
    import torch
    kw = dict(dx=1.0, dt=0.1, lam=1.0, eta=1.0, m2=0.0)
    p = lf2.params(**kw)
    phi0 = inputs.gaussian_field(32, 32, 32, 1, sigma=0.1, seed=inputs.BASE_SEED)
    steps = 100
    records = torch.zeros((steps, 16), dtype=torch.float64, device="cuda")
    with lf2.System((32, 32, 32), 1, "f64") as s:
        s.upload(phi0, np.zeros_like(phi0))
        lf2.lf2_leapfrog_init(s.phi, s.pi, p)
        lf2.lf2_leapfrog(s.phi, s.pi, p, 2)  # warm-up outside the capture, even count
        lf2.lf2_field_upload(s.phi, phi0)
        lf2.lf2_field_upload(s.pi, np.zeros_like(phi0))
        lf2.lf2_leapfrog_init(s.phi, s.pi, p)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            st = torch.cuda.current_stream()
            for n in range(steps):
                lf2.lf2_leapfrog(s.phi, s.pi, p, 1, st)
                lf2.lf2_energy_device(s.phi, s.pi, p, records[n].data_ptr(), st)
        g.replay()
        torch.cuda.synchronize()
        rec = records.cpu().numpy()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        g.replay()  # time one more replay (the state moves on; only the timing is used)
        b.record()
        torch.cuda.synchronize()
        us_per_step = a.elapsed_time(b) * 1e3 / steps
    ophi, opi = ora.evolve(phi0, np.zeros_like(phi0), 0, half_kick=True, **kw)
    for n in range(steps):
        ophi, opi = ora.evolve(ophi, opi, 1, **kw)
        oe = ora.energy(ophi, opi, **kw)
        assert abs(rec[n, 3] - oe["total"]) <= 1e-12 * abs(oe["total"]), n
        assert abs(rec[n, 10] - oe["sum_sq"][0]) <= 1e-12 * oe["sum_sq"][0], n
    print(f"32^3 step + energy, one graph: {us_per_step:.1f} us per step")
    assert us_per_step < 1000
