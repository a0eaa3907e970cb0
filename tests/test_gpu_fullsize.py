"""Parity at full workload sizes, element by element, in the launch configurations that the
benchmark and the tuner run.

The oracle evolves the whole lattice on the host cores (OpenMP over z-planes, the same
per-site arithmetic as one thread): 10 steps of the 256^3 complex lattice take about half a
second on 16 Grace cores, and 10 steps of the 1024^3 real lattice about a minute and a half.
Every site of phi and pi is compared, so a slip at a ragged tile edge (256 = 10 x 24 + 16,
1024 = 18 x 56 + 16) or at a z-chunk boundary fails.  The 1536^3 complex lattice (a 174 GB
device state) is still checked at sampled sites: one site after n steps depends only on the
initial data within n sites of it, so the oracle evolves the periodic (2h+1)^3 box cut around
the site (h >= n + 1) and its centre must match.

Inputs are generated on the device by the seeded generator and copied to the host from that
same array, so both sides start from identical values (FP32 runs: the FP32-rounded values).
"""
import os

import numpy as np
import pytest

from paper_1508_05610_gb300 import inputs

pytestmark = pytest.mark.gpu

STEPS = 10
HALF = STEPS + 2
THREADS = os.cpu_count() or 1
KW = dict(dx=1.0, dt=0.05, lam=1.0, eta=1.0, m2=0.0)


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1508_05610_gb300 import build, lf2
    build.build()
    lf2.load()
    return torch, lf2


def evolve_wrapped(torch, lf2, phi_t, prec, p, steps, cfg=None, tune=False):
    """Evolves a device tensor in place through the C ABI with every buffer borrowed, either
    with an explicit kernel configuration (lf2_leapfrog_ex), or with the tuner's plan
    (lf2_tune, then lf2_leapfrog), or with lf2_leapfrog's default.  Returns the (phi, pi)
    tensors that hold the result and the plan that ran."""
    nz, ny, nx, c = phi_t.shape
    bufs = [phi_t, torch.empty_like(phi_t)]
    if prec == lf2.LF2_F32_KAHAN:
        bufs += [torch.zeros_like(phi_t), torch.zeros_like(phi_t)]
    pis = [torch.zeros_like(phi_t), torch.empty_like(phi_t)]
    lat = lf2.lf2_lattice_create((nx, ny, nz))
    fphi = lf2.lf2_field_wrap(lat, c, prec, [t.data_ptr() for t in bufs])
    fpi = lf2.lf2_field_wrap(lat, c, prec, [t.data_ptr() for t in pis])
    plan = cfg
    try:
        stream = torch.cuda.current_stream()
        lf2.lf2_leapfrog_init(fphi, fpi, p, stream)
        if tune:
            plan = lf2.lf2_tune(fphi, fpi, p, stream=stream)
        if cfg is not None:
            lf2.lf2_leapfrog_ex(fphi, fpi, p, steps, stream=stream, **cfg)
        else:
            lf2.lf2_leapfrog(fphi, fpi, p, steps, stream)
        torch.cuda.synchronize()
        fp, fq = lf2.lf2_field_buffer(fphi, 0), lf2.lf2_field_buffer(fpi, 0)
    finally:
        lf2.lf2_field_free(fphi)
        lf2.lf2_field_free(fpi)
        lf2.lf2_lattice_destroy(lat)
    phi = next(t for t in bufs if t.data_ptr() == fp)
    pi = next(t for t in pis if t.data_ptr() == fq)
    return phi, pi, plan


def relmax_device(torch, got, want_host):
    """max |got - want| / max |want| over every element, in FP64 on the device."""
    want = torch.from_numpy(want_host).to(got.device)
    err = float((got.double() - want).abs().max())
    scale = float(want.abs().max())
    del want
    return err / scale


def oracle_full(ora, phi0_host, steps=STEPS):
    return ora.evolve(phi0_host, np.zeros_like(phi0_host), steps, half_kick=True, threads=THREADS, **KW)


def test_256cube_complex_fp64_stream_every_site(env, ora):
    """The FP64 comparison path of the benchmark: 256^3 complex phi^4 on the one-step streaming
    kernel, 10 steps.  Every element of phi and pi within a relative 1e-12 of the oracle, and
    the energy of the final state too."""
    torch, lf2 = env
    phi0 = inputs.gaussian_field_device(256, 256, 256, 2, sigma=0.1, seed=inputs.BASE_SEED)
    host0 = phi0.cpu().numpy()
    p = lf2.params(**KW)
    phi, pi, _ = evolve_wrapped(torch, lf2, phi0.clone(), lf2.LF2_F64, p, STEPS,
                                cfg=dict(kernel=lf2.LF2_KERNEL_STREAM))
    ophi, opi = oracle_full(ora, host0)
    assert relmax_device(torch, phi, ophi) <= 1e-12
    assert relmax_device(torch, pi, opi) <= 1e-12
    want = ora.energy(ophi, opi, **KW)
    with lf2.System((256, 256, 256), 2, "f64") as s:
        s.upload(phi.cpu().numpy(), pi.cpu().numpy())
        got = lf2.lf2_energy(s.phi, s.pi, p)
    assert abs(got["total"] - want["total"]) <= 1e-12 * abs(want["total"])


def test_256cube_complex_fp64_default_path_every_site(env, ora):
    """lf2_leapfrog's own choice of kernel for the same lattice (no tuned plan) against the
    oracle at every element."""
    torch, lf2 = env
    phi0 = inputs.gaussian_field_device(256, 256, 256, 2, sigma=0.1, seed=inputs.BASE_SEED + 1)
    host0 = phi0.cpu().numpy()
    phi, pi, _ = evolve_wrapped(torch, lf2, phi0.clone(), lf2.LF2_F64, lf2.params(**KW), STEPS)
    ophi, opi = oracle_full(ora, host0)
    assert relmax_device(torch, phi, ophi) <= 1e-12
    assert relmax_device(torch, pi, opi) <= 1e-12


def test_256cube_complex_fp32_kahan_tuned_every_site(env, ora):
    """256^3 complex, FP32 with the compensated drift and the tuner's plan (temporal blocking
    with ragged 24-site tiles), 10 steps: every element of phi and pi within a relative 1e-5 of
    the oracle started from the same FP32 values, and the energy within 1e-5."""
    torch, lf2 = env
    phi0 = inputs.gaussian_field_device(256, 256, 256, 2, sigma=0.1, seed=inputs.BASE_SEED, dtype=torch.float32)
    host0 = phi0.double().cpu().numpy()
    p = lf2.params(**KW)
    phi, pi, plan = evolve_wrapped(torch, lf2, phi0.clone(), lf2.LF2_F32_KAHAN, p, STEPS, tune=True)
    ophi, opi = oracle_full(ora, host0)
    assert relmax_device(torch, phi, ophi) <= 1e-5, plan
    assert relmax_device(torch, pi, opi) <= 1e-5, plan
    want = ora.energy(ophi, opi, **KW)
    with lf2.System((256, 256, 256), 2, "f32k") as s:
        s.upload(phi.double().cpu().numpy(), pi.double().cpu().numpy())
        got = lf2.lf2_energy(s.phi, s.pi, p)
    assert abs(got["total"] - want["total"]) <= 1e-5 * abs(want["total"])


def test_256cube_complex_fp32_kahan_depth_sweep_every_site(env, ora):
    """Each temporal-blocking depth the tuner may choose for this lattice (2, 3, 4 with ragged
    24 x 24 tiles, 6 and 8 with 16 x 16 tiles, two columns per thread; 10 steps leave a
    remainder of single steps for depths 3, 4, 6 and 8) against one oracle run, element by
    element, within 1e-5."""
    torch, lf2 = env
    phi0 = inputs.gaussian_field_device(256, 256, 256, 2, sigma=0.1, seed=inputs.BASE_SEED + 2, dtype=torch.float32)
    ophi, opi = oracle_full(ora, phi0.double().cpu().numpy())
    for depth, tile in ((2, 24), (3, 24), (4, 24), (6, 16), (8, 16)):
        cfg = dict(kernel=lf2.LF2_KERNEL_TBLOCK, depth=depth, cx=2, tile_x=tile, tile_y=tile)
        phi, pi, _ = evolve_wrapped(torch, lf2, phi0.clone(), lf2.LF2_F32_KAHAN, lf2.params(**KW), STEPS, cfg=cfg)
        assert relmax_device(torch, phi, ophi) <= 1e-5, depth
        assert relmax_device(torch, pi, opi) <= 1e-5, depth
        del phi, pi


def test_1024cube_real_grf_fp32_kahan_tuned_every_site(env, ora):
    """1024^3 real phi^4 from a Gaussian random field with P(k) ~ k^-2 cut at pi/4, FP32 with
    the compensated drift and the tuner's plan, 10 steps: every element of phi and pi within a
    relative 1e-5 of the oracle (about 90 s of oracle time on 16 cores)."""
    torch, lf2 = env
    phi0 = inputs.grf_field_device(1024, sigma=0.1, seed=inputs.BASE_SEED, dtype=torch.float32)
    host0 = phi0.double().cpu().numpy()
    phi, pi, plan = evolve_wrapped(torch, lf2, phi0, lf2.LF2_F32_KAHAN, lf2.params(**KW), STEPS, tune=True)
    ophi, opi = oracle_full(ora, host0)
    del host0
    assert relmax_device(torch, phi, ophi) <= 1e-5, plan
    assert relmax_device(torch, pi, opi) <= 1e-5, plan
    del phi, pi, ophi, opi
    torch.cuda.empty_cache()


def sample_sites(n, count, seed):
    g = np.random.default_rng(seed)
    pts = [(0, 0, 0), (n - 1, n - 1, n - 1), (n - 1, 0, n // 2)]
    pts += [tuple(int(v) for v in g.integers(0, n, 3)) for _ in range(count - len(pts))]
    return pts


def box_of(torch, field, center, half):
    """(2 half + 1)^3 periodic box of a device field (nz, ny, nx, c) around center (x, y, z)."""
    nz, ny, nx = field.shape[:3]
    r = torch.arange(-half, half + 1, device=field.device)
    zi = (center[2] + r) % nz
    yi = (center[1] + r) % ny
    xi = (center[0] + r) % nx
    return field[zi][:, yi][:, :, xi].double().cpu().numpy()


def test_1536cube_complex_fp32_kahan_tuned_sampled(env, ora):
    """1536^3 complex phi^4 (the largest lattice of the workloads, the benchmark's), FP32 with
    the compensated drift and the tuned plan: sampled sites, among them tile and lattice edges,
    within 1e-5 of the FP64 oracle after 10 steps.  The oracle's boxes are cut from the initial
    field before it is evolved in place, so the device holds one state."""
    torch, lf2 = env
    torch.cuda.empty_cache()
    n = 1536
    phi = inputs.gaussian_field_device(n, n, n, 2, sigma=0.1, seed=inputs.BASE_SEED, dtype=torch.float32)
    sites = sample_sites(n, 8, seed=3) + [(23, 24, 47), (24, 23, 48), (1535, 767, 1)]
    boxes = [box_of(torch, phi, c, HALF) for c in sites]
    out_phi, out_pi, plan = evolve_wrapped(torch, lf2, phi, lf2.LF2_F32_KAHAN, lf2.params(**KW), STEPS, tune=True)
    for center, box in zip(sites, boxes):
        bphi, bpi = ora.evolve(box, np.zeros_like(box), STEPS, half_kick=True, **KW)
        x, y, z = center
        got_phi = out_phi[z, y, x].double().cpu().numpy()
        got_pi = out_pi[z, y, x].double().cpu().numpy()
        assert np.max(np.abs(got_phi - bphi[HALF, HALF, HALF])) <= 1e-5 * np.max(np.abs(bphi)), (center, plan)
        assert np.max(np.abs(got_pi - bpi[HALF, HALF, HALF])) <= 1e-5 * np.max(np.abs(bpi)), (center, plan)
    del phi, out_phi, out_pi
    torch.cuda.empty_cache()


def test_256cube_complex_energy_of_inputs(env, ora):
    """Full-lattice FP64 energy and checksums of seeded inputs (phi and a non-zero pi)."""
    torch, lf2 = env
    phi0 = inputs.gaussian_field(256, 256, 256, 2, sigma=0.1, seed=11)
    pi0 = inputs.gaussian_field(256, 256, 256, 2, sigma=0.05, seed=12)
    oe = ora.energy(phi0, pi0, **KW)
    p = lf2.params(**KW)
    for prec, tol in (("f64", 1e-12), ("f32k", 1e-6)):
        with lf2.System((256, 256, 256), 2, prec) as s:
            s.upload(phi0, pi0)
            e = lf2.lf2_energy(s.phi, s.pi, p)
        assert abs(e["total"] - oe["total"]) <= tol * abs(oe["total"]), prec
        for a in range(2):
            assert abs(e["sum_sq"][a] - oe["sum_sq"][a]) <= tol * oe["sum_sq"][a], prec


def _ensemble_fields(torch, lf2, members, prec, ncomp=1):
    """Library-owned phi/pi fields for each (side, lambda, seed), filled with the seeded device
    Gaussian (rounded to FP32 for FP32 storage).  Returns (fields, params, host initial data)."""
    fields, plist, hosts = [], [], []
    for side, lam, seed in members:
        dtype = torch.float64 if prec == lf2.LF2_F64 else torch.float32
        phi = inputs.gaussian_field_device(side, side, side, ncomp, sigma=0.1, seed=seed, dtype=dtype)
        host = phi.double().cpu().numpy()
        del phi
        lat = lf2.lf2_lattice_create((side, side, side))
        fphi = lf2.lf2_field_alloc(lat, ncomp, prec)
        fpi = lf2.lf2_field_alloc(lat, ncomp, prec)
        lf2.lf2_field_upload(fphi, host)
        fields.append((lat, fphi, fpi))
        plist.append(lf2.params(dx=1.0, dt=0.05, lam=lam, eta=1.0))
        hosts.append(host)
    return fields, plist, hosts


def _free(lf2, fields):
    for lat, fphi, fpi in fields:
        lf2.lf2_field_free(fphi)
        lf2.lf2_field_free(fpi)
        lf2.lf2_lattice_destroy(lat)


def test_ensemble_of_64_lattices_against_oracle_and_standalone(env, ora):
    """The 64-lattice ensemble (sides from {64, 96, 128, 160, 192}, lambda ~ U[0.5, 2], FP32 with
    the compensated drift, per-lattice seeds), one tuned graph launch of 13 steps:
      * members of every side (the first 64^3 and the first 192^3 among them), each with its own
        lambda, within a relative 1e-5 of the oracle at every element of phi and pi;
      * a spread of members bitwise equal to the same lattice evolved alone with the
        one-thread-per-site kernel."""
    torch, lf2 = env
    torch.cuda.empty_cache()
    members = inputs.ensemble_members()
    steps = 13
    stream = torch.cuda.current_stream()
    fields, plist, hosts = _ensemble_fields(torch, lf2, members, lf2.LF2_F32_KAHAN)
    try:
        for i, (lat, fphi, fpi) in enumerate(fields):
            lf2.lf2_leapfrog_init(fphi, fpi, plist[i], stream)
        e = lf2.lf2_ensemble_create([f[1] for f in fields], [f[2] for f in fields], plist)
        try:
            plan = lf2.lf2_ensemble_tune(e, stream=stream)
            lf2.lf2_ensemble_run(e, steps, stream)
            torch.cuda.synchronize()
            sides = [m[0] for m in members]
            pick = sorted({sides.index(sd) for sd in set(sides)} | {0, 63})
            for i in pick:
                side, lam = members[i][0], members[i][1]
                got = (lf2.lf2_field_download(fields[i][1], (side, side, side, 1)),
                       lf2.lf2_field_download(fields[i][2], (side, side, side, 1)))
                kw = dict(KW, lam=lam)
                ophi, opi = ora.evolve(hosts[i], np.zeros_like(hosts[i]), steps, half_kick=True, threads=THREADS, **kw)
                assert np.max(np.abs(got[0] - ophi)) <= 1e-5 * np.max(np.abs(ophi)), (i, side, plan)
                assert np.max(np.abs(got[1] - opi)) <= 1e-5 * np.max(np.abs(opi)), (i, side, plan)
            for i in (1, 17, 40):
                side = members[i][0]
                got = (lf2.lf2_field_download(fields[i][1], (side, side, side, 1)),
                       lf2.lf2_field_download(fields[i][2], (side, side, side, 1)))
                with lf2.System((side, side, side), 1, "f32k") as s:
                    s.upload(hosts[i], np.zeros_like(hosts[i]))
                    lf2.lf2_leapfrog_init(s.phi, s.pi, plist[i])
                    lf2.lf2_leapfrog_ex(s.phi, s.pi, plist[i], steps, kernel=lf2.LF2_KERNEL_SITE)
                    ref = s.download()
                assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), i
        finally:
            lf2.lf2_ensemble_destroy(e)
    finally:
        _free(lf2, fields)


@pytest.mark.parametrize("ncomp", [1, 2])
def test_fp64_ensemble_against_oracle(env, ora, ncomp):
    """An FP64 ensemble of five lattices of uneven sides (64^3 to 192^3, own lambda and seed),
    real and complex, temporal-blocking passes: every element of every member within a relative
    1e-12 of the oracle after 10 steps."""
    torch, lf2 = env
    members = [(64, 0.7, 901), (96, 1.9, 902), (128, 1.1, 903), (160, 0.55, 904), (192, 1.4, 905)]
    stream = torch.cuda.current_stream()
    fields, plist, hosts = _ensemble_fields(torch, lf2, members, lf2.LF2_F64, ncomp=ncomp)
    try:
        for i, (lat, fphi, fpi) in enumerate(fields):
            lf2.lf2_leapfrog_init(fphi, fpi, plist[i], stream)
        e = lf2.lf2_ensemble_create([f[1] for f in fields], [f[2] for f in fields], plist)
        try:
            lf2.lf2_ensemble_set_config(e, depth=3, cx=1, tile_x=26, tile_y=8)
            lf2.lf2_ensemble_run(e, STEPS, stream)
            torch.cuda.synchronize()
            for i, (side, lam, _) in enumerate(members):
                shape = (side, side, side, ncomp)
                got = (lf2.lf2_field_download(fields[i][1], shape), lf2.lf2_field_download(fields[i][2], shape))
                ophi, opi = ora.evolve(hosts[i], np.zeros_like(hosts[i]), STEPS, half_kick=True, threads=THREADS,
                                       **dict(KW, lam=lam))
                assert np.max(np.abs(got[0] - ophi)) <= 1e-12 * np.max(np.abs(ophi)), i
                assert np.max(np.abs(got[1] - opi)) <= 1e-12 * np.max(np.abs(opi)), i
        finally:
            lf2.lf2_ensemble_destroy(e)
    finally:
        _free(lf2, fields)
