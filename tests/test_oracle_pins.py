"""Pins of the FP64 CPU oracle against facts that do not come from the oracle itself.

Each test checks the oracle against brute force on tiny lattices, a closed form, an exact
invariant of the scheme, or a symmetry; together they are chosen so that a dropped term, a
wrong sign, factor or index, or a transposed axis or component fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

from paper_1508_05610_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ brute-force helpers
def brute_laplacian(phi, dx):
    """7-point Laplacian by explicit (i +- 1) mod N coordinate arithmetic, one site at a time."""
    nz, ny, nx, c = phi.shape
    out = np.zeros_like(phi)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                for a in range(c):
                    s = 0.0
                    for (ddx, ddy, ddz) in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                        s += phi[(z + ddz) % nz, (y + ddy) % ny, (x + ddx) % nx, a] - phi[z, y, x, a]
                    out[z, y, x, a] = s / (dx * dx)
    return out


def plane_wave(shape, n_modes, amp, theta):
    """A cos(k.x + theta) with lattice wave numbers k_i = 2 pi n_i / N_i (coordinates in sites)."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    u = 2 * np.pi * (n_modes[0] * x / nx + n_modes[1] * y / ny + n_modes[2] * z / nz) + theta
    return amp * np.cos(u)


def lattice_omega(shape, n_modes, dx, m2):
    """Free-field lattice dispersion: omega^2 = m^2 + sum_i (2 sin(k_i dx / 2) / dx)^2."""
    nz, ny, nx = shape
    k = [2 * np.pi * n_modes[0] / (nx * dx), 2 * np.pi * n_modes[1] / (ny * dx), 2 * np.pi * n_modes[2] / (nz * dx)]
    return math.sqrt(m2 + sum((2 * math.sin(ki * dx / 2) / dx) ** 2 for ki in k))


# ------------------------------------------------------------------------- P1: halo
@pytest.mark.parametrize("shape", [(4, 4, 4), (5, 4, 3), (2, 3, 7)])
@pytest.mark.parametrize("ncomp", [1, 2])
def test_update_halo_is_periodic_image(ora, shape, ncomp):
    nz, ny, nx = shape
    g = np.random.default_rng(1)
    padded = np.full((nz + 2, ny + 2, nx + 2, ncomp), np.nan)
    padded[1:-1, 1:-1, 1:-1] = g.normal(size=(nz, ny, nx, ncomp))
    out = ora.update_halo(padded)
    interior = padded[1:-1, 1:-1, 1:-1]
    for pz in range(nz + 2):
        for py in range(ny + 2):
            for px in range(nx + 2):
                want = interior[(pz - 1) % nz, (py - 1) % ny, (px - 1) % nx]
                assert np.array_equal(out[pz, py, px], want), (pz, py, px)


def test_site_jumps_and_neighbours_match_paper_example(ora):
    """Golden: the paper's Site example and jump rule (Sec. 3.4)."""
    rows, jumps = [], None
    with open(os.path.join(GOLDEN, "site_neighbours.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            p = line.split()
            if p[0] == "jumps":
                jumps = [int(v) for v in p[1:]]
            else:
                rows.append((p[0], int(p[1]), int(p[2]), int(p[3]), int(p[4]), int(p[5])))
    nx, ny, nz, h, j0, j1, j2 = jumps
    assert (j0, j1, j2) == (1, nx + 2 * h, (nx + 2 * h) * (ny + 2 * h))
    # The oracle's padded layout (nz+2, ny+2, nx+2) in C order has exactly these jumps.
    pad = np.zeros((nz + 2, ny + 2, nx + 2, 1))
    strides = [s // pad.itemsize for s in pad.strides[:3]][::-1]
    assert strides == [j0, j1, j2]
    # Neighbour direction: a unit impulse at x + offset contributes +1/dx^2 to the Laplacian
    # at x, and the paper's offset table names those sites.
    x0 = (1, 2, 3)
    for _, dim, sign, ddx, ddy, ddz in rows:
        assert (ddx, ddy, ddz)[dim] == sign and sum(abs(v) for v in (ddx, ddy, ddz)) == 1
        phi = np.zeros((nz, ny, nx, 1))
        phi[(x0[2] + ddz) % nz, (x0[1] + ddy) % ny, (x0[0] + ddx) % nx, 0] = 1.0
        F = ora.force(phi, dx=1.0, lam=0.0, m2=0.0)
        assert F[x0[2], x0[1], x0[0], 0] == 1.0


# ------------------------------------------------------------------- P1: Laplacian
@pytest.mark.parametrize("shape", [(4, 4, 4), (5, 4, 3), (3, 6, 2)])
@pytest.mark.parametrize("ncomp", [1, 2])
@pytest.mark.parametrize("dx", [1.0, 0.5])
def test_laplacian_bruteforce_integer_exact(ora, shape, ncomp, dx):
    nz, ny, nx = shape
    phi = inputs.integer_field(nx, ny, nz, ncomp, seed=7)
    F = ora.force(phi, dx=dx, lam=0.0, m2=0.0)
    assert np.array_equal(F, brute_laplacian(phi, dx))


def test_potential_force_exact_values(ora):
    """Homogeneous fields: the Laplacian vanishes and F_a = -lambda phi_a (|phi|^2 - eta^2) - m2 phi_a.
    Values chosen so every product is exact; the complex case checks that |phi|^2 sums over
    both components (using phi_a^2 alone would give -1.5 and -8 instead of -2 and -4)."""
    phi = np.full((3, 3, 3, 1), 2.0)
    F = ora.force(phi, lam=1.0, eta=1.0, m2=0.25)
    assert np.all(F == -(2.0 * 3.0) - 0.25 * 2.0)
    phi2 = np.zeros((3, 3, 3, 2))
    phi2[..., 0], phi2[..., 1] = 1.0, 2.0
    F2 = ora.force(phi2, lam=0.5, eta=1.0, m2=0.0)
    assert np.all(F2[..., 0] == -2.0) and np.all(F2[..., 1] == -4.0)


# -------------------------------------------------------------- P2: free dispersion
@pytest.mark.parametrize("dx,dt,m2", [(1.0, 0.1, 0.3), (0.7, 0.05, 0.0), (1.3, 0.2, 1.1)])
def test_plane_wave_dispersion_closed_form(ora, dx, dt, m2):
    """lambda = 0: phi_n = A cos(k.x + theta) cos(n w dt), with (2/dt) sin(w dt/2) = omega and
    omega^2 = m^2 + sum_i (2 sin(k_i dx/2)/dx)^2; pi_{n-1/2} = (phi_n - phi_{n-1})/dt."""
    shape, modes, amp, theta = (16, 12, 8), (1, 2, 3), 0.8, 0.3
    phi0 = plane_wave(shape, modes, amp, theta)[..., None]
    omega = lattice_omega(shape, modes, dx, m2)
    w = 2.0 / dt * math.asin(omega * dt / 2.0)
    nsteps = 1000
    phi, pi = ora.evolve(phi0, np.zeros_like(phi0), nsteps, dx=dx, dt=dt, lam=0.0, m2=m2, half_kick=True)
    want_phi = phi0 * math.cos(nsteps * w * dt)
    want_pi = phi0 * (math.cos(nsteps * w * dt) - math.cos((nsteps - 1) * w * dt)) / dt
    assert np.max(np.abs(phi - want_phi)) <= 1e-11 * amp
    assert np.max(np.abs(pi - want_pi)) <= 1e-11 * amp / dt


def test_plane_wave_components_are_independent_and_ordered(ora):
    """Two components carrying different waves (lambda = 0): each follows its own dispersion,
    so swapping or mixing the interleaved components fails."""
    shape, dt, m2 = (8, 12, 16), 0.1, 0.2
    w0 = plane_wave(shape, (1, 0, 2), 0.5, 0.1)
    w1 = plane_wave(shape, (3, 1, 0), 0.7, -0.4)
    phi0 = np.stack([w0, w1], axis=-1)
    phi, _ = ora.evolve(phi0, np.zeros_like(phi0), 300, dt=dt, lam=0.0, m2=m2, half_kick=True)
    for a, modes, wave in ((0, (1, 0, 2), w0), (1, (3, 1, 0), w1)):
        w = 2.0 / dt * math.asin(lattice_omega(shape, modes, 1.0, m2) * dt / 2.0)
        assert np.max(np.abs(phi[..., a] - wave * math.cos(300 * w * dt))) <= 1e-12


# ------------------------------------------------------------ P3: linear invariant
def test_linear_invariant_exact(ora):
    """lambda = 0, A = -lap + m^2 (symmetric): I_{n+1/2} = |pi_{n+1/2}|^2/2 + <phi_n, A phi_{n+1}>/2
    is conserved exactly by the staggered leapfrog.  A is applied here by brute force."""
    shape, m2, dt = (6, 5, 4), 0.4, 0.15
    nz, ny, nx = shape
    phi0 = inputs.gaussian_field(nx, ny, nz, 2, sigma=0.3, seed=11)
    pi0 = inputs.gaussian_field(nx, ny, nz, 2, sigma=0.2, seed=12)

    def A(v):
        return -brute_laplacian(v, 1.0) + m2 * v

    vals = []
    for n in (0, 7, 40):
        phin, _ = ora.evolve(phi0, pi0, n, dt=dt, lam=0.0, m2=m2)
        phin1, pin1 = ora.evolve(phi0, pi0, n + 1, dt=dt, lam=0.0, m2=m2)
        vals.append(0.5 * np.sum(pin1 ** 2) + 0.5 * np.sum(phin * A(phin1)))
    assert max(abs(v - vals[0]) for v in vals) <= 1e-13 * abs(vals[0])


# ------------------------------------------------------------- P5: homogeneous field
def test_homogeneous_real_converges_to_ode(ora):
    """Homogeneous phi^4 field: the lattice is a single anharmonic oscillator with
    V = lambda/4 (phi^2 - eta^2)^2.  Sites stay bitwise identical, and the trajectory converges to
    an accurate ODE solution at second order in dt."""
    scipy_integrate = pytest.importorskip("scipy.integrate")
    lam, eta, phi_init, t_end = 1.3, 0.9, 0.35, 4.0

    def rhs(_, s):
        return [s[1], -lam * s[0] * (s[0] ** 2 - eta ** 2)]

    exact = scipy_integrate.solve_ivp(rhs, (0, t_end), [phi_init, 0.0], rtol=1e-13, atol=1e-15,
                                      method="DOP853").y[0, -1]
    errs = []
    for dt in (0.04, 0.02, 0.01):
        n = int(round(t_end / dt))
        phi0 = np.full((3, 4, 5, 1), phi_init)
        phi, _ = ora.evolve(phi0, np.zeros_like(phi0), n, dt=dt, lam=lam, eta=eta, half_kick=True)
        assert np.all(phi == phi[0, 0, 0, 0])
        errs.append(abs(phi[0, 0, 0, 0] - exact))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_homogeneous_energy_conserved_to_dt2(ora):
    """E = pi^2/2 + lambda/4 (phi^2 - eta^2)^2, written here from the potential alone, is conserved
    to O(dt^2) only if the oracle's force is -dV/dphi."""
    lam, eta, phi_init, t_end = 1.0, 1.0, 0.2, 6.0

    def drift(dt):
        n = int(round(t_end / dt))
        phi = np.full((3, 3, 3, 1), phi_init)
        pi = np.zeros_like(phi)
        e0 = lam / 4 * (phi_init ** 2 - eta ** 2) ** 2
        worst = 0.0
        phi, pi = ora.evolve(phi, pi, 0, dt=dt, lam=lam, eta=eta, half_kick=True)
        for _ in range(0, n, 10):
            phi, pi = ora.evolve(phi, pi, 10, dt=dt, lam=lam, eta=eta)
            f = -lam * phi[0, 0, 0, 0] * (phi[0, 0, 0, 0] ** 2 - eta ** 2)
            pin = pi[0, 0, 0, 0] + 0.5 * dt * f
            e = 0.5 * pin ** 2 + lam / 4 * (phi[0, 0, 0, 0] ** 2 - eta ** 2) ** 2
            worst = max(worst, abs(e - e0))
        return worst

    d1, d2 = drift(0.1), drift(0.05)
    assert d1 < 1e-2 * 0.25 and 3.0 < d1 / d2 < 5.0


def test_complex_circular_orbit_exact(ora):
    """Complex homogeneous field on a circle of radius r: with Omega^2 = lambda (r^2 - eta^2) + m^2
    the discrete orbit phi_n = r (cos n th, sin n th), 2 (1 - cos th) = dt^2 Omega^2, is exact for
    the scheme when pi_0 = (0, r sin th / dt)."""
    r, lam, eta, m2, dt, n = 1.5, 1.0, 1.0, 0.1, 0.05, 400
    Om2 = lam * (r * r - eta * eta) + m2
    th = math.acos(1 - dt * dt * Om2 / 2)
    phi0 = np.zeros((2, 3, 4, 2))
    phi0[..., 0] = r
    pi0 = np.zeros_like(phi0)
    pi0[..., 1] = r * math.sin(th) / dt
    phi, _ = ora.evolve(phi0, pi0, n, dt=dt, lam=lam, eta=eta, m2=m2, half_kick=True)
    assert np.max(np.abs(phi[..., 0] - r * math.cos(n * th))) <= 1e-12
    assert np.max(np.abs(phi[..., 1] - r * math.sin(n * th))) <= 1e-12


def test_fixed_points_stay_fixed(ora):
    for v in (0.0, 1.0, -1.0):
        phi0 = np.full((4, 4, 4, 1), v)
        phi, pi = ora.evolve(phi0, np.zeros_like(phi0), 50, dt=0.1, lam=1.0, eta=1.0, half_kick=True)
        assert np.all(phi == v) and np.all(pi == 0.0)


# ----------------------------------------------------------------------- energy pins
def test_energy_closed_form_plane_wave(ora):
    """phi_n = A cos(u), pi_n = B cos(u') with lattice plane waves (no aliasing of 2k, 4k):
    kinetic = dx^3 V B^2/4, gradient = dx^3 V A^2 sum_i (1 - cos k_i dx)/(2 dx^2),
    potential = dx^3 V [lambda/4 (3A^4/8 - A^2 eta^2 + eta^4) + m2 A^2/4]."""
    shape, dx, dt, lam, eta, m2 = (8, 12, 16), 0.8, 0.1, 0.7, 1.1, 0.3
    modes, A, B = (1, 1, 1), 0.6, 0.45
    nz, ny, nx = shape
    V = nx * ny * nz
    phi = plane_wave(shape, modes, A, 0.2)[..., None]
    pin = plane_wave(shape, (2, 1, 3), B, -0.5)[..., None]
    F = ora.force(phi, dx=dx, lam=lam, eta=eta, m2=m2)
    pi_half = pin - 0.5 * dt * F  # energy() re-synchronises pi_{n-1/2} with +dt/2 F
    e = ora.energy(phi, pi_half, dx=dx, dt=dt, lam=lam, eta=eta, m2=m2)
    k = [2 * np.pi * modes[0] / nx, 2 * np.pi * modes[1] / ny, 2 * np.pi * modes[2] / nz]
    vol = dx ** 3
    assert e["kinetic"] == pytest.approx(vol * V * B * B / 4, rel=1e-12)
    assert e["gradient"] == pytest.approx(vol * V * A * A * sum(1 - math.cos(kk) for kk in k) / (2 * dx * dx), rel=1e-12)
    pot = vol * V * (lam / 4 * (3 * A ** 4 / 8 - A * A * eta * eta + eta ** 4) + m2 * A * A / 4)
    assert e["potential"] == pytest.approx(pot, rel=1e-12)
    assert e["total"] == pytest.approx(e["kinetic"] + e["gradient"] + e["potential"], rel=1e-15)


@pytest.mark.parametrize("ncomp", [1, 2])
def test_energy_gradient_is_minus_force(ora, ncomp):
    """With dt = 0 (so pi_n = pi), dE/dphi_a(x) = -dx^3 F_a(x): the forward-difference gradient
    energy and the potential are consistent with the 7-point Laplacian and the force."""
    nx, ny, nz = 5, 4, 6
    dx, lam, eta, m2 = 0.9, 1.2, 0.8, 0.15
    phi = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.5, seed=3)
    pi = inputs.gaussian_field(nx, ny, nz, ncomp, sigma=0.5, seed=4)
    F = ora.force(phi, dx=dx, lam=lam, eta=eta, m2=m2)
    h = 1e-5
    for (z, y, x, a) in [(0, 0, 0, 0), (5, 3, 4, ncomp - 1), (2, 1, 3, 0)]:
        p, m = phi.copy(), phi.copy()
        p[z, y, x, a] += h
        m[z, y, x, a] -= h
        ep = ora.energy(p, pi, dx=dx, dt=0.0, lam=lam, eta=eta, m2=m2)["total"]
        em = ora.energy(m, pi, dx=dx, dt=0.0, lam=lam, eta=eta, m2=m2)["total"]
        assert (ep - em) / (2 * h) == pytest.approx(-dx ** 3 * F[z, y, x, a], rel=1e-7, abs=1e-9)


def test_checksums(ora):
    phi = inputs.gaussian_field(7, 5, 3, 2, sigma=1.0, seed=9)
    e = ora.energy(phi, np.zeros_like(phi))
    for a in range(2):
        assert e["sum"][a] == math.fsum(phi[..., a].ravel())
        assert e["sum_sq"][a] == pytest.approx(math.fsum((phi[..., a] ** 2).ravel()), rel=1e-15)


# ------------------------------------------------------------------ P4: nonlinear run
def test_energy_conservation_scales_as_dt2(ora):
    nx = ny = nz = 12
    phi0 = inputs.gaussian_field(nx, ny, nz, 1, sigma=0.1, seed=inputs.BASE_SEED)

    def max_drift(dt, t_end=8.0, every=0.4):
        phi, pi = ora.evolve(phi0, np.zeros_like(phi0), 0, dt=dt, half_kick=True)
        e0 = ora.energy(phi, pi, dt=dt)["total"]
        worst, k = 0.0, int(round(every / dt))
        for _ in range(int(round(t_end / every))):
            phi, pi = ora.evolve(phi, pi, k, dt=dt)
            worst = max(worst, abs(ora.energy(phi, pi, dt=dt)["total"] - e0) / abs(e0))
        return worst

    d1, d2 = max_drift(0.1), max_drift(0.05)
    print(d1, d2, d1 / d2)
    assert d1 < 5e-3
    assert 3.0 < d1 / d2 < 5.0


# ------------------------------------------------------------------- P6, P7: symmetry
def test_translation_z2_u1_bitwise(ora):
    nx, ny, nz = 6, 5, 4
    phi0 = inputs.gaussian_field(nx, ny, nz, 2, sigma=0.4, seed=21)
    pi0 = inputs.gaussian_field(nx, ny, nz, 2, sigma=0.1, seed=22)
    kw = dict(dt=0.1, lam=1.0, eta=1.0, m2=0.05, half_kick=True)
    phi, pi = ora.evolve(phi0, pi0, 15, **kw)
    sh = (1, 3, 2)
    tphi, tpi = ora.evolve(np.roll(phi0, sh, axis=(0, 1, 2)), np.roll(pi0, sh, axis=(0, 1, 2)), 15, **kw)
    assert np.array_equal(tphi, np.roll(phi, sh, axis=(0, 1, 2))) and np.array_equal(tpi, np.roll(pi, sh, axis=(0, 1, 2)))
    zphi, zpi = ora.evolve(-phi0, -pi0, 15, **kw)
    assert np.array_equal(zphi, -phi) and np.array_equal(zpi, -pi)

    def rot(v):
        return np.stack([-v[..., 1], v[..., 0]], axis=-1)

    uphi, upi = ora.evolve(rot(phi0), rot(pi0), 15, **kw)
    assert np.array_equal(uphi, rot(phi)) and np.array_equal(upi, rot(pi))


def test_time_reversibility(ora):
    nx, ny, nz, n = 6, 6, 6, 40
    kw = dict(lam=1.0, eta=1.0)
    dt = 0.05
    phi0 = inputs.gaussian_field(nx, ny, nz, 1, sigma=0.3, seed=5)
    pi_h = inputs.gaussian_field(nx, ny, nz, 1, sigma=0.1, seed=6)  # pi_{-1/2}
    phi, pi = ora.evolve(phi0, pi_h, n, dt=dt, **kw)
    pi = pi + dt * ora.force(phi, dt=dt, **kw)  # pi_{n+1/2}
    back, _ = ora.evolve(phi, pi, n, dt=-dt, **kw)
    assert np.max(np.abs(back - phi0)) <= 1e-12


def test_threads_bitwise_and_light_cone_box(ora):
    nx = ny = nz = 14
    phi0 = inputs.gaussian_field(nx, ny, nz, 1, seed=31)
    kw = dict(dt=0.1, lam=1.0, eta=1.0, half_kick=True)
    phi1, pi1 = ora.evolve(phi0, np.zeros_like(phi0), 5, threads=1, **kw)
    phi4, pi4 = ora.evolve(phi0, np.zeros_like(phi0), 5, threads=4, **kw)
    assert np.array_equal(phi1, phi4) and np.array_equal(pi1, pi4)
    half = 6
    for center in [(0, 0, 0), (13, 7, 2), (5, 11, 13)]:
        box = ora.light_cone_box(phi0, center, half)
        bphi, bpi = ora.evolve(box, np.zeros_like(box), half - 1, **kw)
        full, fpi = ora.evolve(phi0, np.zeros_like(phi0), half - 1, **kw)
        cx, cy, cz = center
        assert np.array_equal(bphi[half, half, half], full[cz, cy, cx])
        assert np.array_equal(bpi[half, half, half], fpi[cz, cy, cx])


# ------------------------------------------------- O(N) fields and the derivative operation
@pytest.mark.parametrize("ncomp", [3, 6])
def test_on_components_dispersion_and_coupling(ora, ncomp):
    """N-component fields: with lambda = 0 each component follows its own plane-wave dispersion;
    with lambda != 0 a homogeneous field's force couples all components through |phi|^2."""
    shape, dt, m2 = (8, 12, 16), 0.1, 0.2
    waves = [plane_wave(shape, (a % 3 + 1, (a + 1) % 3, a % 2), 0.3 + 0.1 * a, 0.2 * a) for a in range(ncomp)]
    phi0 = np.stack(waves, axis=-1)
    phi, _ = ora.evolve(phi0, np.zeros_like(phi0), 200, dt=dt, lam=0.0, m2=m2, half_kick=True)
    for a in range(ncomp):
        modes = (a % 3 + 1, (a + 1) % 3, a % 2)
        w = 2.0 / dt * math.asin(lattice_omega(shape, modes, 1.0, m2) * dt / 2.0)
        assert np.max(np.abs(phi[..., a] - waves[a] * math.cos(200 * w * dt))) <= 1e-12
    vals = np.arange(1, ncomp + 1, dtype=np.float64) * 0.5
    hom = np.broadcast_to(vals, (3, 3, 3, ncomp)).copy()
    F = ora.force(hom, lam=0.5, eta=1.0, m2=0.0)
    s2 = float(np.sum(vals * vals))
    assert np.allclose(F, -0.5 * vals * (s2 - 1.0), rtol=1e-15, atol=0)


@pytest.mark.parametrize("dim", [0, 1, 2])
def test_derivative_bruteforce_and_plane_wave(ora, dim):
    nz, ny, nx = 5, 6, 7
    phi = inputs.integer_field(nx, ny, nz, 3, seed=81)
    d = ora.derivative(phi, dim, dx=0.5)
    axis = 2 - dim  # arrays are (z, y, x, c)
    want = (np.roll(phi, -1, axis=axis) - np.roll(phi, 1, axis=axis)) / (2 * 0.5)
    assert np.array_equal(d, want)
    # plane wave: (cos(u + k) - cos(u - k)) / 2 = -sin(k) sin(u), with k along dim
    shape, modes = (16, 12, 8), [0, 0, 0]
    modes[dim] = 1
    w = plane_wave(shape, tuple(modes), 1.0, 0.3)[..., None]
    n_dim = (shape[2], shape[1], shape[0])[dim]
    k = 2 * np.pi / n_dim
    z, y, x = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), np.arange(shape[2]), indexing="ij")
    u = 2 * np.pi * (modes[0] * x / shape[2] + modes[1] * y / shape[1] + modes[2] * z / shape[0]) + 0.3
    assert np.max(np.abs(ora.derivative(w, dim)[..., 0] + math.sin(k) * np.sin(u))) <= 1e-14


# ------------------------------------------------------------- power spectrum (diagnostic)
def test_power_spectrum_parseval_and_plane_wave(ora):
    """Parseval: sum over modes of |phi~|^2 / V = sum_x phi^2, so sum_b P_b n_b equals the field's
    sum of squares when every mode falls in a bin; a plane wave A cos(k.x) puts V A^2 / 2 of
    power into the two modes +-k, i.e. the bin of |k| holds P = V A^2 / 4 per mode."""
    N = 8
    phi = inputs.gaussian_field(N, N, N, 2, sigma=1.0, seed=91)
    P, K, n = ora.power_spectrum(phi, comp=1, nbins=64)
    assert n.sum() == N ** 3
    assert np.sum(P * n) == pytest.approx(np.sum(phi[..., 1] ** 2), rel=1e-12)
    A, modes = 0.7, (2, 1, 3)
    w = plane_wave((N, N, N), modes, A, 0.0)
    P, K, n = ora.power_spectrum(w[..., None], nbins=64)
    b = math.isqrt(sum(m * m for m in modes))
    assert P[b] * n[b] == pytest.approx(N ** 3 * A * A / 2, rel=1e-12)
    assert np.sum(P * n) == pytest.approx(N ** 3 * A * A / 2, rel=1e-12)
    # all components (comp = -1): Parseval over both components, and for a complex field the
    # shell means of |FFT(re + i im)|^2 / V (one complex transform, an independent route: the
    # cross terms of the two components cancel between k and -k, which share a shell)
    P, K, n = ora.power_spectrum(phi, comp=-1, nbins=64)
    assert np.sum(P * n) == pytest.approx(np.sum(phi ** 2), rel=1e-12)
    Z = np.abs(np.fft.fftn(phi[..., 0] + 1j * phi[..., 1])) ** 2 / N ** 3
    m = np.fft.fftfreq(N) * N
    shell = np.floor(np.sqrt(m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2) + 1e-9).astype(int)
    for b in range(int(shell.max()) + 1):
        sel = shell == b
        assert n[b] == sel.sum(), b
        assert P[b] == pytest.approx(Z[sel].mean(), rel=1e-12), b
    # mode counts of the first shells of an 8^3 lattice: |m|^2 = 0 | 1,2,3 | 4..8 ...
    assert n[0] == 1 and n[1] == 6 + 12 + 8
