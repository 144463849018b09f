"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the property it checks and the passage that fixes it.  None of them
retypes the oracle's formulas: they use exact shifts, exact cell averages of
polynomials and sines computed from antiderivatives, convergence order, conservation,
positivity, closed-form spectra and brute-force sums.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2110_15867_gb300 import inputs as I


def cell_avgs(antider, n, shift=0.0, L=1.0):
    """Exact cell averages of a function with antiderivative `antider` on n cells."""
    x = np.arange(n + 1) * (L / n)
    return (antider(x[1:] - shift) - antider(x[:-1] - shift)) * (n / L)


# ---------------------------------------------------------------------------
# 1D operator: Sec. 4.2 (SL-MPP5 = conservative SL flux + MP + positivity)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nu", [0.0, 1.0, 2.0, 5.0, -1.0, -3.0, 17.0, -40.0])
def test_integer_courant_is_exact_shift(nu):
    # A semi-Lagrangian step at integer Courant number moves every cell by exactly
    # nu cells (Eq. 3 has the exact solution f(x - u t / a^2)).
    c = np.random.default_rng(1).random(16)
    out = O.sweep_line(c, nu, periodic=True)
    assert np.array_equal(out, np.roll(c, int(nu)))


def test_fractional_flux_endpoints():
    # s -> 0 moves nothing; s -> 1 moves exactly the donor cell (the departure
    # interval is then the whole donor cell).
    st = np.array([0.3, 1.7, 0.2, 2.5, 0.9])
    assert O.sl5_raw_flux(st, 0.0) == 0.0
    assert O.sl5_raw_flux(st, 1.0) == pytest.approx(0.2, abs=1e-15)


@pytest.mark.parametrize("deg", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("nu", [0.3, 0.77, -0.45, 2.6, -3.2])
def test_polynomial_exactness_unlimited(deg, nu):
    # 5th order: cell averages of any polynomial of degree <= 4 are advected
    # exactly by the unlimited scheme (the interpolated primitive is then exact).
    rng = np.random.default_rng(deg)
    coef = rng.standard_normal(deg + 1)
    p = np.polynomial.Polynomial(coef)
    P = p.integ()
    n = 40
    c = cell_avgs(P, n)
    out = O.sweep_line(c, nu, periodic=True, flags=0)
    exact = cell_avgs(P, n, shift=nu / n)
    k = int(math.ceil(abs(nu))) + 4  # stay clear of the periodic seam
    sl = slice(k, n - k)
    assert np.max(np.abs(out[sl] - exact[sl])) < 1e-12 * max(1.0, np.abs(exact).max())


def _advect_sine(n, nu, flags, steps):
    P = lambda x: x - 0.5 / (2 * np.pi) * np.cos(2 * np.pi * x)  # 1 + 0.5 sin(2 pi x)
    c = cell_avgs(P, n)
    for _ in range(steps):
        c = O.sweep_line(c, nu, periodic=True, flags=flags)
    return np.abs(c - cell_avgs(P, n, shift=nu * steps / n)).mean()


@pytest.mark.parametrize("flags", [0, O.MPP])
def test_convergence_order_five(flags):
    # Spatially 5th-order accuracy (Sec. 4.1.1 and 4.2) with a single-stage step:
    # advect a smooth periodic profile about one period at nu = 0.7.
    errs = []
    for n in (32, 64, 128):
        errs.append(_advect_sine(n, 0.7, flags, int(round(n / 0.7))))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 4.7, orders


def test_limiter_inactive_on_resolved_smooth_data():
    # MP constraints must not clip smooth extrema (accuracy preservation of the
    # Suresh-Huynh constraint): on a resolved sine the limited and unlimited
    # updates agree to round-off.
    P = lambda x: x - 0.5 / (2 * np.pi) * np.cos(2 * np.pi * x)
    c = cell_avgs(P, 128)
    for nu in (0.1, 0.35, 0.7, 0.95, -0.6, 2.3):
        a = O.sweep_line(c, nu, flags=0)
        b = O.sweep_line(c, nu, flags=O.MPP)
        assert np.max(np.abs(a - b)) < 1e-14


@pytest.mark.parametrize("periodic", [True, False])
def test_conservation(periodic):
    # Finite-volume flux form: the update telescopes (periodic line, or zero-flux
    # outer faces on velocity lines), so the line sum is unchanged.
    rng = np.random.default_rng(7)
    for t in range(200):
        c = rng.random(24) ** 3
        nu = rng.uniform(-0.99, 0.99) if not periodic else rng.uniform(-5, 5)
        out = O.sweep_line(c, nu, periodic=periodic)
        assert abs(out.sum() - c.sum()) <= 1e-14 * c.sum()


def test_positivity_preserved():
    # Positivity preservation of SL-MPP5 (Sec. 4.2): non-negative data stay
    # non-negative, including a delta spike and sparse random data; the MP
    # constraint alone does not guarantee it.
    rng = np.random.default_rng(3)
    worst_mp, worst_mpp = 0.0, 0.0
    for t in range(3000):
        c = rng.random(12) ** 4 * (rng.random(12) < 0.5)
        nu = rng.uniform(-0.999, 0.999) if t % 2 else rng.uniform(-4, 4)
        per = bool(t % 2 == 0)
        worst_mp = min(worst_mp, O.sweep_line(c, nu, per, O.MP).min())
        worst_mpp = min(worst_mpp, O.sweep_line(c, nu, per, O.MPP).min())
    assert worst_mpp >= 0.0
    assert worst_mp < -1e-3  # the clamp is what keeps f >= 0
    spike = np.zeros(32)
    spike[5] = 1.0
    for _ in range(60):
        spike = O.sweep_line(spike, 0.55)
    assert spike.min() >= 0.0 and abs(spike.sum() - 1.0) < 1e-14


def test_mp_constraint_reflection_and_affine_invariance():
    # The Suresh-Huynh constraint is built from minmod (odd), paired min/max
    # bounds and a median, so it commutes with f -> -f and with f -> a f + b,
    # a > 0: increasing and decreasing data are limited alike.
    rng = np.random.default_rng(5)
    for _ in range(5000):
        st = rng.standard_normal(5)
        s = rng.uniform(0.01, 0.99)
        fb = 2.0 * rng.standard_normal()
        a, b = rng.uniform(0.5, 3.0), rng.standard_normal()
        l1 = O.mp_limit(fb, st, s)
        assert O.mp_limit(-fb, -st, s) == pytest.approx(-l1, abs=1e-12)
        assert O.mp_limit(a * fb + b, a * st + b, s) == pytest.approx(a * l1 + b, abs=1e-9)


def test_mp_constraint_never_clips_a_parabola():
    # Accuracy preservation at smooth extrema: for cell averages of any parabola
    # the exact mean over the departure interval passes the constraint untouched.
    rng = np.random.default_rng(0)
    edges = np.arange(-3, 3)
    for _ in range(5000):
        A = rng.choice([-1, 1]) * rng.uniform(0.1, 2.0)
        x0, B = rng.uniform(-4, 3), rng.uniform(-3, 3)
        P = lambda x: A * (x - x0) ** 3 / 3 + B * x
        st = P(edges[1:]) - P(edges[:-1])
        s = rng.uniform(0.02, 0.98)
        fb = (P(0) - P(-s)) / s
        assert O.mp_limit(fb, st, s) == pytest.approx(fb, abs=1e-12 * (1 + abs(fb)))


def _tv(c):
    return np.abs(np.diff(np.r_[c, c[0]])).sum()


def test_monotonicity_preserving_top_hat():
    # Monotonicity preservation (Sec. 4.2): a top hat advected 300 times with
    # mixed Courant numbers keeps its overshoot and total-variation growth at
    # the percent level, against more than 10 % for the unlimited scheme.  (The
    # Suresh-Huynh large-curvature bound allows small overshoots at corners.)
    c0 = ((np.arange(64) >= 20) & (np.arange(64) < 35)).astype(float)
    res = {}
    for flags in (0, O.MPP):
        c = c0.copy()
        mx, tvm = 0.0, 0.0
        for k in range(300):
            c = O.sweep_line(c, [0.7, -0.37, 0.93, 0.11][k % 4], True, flags)
            mx, tvm = max(mx, c.max()), max(tvm, _tv(c))
        res[flags] = (mx, tvm)
    assert res[0][0] > 1.10 and res[0][1] > 2.5
    assert res[O.MPP][0] < 1.02 and res[O.MPP][1] < 2.04


def test_mirror_of_free_streaming_exact_negative_velocity():
    # Negative Courant numbers advect toward lower index: compare with the exact
    # shifted cell averages of a smooth profile (closed form of Eq. 3).
    P = lambda x: x - 0.5 / (2 * np.pi) * np.cos(2 * np.pi * x)
    n = 64
    c = cell_avgs(P, n)
    out = O.sweep_line(c, -0.6)
    assert np.max(np.abs(out - cell_avgs(P, n, shift=-0.6 / n))) < 1e-8


def test_velocity_line_matches_periodic_away_from_edges():
    # A zero-flux velocity line with compact data far from its edges behaves as
    # the periodic operator: the outer faces carry nothing either way.
    c = np.zeros(24)
    c[8:16] = np.random.default_rng(2).random(8)
    for nu in (0.4, -0.8):
        a = O.sweep_line(c, nu, periodic=False)
        b = O.sweep_line(c, nu, periodic=True)
        assert np.array_equal(a, b)


# ---------------------------------------------------------------------------
# 6D sweeps: Eq. (3) free streaming, Eq. (4) velocity advection
# ---------------------------------------------------------------------------

def _plane_wave_f(g, k, A, t):
    """Exact cell averages of (1 + A sin(2 pi k.(x - u t))) F(u), discrete velocities."""
    n = list(g.n)
    nu = list(g.nu)
    Fu = I.fermi_dirac(nu, g.V)
    dx = [g.L / m for m in n]
    xc = [I.spatial_centres(m, g.L) for m in n]
    uc = [I.velocity_centres(m, g.V) for m in nu]
    sinc = np.prod([np.sinc(k[d] * dx[d] / g.L) for d in range(3)])
    X = np.meshgrid(*xc, indexing="ij")
    U = np.meshgrid(*uc, indexing="ij")
    phase_x = sum(k[d] * X[d] for d in range(3))[:, :, :, None, None, None]
    phase_u = sum(k[d] * U[d] for d in range(3))[None, None, None, :, :, :]
    wave = np.sin(2 * np.pi * (phase_x - phase_u * t) / g.L)
    return (1.0 + A * sinc * wave) * Fu[None, None, None]


@pytest.mark.parametrize("k", [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, -1)])
def test_free_streaming_closed_form(k):
    # phi = 0: f(x, u, t) = f0(x - u t / a^2, u) (Eq. 1 with no force).  The
    # drift D_x D_y D_z must reproduce it to the scheme's accuracy, converging
    # at 5th order.
    errs = []
    a = 1.3
    for n in (16, 32):
        g = O.grid(n, 2, V=5.0)
        dt = 0.7 * a * a * (g.L / n) / I.velocity_centres(2, g.V).max()
        f = _plane_wave_f(g, k, 0.3, 0.0)
        for ax in (2, 1, 0):
            O.sweep(g, f, ax, dt, a)
        exact = _plane_wave_f(g, k, 0.3, dt / a ** 2)
        errs.append(np.abs(f - exact).max() / exact.max())
    assert errs[1] < 1e-5
    assert math.log2(errs[0] / errs[1]) > 4.5


def test_sweeps_conserve_mass_6d():
    g = O.grid((6, 5, 7), (6, 8, 5), V=5.0)
    rng = np.random.default_rng(11)
    f = rng.random((6, 5, 7, 6, 8, 5)) ** 2
    phi = I.fourier_potential((6, 5, 7), seed=3)
    m0 = math.fsum(f.ravel())
    for ax in range(6):
        dt = 0.8 / max(O.max_abs_nu(g, ax, 1.0, 1.0, phi), 1e-30)
        O.sweep(g, f, ax, dt, 1.0, phi)
        assert abs(math.fsum(f.ravel()) - m0) < 1e-13 * m0
        assert f.min() >= 0.0


def test_velocity_sweep_uses_minus_grad_phi():
    # Eq. (4): each cell's velocity cube advects with speed -d phi/d x_i.  A
    # compact velocity profile in a spatially uniform f moves by the exact
    # single-line result with nu = -g dt / du, g the 4th-order gradient.
    g = O.grid(8, (12, 12, 12), V=3.0)
    phi = I.fourier_potential(8, seed=5)
    prof = np.zeros((12, 12, 12))
    prof[4:8, 3:9, 5:7] = np.random.default_rng(4).random((4, 6, 2)) + 0.5
    f = np.broadcast_to(prof, (8, 8, 8, 12, 12, 12)).copy()
    for ax in (3, 4, 5):
        d = ax - 3
        dt = 0.5 / O.max_abs_nu(g, ax, 1.0, 1.0, phi)
        grad = O.gradient(g, phi, d)
        h = f.copy()
        O.sweep(g, h, ax, dt, 1.0, phi)
        for cell in [(0, 0, 0), (3, 5, 1), (7, 2, 6)]:
            nu = -grad[cell] * dt / (2 * g.V / 12)
            line_in = np.moveaxis(f[cell], d, -1)
            line_out = np.moveaxis(h[cell], d, -1)
            for idx in [(4, 3), (7, 8), (5, 6)]:
                ref = O.sweep_line(line_in[idx], nu, periodic=True)
                assert np.array_equal(line_out[idx], ref)


# ---------------------------------------------------------------------------
# moment, gradient, Poisson
# ---------------------------------------------------------------------------

def test_moment_constant_and_bruteforce():
    # rho_nu = int f d^3u as the velocity-cell sum times du^3 (Sec. 4.1.3).
    g = O.grid((3, 4, 2), (6, 8, 10), V=2.5)
    f = np.full((3, 4, 2, 6, 8, 10), 0.37)
    rho, mass = O.moment(g, f)
    assert np.allclose(rho, 0.37 * (2 * 2.5) ** 3, rtol=1e-15, atol=0)
    assert mass == pytest.approx(0.37 * (2 * 2.5) ** 3, rel=1e-15)
    Fu = I.fermi_dirac((6, 8, 10), 2.5)
    delta = I.gaussian_field((3, 4, 2), 0.1, seed=1)
    f = I.initial_f(delta, Fu, np.float64)
    rho, mass = O.moment(g, f)
    du3 = (5.0 / 6) * (5.0 / 8) * (5.0 / 10)
    for idx in np.ndindex(3, 4, 2):
        assert rho[idx] == pytest.approx(du3 * math.fsum(f[idx].ravel()), rel=1e-15)
    dx3 = 1.0 / 24
    assert mass == pytest.approx(dx3 * math.fsum(rho.ravel()), rel=1e-15)


def test_gradient_single_mode_closed_form():
    # 4th-order central difference of sin: g = cos(kx) (8 sin kh - sin 2kh) / (6h).
    n = (16, 12, 10)
    g = O.grid(n, 2)
    for d in range(3):
        for m in (1, 3):
            x = I.spatial_centres(n[d])
            shape = [1, 1, 1]
            shape[d] = n[d]
            phi = np.broadcast_to(np.sin(2 * np.pi * m * x).reshape(shape), n).copy()
            h = 1.0 / n[d]
            kk = 2 * np.pi * m
            exact = np.cos(kk * x) * (8 * np.sin(kk * h) - np.sin(2 * kk * h)) / (6 * h)
            out = O.gradient(g, phi, d)
            assert np.allclose(out, np.broadcast_to(exact.reshape(shape), n), atol=1e-11)


@pytest.mark.parametrize("mode", [(1, 0, 0), (0, 2, 1), (-3, 1, 4), (8, 0, 0)])
def test_poisson_single_mode(mode):
    # Eq. (2) in Fourier space: nabla^2 phi = four_pi_G a^2 (rho - mean) gives
    # phi = -four_pi_G a^2 (rho - mean) / |k|^2 for a single mode.
    n = (16, 12, 10)
    g = O.grid(n, 2)
    X = np.meshgrid(*[I.spatial_centres(m) for m in n], indexing="ij")
    ph = 2 * np.pi * sum(mode[d] * X[d] for d in range(3))
    rho = 5.0 + np.cos(ph + 0.3)
    k2 = sum((2 * np.pi * mode[d]) ** 2 for d in range(3))
    a, G4 = 0.7, 2.5
    phi = O.poisson(g, rho, a, G4)
    assert np.allclose(phi, -G4 * a * a * np.cos(ph + 0.3) / k2, atol=1e-12)


# ---------------------------------------------------------------------------
# one step, Eq. (5)
# ---------------------------------------------------------------------------

def test_step_zero_potential_is_free_streaming():
    # With phi = 0 the kicks of Eq. (5) are identities (nu = 0) and the step is
    # the drift only, taken at the mid-step scale factor: compare with the closed
    # form f0(x - u dt / a_half^2, u).
    n = 32
    g = O.grid(n, 2, V=5.0)
    a_half, a_full = 1.1, 1.3
    dt = 0.7 * a_half ** 2 * (g.L / n) / I.velocity_centres(2, g.V).max()
    f = _plane_wave_f(g, (1, 1, -1), 0.3, 0.0)
    O.step(g, f, dt, a_half, a_full, np.zeros((n, n, n)))
    exact = _plane_wave_f(g, (1, 1, -1), 0.3, dt / a_half ** 2)
    assert np.abs(f - exact).max() / exact.max() < 1e-5


def test_step_conserves_mass_and_self_consistency():
    n, nu = 8, 8
    g = O.grid(n, nu, V=5.0)
    Fu = I.fermi_dirac(nu, 5.0)
    delta = I.gaussian_field(n, 0.05, seed=2)
    f = I.initial_f(delta, Fu, np.float64)
    bg = 3.0 * (1.0 + I.gaussian_field(n, 0.5, seed=3))
    rho0, m0 = O.moment(g, f)
    phi0 = O.poisson(g, rho0 + bg, 0.5, 1.0)
    phi1, rho1 = O.step(g, f, 0.01, 0.52, 0.55, phi0, rho_bg=bg, four_pi_G=1.0,
                        self_consistent=True)
    _, m1 = O.moment(g, f)
    assert abs(m1 - m0) < 1e-13 * m0
    assert f.min() >= 0.0
    assert np.allclose(phi1, O.poisson(g, rho1 + bg, 0.55, 1.0), atol=1e-14)


# ---------------------------------------------------------------------------
# the kicks of one step, Eq. (5): half steps, phi^n first, phi^{n+1} second
# ---------------------------------------------------------------------------
# Setup shared by the two pins below: 8 x 2 x 2 spatial cells with f and phi
# uniform along y and z (every y and z line is uniform, so D_y, D_z, D_uy and D_uz
# leave f unchanged bit for bit), 8^3 velocity cells with V = 4 (du = 1, u_j =
# j - 7/2), dyadic data.  dt and a_half make every x-drift Courant number
# u_j dt / (a_half^2 dx) a whole number of cells, so the drift of Eq. (3) is an
# exact translation.  phi is zero except at cells i0 - 1 and i0 + 1 and is chosen
# so that the periodic 4th-order gradient at i0 is a dyadic number: the kick
# Courant number -g (dt / 2) / du there is a whole number N, and Eq. (4) moves that
# cell's velocity cube by exactly N cells along u_x per kick.  The two outer
# neighbours i0 -+ 2 of i0 + 4 carry no potential either, so that cell's kick is
# the identity.

def _kick_pin_setup(a_levels):
    n, nu, V = (8, 2, 2), 8, 4.0
    g = O.grid(n, nu, V=V)
    rng = np.random.default_rng(21)
    prof = np.zeros((nu, nu, nu))
    # compact along u_x (j_x = 1, 2: room for shifts of up to 3 cells before the edge),
    # multiples of 1/16 in [1/2, 2): every difference and sum of the exact shifts is exact
    prof[1:3] = rng.integers(8, 32, size=(2, nu, nu)) / 16.0
    f = np.empty(n + (nu, nu, nu))
    for ix in range(n[0]):
        f[ix] = a_levels[ix] * prof
    return g, f, prof


def _phi_with_gradient_at(n, i0, ghalf):
    # phi along x only, nonzero at i0 -+ 1, such that the 4th-order central difference
    # [8 (phi_{i+1} - phi_{i-1}) - (phi_{i+2} - phi_{i-2})] / (12 dx) at i0 equals ghalf
    # (dx = 1/8, so 12 dx = 3/2 and the two values are +- 3 ghalf / 32)
    phi = np.zeros(n)
    phi[(i0 + 1) % n[0]] = 3.0 * ghalf / 32.0
    phi[(i0 - 1) % n[0]] = -3.0 * ghalf / 32.0
    return phi


def test_step_kicks_are_half_steps_with_phi_n():
    # Eq. (5) with an external potential: D_u(dt/2) D_x(dt) D_u(dt/2), both kicks with
    # phi.  dt / a_half^2 = 2 makes the x-drift Courant numbers 16 u_j = 8 (2 j - 7):
    # whole periods of the 8-cell line, so the drift is the identity.  With g = -1/4 at
    # cell 2 each half kick has nu = -g (dt / 2) / du = 1: the cube moves by exactly
    # 2 cells along u_x over the step (a kick of dt would move it by 4).  Cell 6 feels
    # no force and must come back bit for bit.  a_full = 3 is unused here (an x drift
    # at a_full would not be a whole-period translation).
    g, f, prof = _kick_pin_setup([1.0] * 8)
    n = (8, 2, 2)
    phi = _phi_with_gradient_at(n, 2, -0.25)
    dt, a_half, a_full = 8.0, 2.0, 3.0
    assert O.gradient(g, phi, 0)[2, 0, 0] == -0.25
    O.step(g, f, dt, a_half, a_full, phi)
    want = np.zeros_like(prof)
    want[3:5] = prof[1:3]
    for iy in range(2):
        for iz in range(2):
            assert np.array_equal(f[2, iy, iz], want)
            assert np.array_equal(f[6, iy, iz], prof)


def test_step_second_kick_uses_post_drift_potential():
    # Eq. (5), self-consistent: the first kick uses phi^n, the drift runs at a_half,
    # the density rho_nu of the drifted f plus rho_bg gives phi^{n+1} through Eq. (2)
    # at a_full, and the second kick uses phi^{n+1}.  dt / a_half^2 = 1 makes the x
    # drift a translation by half the box (Courant numbers 8 u_j = 4 (2 j - 7)), so
    # the drifted density differs from the initial one (the two halves of the box
    # hold f at levels 1 and 3/2).  phi^n gives nu = 1 at cell 2 (g = -1/2, dt / 2
    # = 2).  rho_bg is chosen so that phi^{n+1} = phi_T exactly when the density of
    # the drifted f is used: Laplacian(phi_T) / (4 pi G a_full^2) minus that density.
    # phi_T gives nu = 2 at cell 6.  Cell 2's cube, kicked by 1, lands on cell 6 and
    # is kicked by 2: 3 cells in all.  phi^n for the second kick would give 1 + 0,
    # the pre-drift density a phi^{n+1} whose nu at cell 6 is not 2, a kick of dt
    # 2 + 4; each fails this check.
    levels = [1.0] * 4 + [1.5] * 4
    g, f, prof = _kick_pin_setup(levels)
    n = (8, 2, 2)
    dt, a_half, a_full, G4 = 4.0, 2.0, 0.75, 1.0
    phi_n = _phi_with_gradient_at(n, 2, -0.5)
    phi_T = _phi_with_gradient_at(n, 6, -1.0)
    du3 = 1.0
    # density of the drifted f: the initial density translated by 4 cells along x
    # (each kick keeps every cell's mass: its velocity faces carry no flux)
    rho0 = np.array([levels[ix] * prof.sum() * du3 for ix in range(8)])
    rho_post = np.roll(rho0, 4)[:, None, None] * np.ones(n)
    kx = 2 * np.pi * np.fft.fftfreq(8) * 8
    lap = np.real(np.fft.ifftn(-(kx ** 2)[:, None, None] * np.fft.fftn(phi_T)))
    rho_bg = lap / (G4 * a_full ** 2) - rho_post
    phi_next, rho_nu = O.step(g, f, dt, a_half, a_full, phi_n, rho_bg=rho_bg, four_pi_G=G4,
                              self_consistent=True)
    assert np.allclose(rho_nu, rho_post, rtol=1e-14, atol=0)
    assert np.abs(phi_next - phi_T).max() < 1e-14
    want6 = np.zeros_like(prof)
    want6[4:6] = levels[2] * prof[1:3]
    for iy in range(2):
        for iz in range(2):
            assert np.abs(f[6, iy, iz] - want6).max() < 1e-12
            # cell 2 holds cell 6's cube, which neither kick moves (no force at 6 from
            # phi^n, none at 2 from phi_T)
            assert np.abs(f[2, iy, iz] - levels[6] * prof).max() < 1e-12


def test_sweep_cells_is_the_velocity_sweep_at_given_courant_numbers():
    # Eq. (4) with nu(x) given per spatial cell: with nu = -g dt / du (g the pinned
    # 4th-order gradient) it is the velocity sweep of orc_sweep bit for bit, and with
    # whole numbers per cell every cube moves by exactly that many cells
    n, nu, V = (4, 3, 5), (8, 12, 10), 5.0
    g = O.grid(n, nu, V=V)
    f0 = I.initial_f(I.gaussian_field(n, 0.1, seed=2), I.fermi_dirac(nu, V), np.float64)
    phi = I.fourier_potential(n, seed=6)
    for ax in (3, 4, 5):
        d = ax - 3
        dt = 0.6 / O.max_abs_nu(g, ax, 1.0, 1.0, phi)
        a = f0.copy()
        b = f0.copy()
        O.sweep(g, a, ax, dt, 1.0, phi)
        O.sweep_cells(g, b, ax, -O.gradient(g, phi, d) * dt / (2 * V / nu[d]))
        assert np.array_equal(a, b)
    prof = np.zeros(nu)
    prof[3:5, 4:7, 2:6] = np.random.default_rng(1).integers(8, 32, size=(2, 3, 4)) / 16.0
    f = np.broadcast_to(prof, n + nu).copy()
    shifts = np.random.default_rng(2).integers(-2, 3, size=n).astype(np.float64)
    O.sweep_cells(g, f, 3, shifts)
    for idx in np.ndindex(*n):
        assert np.array_equal(f[idx], np.roll(prof, int(shifts[idx]), axis=0))
