"""Pins of the oracle's adjoint (reverse mode of the sweeps and of one Eq. (5) step).

A sweep is piecewise linear in f (every limiter operation is a selection or a linear
combination) and piecewise polynomial in the Courant number, so a central difference
that stays inside one branch is exact up to rounding: the adjoint must satisfy the
dot-product identity <J v, w> = <v, J^T w> against such differences, and samples whose
one-sided differences disagree (a kink within +-h) are rejected.
"""
import numpy as np
import pytest

import oracle as O
from paper_2110_15867_gb300 import inputs as I


def test_dual_flux_matches_plain_flux():
    rng = np.random.default_rng(0)
    for _ in range(3000):
        st = rng.random(5) * (rng.random(5) < 0.8)
        s = rng.uniform(0.01, 0.99)
        for flags in (0, O.MP, O.MPP):
            F, _ = O.frac_flux_grad(st, s, flags)
            assert F == pytest.approx(O.frac_flux(st, s, flags), abs=1e-14)


def _fd_ok(f, x, v, h, mag=None):
    """Central difference of f at x along v, or None if a kink lies within +-h.
    mag: size of the terms summed into f (for the rounding estimate), default |f|."""
    fp, f0, fm = f(x + h * v), f(x), f(x - h * v)
    c = (fp - fm) / (2 * h)
    a, b = (fp - f0) / h, (f0 - fm) / h
    # one-sided quotients differ by O(h) curvature (none inside a branch) plus rounding
    rnd = 64 * np.finfo(float).eps * (np.max(np.abs(f0)) if mag is None else mag) / h
    if np.max(np.abs(a - b)) > 1e-6 * np.max(np.abs(c)) + rnd:
        return None
    _fd_ok.rounding = rnd
    return c


def test_flux_gradient_matches_differences():
    rng = np.random.default_rng(1)
    checked = 0
    for _ in range(2000):
        st = rng.random(5)
        s = rng.uniform(0.05, 0.95)
        F, gr = O.frac_flux_grad(st, s, O.MPP)
        x = np.r_[st, s]
        f = lambda y: np.array([O.frac_flux(y[:5], y[5], O.MPP)])
        for k in range(6):
            e = np.zeros(6)
            e[k] = 1.0
            c = _fd_ok(f, x, e, 1e-7)
            if c is None:
                continue
            checked += 1
            assert abs(c[0] - gr[k]) <= 1e-6 * abs(gr[k]) + _fd_ok.rounding
    assert checked > 8000


@pytest.mark.parametrize("periodic", [True, False])
def test_line_adjoint_dot_product(periodic):
    rng = np.random.default_rng(2)
    n = 20
    checked = 0
    for t in range(300):
        c = rng.random(n) + 0.1 * (t % 2)
        nu = rng.uniform(-0.97, 0.97) if not periodic else rng.uniform(-3.5, 3.5)
        v, w = rng.standard_normal(n), rng.standard_normal(n)
        f = lambda y: O.sweep_line(y, nu, periodic)
        jv = _fd_ok(f, c, v, 1e-7)
        if jv is None:
            continue
        jtw, _ = O.sweep_line_adjoint(c, w, nu, periodic)
        checked += 1
        # a difference quotient carries ~eps/h of rounding per element
        scale = np.linalg.norm(v) * np.linalg.norm(w)
        assert abs(np.dot(jv, w) - np.dot(v, jtw)) <= 1e-7 * scale + _fd_ok.rounding * np.linalg.norm(w) * np.sqrt(n)
    assert checked > 200


@pytest.mark.parametrize("periodic", [True, False])
def test_line_adjoint_courant_derivative(periodic):
    rng = np.random.default_rng(3)
    n = 16
    checked = 0
    for _ in range(300):
        c = rng.random(n)
        nu = rng.uniform(0.05, 0.95) * rng.choice([-1, 1])
        w = rng.standard_normal(n)
        f = lambda y: np.array([np.dot(O.sweep_line(c, y[0], periodic), w)])
        d = _fd_ok(f, np.array([nu]), np.array([1.0]), 1e-7)
        if d is None:
            continue
        _, dnu = O.sweep_line_adjoint(c, w, nu, periodic)
        checked += 1
        assert abs(d[0] - dnu) <= 1e-6 * abs(dnu) + _fd_ok.rounding
    assert checked > 200


@pytest.mark.parametrize("axis", [0, 1, 2, 3, 4, 5])
def test_sweep_adjoint_dot_product_and_potential(axis):
    # 6D sweep: <J v, w> = <v, J^T w>; velocity sweeps also dL/dphi through the
    # 4th-order gradient, checked by a central difference in phi.
    n, nu = (6, 5, 4), (8, 4, 6)
    g = O.grid(n, nu, V=3.0)
    rng = np.random.default_rng(10 + axis)
    f0 = I.initial_f(I.gaussian_field(n, 0.05, seed=1), I.fermi_dirac(nu, 3.0), np.float64)
    phi = I.fourier_potential(n, seed=2)
    dt = 0.6 / O.max_abs_nu(g, axis, 1.0, 1.0, phi)
    v, w = rng.standard_normal(f0.shape), rng.standard_normal(f0.shape)

    def S(x, ph=phi):
        y = x.copy()
        O.sweep(g, y, axis, dt, 1.0, ph)
        return y

    jv = _fd_ok(S, f0, v, 1e-7)
    lam = w.copy()
    dLdg = O.sweep_adjoint(g, f0, lam, axis, dt, 1.0, phi)
    if jv is not None:
        scale = np.linalg.norm(v) * np.linalg.norm(w)
        assert abs(np.sum(jv * w) - np.sum(v * lam)) <= 1e-7 * scale + _fd_ok.rounding * np.linalg.norm(w) * np.sqrt(w.size)
    if axis >= 3:
        dphi = np.zeros(n)
        O.gradient_adjoint(g, dLdg, axis - 3, dphi)
        p = rng.standard_normal(n)
        L = lambda ph: np.array([np.sum(S(f0, ph) * w)])
        d = _fd_ok(L, phi, p, 1e-7)
        assert d is not None
        assert abs(d[0] - np.sum(dphi * p)) <= 1e-6 * abs(np.sum(dphi * p)) + _fd_ok.rounding


def test_step_adjoint_finite_differences_8cubed():
    # One Eq. (5) step with an external potential at 8^3 x 8^3 (FP64): dL/df^n and
    # dL/dphi from the adjoint against central differences with 1e-6 relative
    # perturbations of single cells of f and of phi, for L = <w, f^{n+1}>; samples
    # with a limiter kink inside +-h are rejected.
    n, nu = 8, 8
    g = O.grid(n, nu, V=5.0)
    f0 = I.initial_f(I.gaussian_field(n, 0.05, seed=4), I.fermi_dirac(nu, 5.0), np.float64)
    phi = I.fourier_potential(n, seed=5)
    dt = min(0.7 / O.max_abs_nu(g, ax, 1.0, 1.0, phi) * (2 if ax >= 3 else 1) for ax in range(6))
    rng = np.random.default_rng(6)
    w = rng.standard_normal(f0.shape)
    mag = np.sum(np.abs(f0 * w))

    def L_of(f, ph):
        y = f.copy()
        O.step(g, y, dt, 1.0, 1.0, ph)
        return np.array([np.sum(y * w)])

    lam = w.copy()
    dphi = O.step_adjoint(g, f0, lam, dt, 1.0, phi)
    ok_f = ok_p = 0
    for t in range(20):
        k = tuple(rng.integers(0, m) for m in f0.shape)
        v = np.zeros_like(f0)
        v[k] = f0[k]
        d = _fd_ok(lambda f: L_of(f, phi), f0, v, 1e-6, mag)
        if d is not None:
            ok_f += 1
            assert abs(d[0] - lam[k] * f0[k]) <= 1e-6 * abs(lam[k] * f0[k]) + _fd_ok.rounding
        q = tuple(rng.integers(0, n, size=3))
        p = np.zeros_like(phi)
        p[q] = np.abs(phi).max()
        d = _fd_ok(lambda ph: L_of(f0, ph), phi, p, 1e-6, mag)
        if d is not None:
            ok_p += 1
            assert abs(d[0] - dphi[q] * p[q]) <= 1e-5 * abs(dphi[q] * p[q]) + _fd_ok.rounding
    assert ok_f >= 8 and ok_p >= 8, (ok_f, ok_p)


def test_poisson_is_its_own_transpose():
    # phi = P rho is a real circulant with an even multiplier: <P x, y> = <x, P y>
    g = O.grid((6, 8, 5), (4, 4, 4))
    rng = np.random.default_rng(21)
    x, y = rng.standard_normal((2, 6, 8, 5))
    px, py = O.poisson(g, x, 0.7, 1.3), O.poisson(g, y, 0.7, 1.3)
    a, b = float((px * y).sum()), float((x * py).sum())
    assert abs(a - b) <= 1e-13 * max(abs(a), 1.0)


def test_self_consistent_step_adjoint_matches_differences():
    # L = <w_f, f^{n+1}> + <w_phi, phi^{n+1}> for one self-consistent step: the adjoint's
    # directional derivatives along f_n, phi_n and rho_bg against one-sided differences.
    # The step is piecewise linear in f with many switching surfaces, so f is moved by
    # h = 1e-8 (one side must stay on one linear piece); phi_n and rho_bg enter through
    # the Courant numbers and the Poisson solve, smoothly almost everywhere, and are moved
    # by 1e-5 and 1e-6 where FP64 rounding of the differences is smaller.  Differences of
    # L are formed from differences of the outputs (no cancellation in the sums).
    n, nu = (6, 6, 6), (8, 8, 8)
    V = 5.0
    g = O.grid(n, nu, V=V)
    f0 = I.initial_f(I.gaussian_field(n, 0.05, seed=2), I.fermi_dirac(nu, V), np.float64)
    bg = 3.0 * (1.0 + I.gaussian_field(n, 0.5, seed=4))
    rho0, _ = O.moment(g, f0)
    phi0 = O.poisson(g, rho0 + bg, 0.5, 1.0)
    dt, ah, af = 0.02, 0.52, 0.55
    rng = np.random.default_rng(8)
    wf = rng.standard_normal(f0.shape)
    wp = rng.standard_normal(n)

    def out(f, p, b):
        f = f.copy()
        p1, _ = O.step(g, f, dt, ah, af, p, rho_bg=b, self_consistent=True)
        return f, p1

    lam = wf.copy()
    dphi, dbg = O.step_adjoint_sc(g, f0, lam, dt, ah, af, phi0, bg, 1.0, lam_phi_next=wp)
    F0, P0 = out(f0, phi0, bg)
    dirs = [(f0 * rng.standard_normal(n)[..., None, None, None], 0, 0, 1e-8),
            (0, phi0.std() * rng.standard_normal(n), 0, 1e-5),
            (0, 0, bg.std() * rng.standard_normal(n), 1e-6)]
    for ef, ep, eb, h in dirs:
        an = float((lam * ef).sum() + (dphi * ep).sum() + (dbg * eb).sum())
        Fp, Pp = out(f0 + h * ef, phi0 + h * ep, bg + h * eb)
        Fm, Pm = out(f0 - h * ef, phi0 - h * ep, bg - h * eb)
        fw = float((wf * (Fp - F0)).sum() + (wp * (Pp - P0)).sum()) / h
        bw = float((wf * (F0 - Fm)).sum() + (wp * (P0 - Pm)).sum()) / h
        assert min(abs(fw - an), abs(bw - an)) <= 1e-5 * abs(an), (h, fw, bw, an)
