"""Pins of the oracle's velocity moments (Sec. 4.1.3: density, mean velocity, velocity
dispersion tensor) against closed forms: a single occupied velocity cell, a two-point
distribution, the symmetries of an isotropic distribution on the symmetric velocity grid,
and Galilean invariance under whole-cell shifts in velocity."""
import numpy as np

import oracle as O
from paper_2110_15867_gb300 import inputs as I

V = 5.0
PAIRS = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


def _u(nu, j, V=V):
    du = 2 * V / nu
    return -V + (j + 0.5) * du


def test_single_velocity_cell_has_its_centre_and_no_dispersion():
    n, nu = (2, 3, 2), (8, 12, 16)
    g = O.grid(n, nu, V=V)
    f = np.zeros(n + nu)
    j = (5, 2, 11)
    f[1, 2, 0][j] = 2.5
    rho, um, s2 = O.moments(g, f)
    du3 = np.prod([2 * V / m for m in nu])
    assert rho[1, 2, 0] == du3 * 2.5 and np.count_nonzero(rho) == 1
    for i in range(3):
        assert um[i, 1, 2, 0] == _u(nu[i], j[i])
    assert np.abs(s2[:, 1, 2, 0]).max() <= 1e-13 * V * V
    # empty cells: everything 0
    assert np.all(um[:, 0, 0, 0] == 0) and np.all(s2[:, 0, 0, 0] == 0)


def test_two_point_distribution():
    # a at u_A, b at u_B: mean (a u_A + b u_B)/(a + b), dispersion a b/(a + b)^2 (u_A - u_B)(u_A - u_B)^T
    n, nu = (1, 1, 1), (8, 8, 12)
    g = O.grid(n, nu, V=V)
    f = np.zeros(n + nu)
    jA, jB, a, b = (1, 6, 3), (5, 2, 10), 0.7, 1.9
    f[0, 0, 0][jA] = a
    f[0, 0, 0][jB] = b
    _, um, s2 = O.moments(g, f)
    uA = np.array([_u(nu[i], jA[i]) for i in range(3)])
    uB = np.array([_u(nu[i], jB[i]) for i in range(3)])
    mean = (a * uA + b * uB) / (a + b)
    d = uA - uB
    assert np.allclose(um[:, 0, 0, 0], mean, rtol=0, atol=1e-14 * V)
    for k, (p, q) in enumerate(PAIRS):
        assert abs(s2[k, 0, 0, 0] - a * b / (a + b) ** 2 * d[p] * d[q]) <= 1e-13 * V * V


def test_isotropic_distribution_symmetries():
    n, nu = (3, 2, 2), (16, 16, 16)
    g = O.grid(n, nu, V=V)
    F = I.fermi_dirac(nu, V)
    f = np.broadcast_to(F, n + nu).copy() * (1 + np.arange(np.prod(n)).reshape(n))[..., None, None, None]
    rho, um, s2 = O.moments(g, f)
    # mirror symmetry of the velocity grid: no mean velocity, no off-diagonal dispersion
    assert np.abs(um).max() <= 1e-13 * V
    assert np.abs(s2[3:]).max() <= 1e-13 * V * V
    # rotation by axis permutation: equal diagonal entries, independent of the cell's amplitude
    assert np.allclose(s2[0], s2[1], rtol=1e-13) and np.allclose(s2[0], s2[2], rtol=1e-13)
    assert np.allclose(s2[0], s2[0, 0, 0, 0], rtol=1e-13)
    # rho agrees with the density routine
    rho1, _ = O.moment(g, f)
    assert np.allclose(rho, rho1, rtol=1e-14, atol=0)


def test_galilean_shift_in_velocity():
    # a compact blob shifted by k whole cells along u_y: mean moves by k du, dispersion unchanged
    n, nu = (2, 2, 1), (12, 16, 12)
    g = O.grid(n, nu, V=V)
    rng = np.random.default_rng(3)
    f = np.zeros(n + nu)
    f[..., 3:8, 4:9, 2:9] = rng.random(n + (5, 5, 7))
    k = 5
    f2 = np.roll(f, k, axis=4)
    _, um, s2 = O.moments(g, f)
    _, um2, s22 = O.moments(g, f2)
    du = 2 * V / nu[1]
    assert np.allclose(um2[1], um[1] + k * du, rtol=0, atol=1e-13 * V)
    assert np.allclose(um2[[0, 2]], um[[0, 2]], rtol=0, atol=1e-13 * V)
    assert np.allclose(s22, s2, rtol=0, atol=1e-12 * V * V)
