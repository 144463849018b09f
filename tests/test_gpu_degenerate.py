"""Degenerate inputs of the sweeps and the step, through the C ABI, that have exact answers.

- dt = 0: every Courant number is 0, the fractional flux s * fbar is 0 on every face, so
  each sweep (and a whole Eq. (5) step) must return f bit for bit, and the step's rho_nu
  must be the moment of f.
- f = 0: stays 0 with no error raised (the NaN / negative-sum check sees a zero sum).
- f uniform in position (f = F(u) in every cell): the curvatures are exactly 0, so the
  limiter bounds collapse to [c, c] and every face carries the same flux; position sweeps
  must leave f unchanged bit for bit, whatever the Courant number.
"""
import numpy as np
import pytest

import oracle as O
from paper_2110_15867_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

V = 5.0
SHAPES = [((8, 6, 5), (16, 16, 32)), ((4, 5, 4), (48, 24, 48)), ((6, 4, 5), (8, 20, 12))]


def _lib():
    from paper_2110_15867_gb300 import binding as B
    B.load()
    return B


def _f0(n, nu, dtype, rms=0.05):
    return I.initial_f(I.gaussian_field(n, rms, seed=7), I.fermi_dirac(nu, V), dtype)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("n,nu", SHAPES)
def test_zero_dt_sweeps_and_step_are_identity(dtype, n, nu):
    B = _lib()
    f0 = _f0(n, nu, dtype)
    phi = torch.from_numpy(I.fourier_potential(n, seed=17).astype(np.float32)).cuda()
    ft = torch.from_numpy(f0.copy()).cuda()
    v = B.Vlasov(ft, V=V)
    for axis in range(6):
        v.sweep(axis, 0.0, 1.0, phi)
        v.status()
        assert np.array_equal(ft.cpu().numpy(), f0), axis
    rho_step = torch.empty(n, dtype=torch.float64, device="cuda")
    v.step(0.0, 1.0, 1.0, phi, rho_nu=rho_step)
    v.status()
    assert np.array_equal(ft.cpu().numpy(), f0)
    rho_ref, _ = O.moment(O.grid(n, nu, V=V), f0.astype(np.float64))
    tol = 1e-14 if dtype == np.float64 else 10 * 2.0 ** -24
    assert np.abs(rho_step.cpu().numpy() - rho_ref).max() <= tol * np.abs(rho_ref).max()
    v.close()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_zero_f_stays_zero(dtype):
    B = _lib()
    n, nu = (8, 6, 5), (16, 16, 32)
    phi_np = I.fourier_potential(n, seed=18).astype(np.float32)
    g = O.grid(n, nu, V=V)
    dt = 0.7 / max(O.max_abs_nu(g, ax, 1.0, 1.0, phi_np.astype(np.float64)) for ax in range(6))
    ft = torch.zeros(n + nu, dtype=torch.from_numpy(np.zeros(1, dtype)).dtype, device="cuda")
    v = B.Vlasov(ft, V=V)
    rho = torch.empty(n, dtype=torch.float64, device="cuda")
    v.step(dt, 1.0, 1.0, torch.from_numpy(phi_np).cuda(), rho_nu=rho)
    v.status()
    assert int(torch.count_nonzero(ft).item()) == 0 and int(torch.count_nonzero(rho).item()) == 0
    v.close()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("n,nu", SHAPES)
def test_uniform_in_position_is_a_fixed_point(dtype, n, nu):
    B = _lib()
    f0 = I.initial_f(np.zeros(n), I.fermi_dirac(nu, V), dtype)
    g = O.grid(n, nu, V=V)
    ft = torch.from_numpy(f0.copy()).cuda()
    v = B.Vlasov(ft, V=V)
    for axis in (0, 1, 2):
        for cfl in (0.3, 0.97):
            dt = cfl / O.max_abs_nu(g, axis, 1.0, 1.0, None)
            v.sweep(axis, dt, 1.0)
            v.status()
            assert np.array_equal(ft.cpu().numpy(), f0), (axis, cfl)
    v.close()
