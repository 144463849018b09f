"""The moment rho_nu (Sec. 4.1.3) summed by the step's x sweep (vlasov_set_fused_moment)
against the separate moment kernel on the same post-drift state.

With an external potential both kicks use phi, so f is the same bit for bit whichever
kernel sums the moment.  rho: the fused path adds each block's 256 FP32 values of a row
pairwise (8 levels: error at most 8 units in the last place of their sum) and those
partials in FP64; the separate kernel's compensated sums are exact to about two units,
so the two agree to 10 units (6e-7) per cell for FP32 storage and to 1e-14 for FP64.
When the x sweep shifts whole cells (|nu| >= 1, small a) it is not streamed and the
separate kernel runs: rho is then the same bit for bit.  The self-consistent step with the fused
moment is pinned against the oracle in test_gpu_parity.
"""
import numpy as np
import pytest

import oracle as O
from paper_2110_15867_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

V = 5.0


def _lib():
    from paper_2110_15867_gb300 import binding as B
    B.load()
    return B


def _run(B, f0, phi, dt, a_half, fused, n):
    ft = torch.from_numpy(f0.copy()).cuda()
    v = B.Vlasov(ft, V=V)
    v.set_fused_moment(fused)
    rho = torch.empty(n, dtype=torch.float64, device="cuda")
    v.step(dt, a_half, 1.0, torch.from_numpy(phi).cuda(), rho_nu=rho)
    v.status()
    out = ft.cpu().numpy(), rho.cpu().numpy()
    v.close()
    return out


@pytest.mark.parametrize("dtype,tol", [(np.float32, 10 * 2.0 ** -24), (np.float64, 1e-14)])
@pytest.mark.parametrize("n,nu", [((16, 8, 8), (16, 16, 16)), ((8, 4, 4), (8, 8, 8))])
def test_fused_moment_matches_separate_kernel(dtype, tol, n, nu):
    B = _lib()
    f0 = I.initial_f(I.gaussian_field(n, 0.05, seed=2), I.fermi_dirac(nu, V), dtype)
    phi = I.fourier_potential(n, seed=12).astype(np.float32)
    g = O.grid(n, nu, V=V)
    dt = min(0.7 / O.max_abs_nu(g, ax, 1.0, 1.0, phi.astype(np.float64)) * (2 if ax >= 3 else 1)
             for ax in range(6))
    f_on, rho_on = _run(B, f0, phi, dt, 1.0, True, n)
    f_off, rho_off = _run(B, f0, phi, dt, 1.0, False, n)
    assert np.array_equal(f_on, f_off)
    rel = np.abs(rho_on - rho_off).max() / np.abs(rho_off).min()
    print("fused vs separate moment: max relative difference %.2e" % rel)
    assert rel <= tol
    # reproducible run to run
    _, rho_again = _run(B, f0, phi, dt, 1.0, True, n)
    assert np.array_equal(rho_on, rho_again)


def test_whole_cell_x_shift_uses_the_separate_kernel():
    # a = 0.3 multiplies the position Courant numbers by 11: the x sweep shifts whole
    # cells, is not streamed, and the separate moment kernel sums rho
    B = _lib()
    n, nu = (16, 8, 8), (16, 16, 16)
    f0 = I.initial_f(I.gaussian_field(n, 0.05, seed=3), I.fermi_dirac(nu, V), np.float32)
    phi = I.fourier_potential(n, seed=13).astype(np.float32)
    g = O.grid(n, nu, V=V)
    dt = min(0.7 / O.max_abs_nu(g, ax, 1.0, 1.0, phi.astype(np.float64)) * 2 for ax in (3, 4, 5))
    assert max(O.max_abs_nu(g, ax, 1.0, 0.3, phi.astype(np.float64)) * dt for ax in (0, 1, 2)) > 1.0
    f_on, rho_on = _run(B, f0, phi, dt, 0.3, True, n)
    f_off, rho_off = _run(B, f0, phi, dt, 0.3, False, n)
    assert np.array_equal(f_on, f_off) and np.array_equal(rho_on, rho_off)
