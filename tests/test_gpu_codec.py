"""BF16 / FP16 storage of f with one FP32 scale per u_z line (FP32 arithmetic).

Per sweep the GPU result, decoded, is compared with the FP64 oracle run on the same
decoded input.  Each stored value is re-encoded once per sweep with stochastic rounding
relative to its line's scale: the error of an element is below one unit in the last
place of its code, and a code stays below 2 between two refreshes of the line scale, so
the error is below 2^-7 (BF16, 8 significant bits) or 2^-10 (FP16) of the line scale
(taken as 1.5 max f); its mean is at most half that.  Hence per sweep: relative L1 <=
2^-8 / 2^-11 and L_inf <= 1.5 x 2^-7 / 2^-10 of max f, plus 1e-6 for the FP32
arithmetic.  Over 20 steps of the 24^3 x 16^3 workload the density must stay within 1e-3
relative L1 of the FP64 oracle.
"""
import numpy as np
import pytest

import oracle as O
from paper_2110_15867_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOUND = {"bf16": 2.0 ** -8, "f16": 2.0 ** -11}
TDT = {"bf16": torch.bfloat16, "f16": torch.float16}


def _setup(n, nu, V=5.0, seed=1, rms=0.01):
    f0 = I.initial_f(I.gaussian_field(n, rms, seed=seed), I.fermi_dirac(nu, V), np.float64)
    phi = I.fourier_potential(n, seed=seed + 10).astype(np.float32)
    return f0, phi


# u_z lines of 16/32 cells (TMA tiles of 256 lines), and of 48/24/40 cells (rows staged
# per warp; the streamed sweeps' 256-column blocks then cut u_z lines, and the u_y
# blocks hold 5, 10 or 6 whole lines)
CODEC_SHAPES = [((8, 6, 5), (16, 16, 32)), ((6, 5, 4), (24, 16, 48)), ((5, 4, 6), (48, 24, 24)),
                ((4, 5, 4), (16, 8, 40))]


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
@pytest.mark.parametrize("axis", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("n,nu", CODEC_SHAPES)
def test_codec_single_sweep(fmt, axis, n, nu):
    from paper_2110_15867_gb300 import binding as B
    B.load()
    f0, phi = _setup(n, nu)
    codes, scale = B.encode_lines(torch.from_numpy(f0).cuda(), TDT[fmt])
    ref = B.decode_lines(codes, scale).cpu().numpy()
    g = O.grid(n, nu, V=5.0)
    dt = 0.7 / O.max_abs_nu(g, axis, 1.0, 1.0, phi.astype(np.float64))
    O.sweep(g, ref, axis, dt, 1.0, phi.astype(np.float64))
    v = B.Vlasov(codes, V=5.0, scale=scale)
    v.sweep(axis, dt, 1.0, torch.from_numpy(phi).cuda())
    v.status()
    out = B.decode_lines(codes, scale).cpu().numpy()
    err = np.abs(out - ref)
    tol = BOUND[fmt] + 1e-6
    assert err.sum() <= tol * np.abs(ref).sum()
    assert err.max() <= 1.5 * (2 * BOUND[fmt] + 1e-6) * np.abs(ref).max()
    v.close()


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
@pytest.mark.parametrize("nu", [(16, 16, 16), (8, 12, 24), (16, 8, 40), (12, 8, 48)])
def test_codec_moment(fmt, nu):
    from paper_2110_15867_gb300 import binding as B
    B.load()
    n = (4, 4, 4)
    f0, _ = _setup(n, nu, rms=0.3)
    codes, scale = B.encode_lines(torch.from_numpy(f0).cuda(), TDT[fmt])
    dec = B.decode_lines(codes, scale).cpu().numpy()
    rho_ref, mass_ref = O.moment(O.grid(n, nu, V=5.0), dec)
    v = B.Vlasov(codes, V=5.0, scale=scale)
    rho, mass = v.moment(mass=True)
    assert np.allclose(rho.cpu().numpy(), rho_ref, rtol=1e-12, atol=0)
    assert mass == pytest.approx(mass_ref, rel=1e-12)
    v.close()


_REF = {}


def _oracle_20_steps():
    # the 24^3 x 16^3 sub-run of the reduced-precision workload: 20 Eq. (5) steps of the
    # 16^3-parity setup (delta rms 0.01, external phi, CFL 0.7, a = 1) in FP64
    if "rho" not in _REF:
        n, nu = 24, 16
        f0, phi = _setup(n, nu)
        g = O.grid(n, nu, V=5.0)
        dt = min(0.7 / O.max_abs_nu(g, ax, 1.0, 1.0, phi.astype(np.float64)) * (2 if ax >= 3 else 1)
                 for ax in range(6))
        f = f0.copy()
        for _ in range(20):
            _, rho = O.step(g, f, dt, 1.0, 1.0, phi.astype(np.float64))
        _REF.update(rho=rho, f0=f0, phi=phi, dt=dt)
    return _REF


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_codec_density_after_20_steps(fmt):
    from paper_2110_15867_gb300 import binding as B
    B.load()
    ref = _oracle_20_steps()
    codes, scale = B.encode_lines(torch.from_numpy(ref["f0"]).cuda(), TDT[fmt])
    v = B.Vlasov(codes, V=5.0, scale=scale)
    phi = torch.from_numpy(ref["phi"]).cuda()
    rho = torch.empty((24, 24, 24), dtype=torch.float64, device="cuda")
    for _ in range(20):
        v.step(ref["dt"], 1.0, 1.0, phi, rho_nu=rho)
    v.status()
    r = rho.cpu().numpy()
    l1 = np.abs(r - ref["rho"]).sum() / np.abs(ref["rho"]).sum()
    print("%s density rel L1 after 20 steps: %.3e" % (fmt, l1))
    assert l1 <= 1e-3
    v.close()


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_codec_steps_with_48_cell_rows(fmt):
    # five Eq. (5) steps with u_z lines of 48 cells (the staged-rows u_z sweep and the
    # streamed sweeps whose blocks cut u_z lines): density within 1e-3 relative L1 of
    # the FP64 oracle, the bound of the 20-step run above
    from paper_2110_15867_gb300 import binding as B
    B.load()
    n, nu = (8, 6, 6), (16, 24, 48)
    f0, phi = _setup(n, nu, seed=3)
    g = O.grid(n, nu, V=5.0)
    dt = min(0.7 / O.max_abs_nu(g, ax, 1.0, 1.0, phi.astype(np.float64)) * (2 if ax >= 3 else 1)
             for ax in range(6))
    f = f0.copy()
    for _ in range(5):
        _, rho_ref = O.step(g, f, dt, 1.0, 1.0, phi.astype(np.float64))
    codes, scale = B.encode_lines(torch.from_numpy(f0).cuda(), TDT[fmt])
    v = B.Vlasov(codes, V=5.0, scale=scale)
    phit = torch.from_numpy(phi).cuda()
    rho = torch.empty(n, dtype=torch.float64, device="cuda")
    for _ in range(5):
        v.step(dt, 1.0, 1.0, phit, rho_nu=rho)
    v.status()
    r = rho.cpu().numpy()
    l1 = np.abs(r - rho_ref).sum() / np.abs(rho_ref).sum()
    fl1 = np.abs(B.decode_lines(codes, scale).cpu().numpy() - f).sum() / np.abs(f).sum()
    print("%s n_uz 48: density rel L1 after 5 steps %.3e, f rel L1 %.3e" % (fmt, l1, fl1))
    assert l1 <= 1e-3
    v.close()
