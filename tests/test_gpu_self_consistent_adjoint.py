"""Self-consistent reverse mode (state f, phi; phi^{n+1} from the post-drift moment
through the Poisson solve) on the GPU against the oracle's self-consistent step adjoint
(pinned in tests/test_oracle_adjoint.py).  The GPU keeps phi in FP32, so the oracle runs
with phi^{n+1} rounded to FP32 (its PHI32 flag): FP64 storage then agrees to rounding."""
import numpy as np
import pytest

import oracle as O
from paper_2110_15867_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
V = 5.0
FLAGS = O.MPP | O.PHI32


def _mods():
    from paper_2110_15867_gb300 import autograd as A
    from paper_2110_15867_gb300 import binding as B
    B.load()
    return A, B


def _setup(n, nu, dtype):
    g = O.grid(n, nu, V=V)
    f0 = I.initial_f(I.gaussian_field(n, 0.05, seed=2), I.fermi_dirac(nu, V), dtype)
    bg = 3.0 * (1.0 + I.gaussian_field(n, 0.5, seed=4))
    rho0, _ = O.moment(g, f0.astype(np.float64))
    phi0 = O.poisson(g, rho0 + bg, 0.5, 1.0).astype(np.float32)
    return g, f0, bg, phi0


def _rel(x, y):
    return np.abs(np.asarray(x, np.float64) - y).max() / np.abs(y).max()


def test_step_adjoint_sc_matches_oracle_fp64():
    A, B = _mods()
    n, nu = (6, 6, 6), (8, 8, 8)
    g, f0, bg, phi0 = _setup(n, nu, np.float64)
    dt, ah, af = 0.004, 0.52, 0.55
    rng = np.random.default_rng(3)
    lam0 = rng.standard_normal(f0.shape)
    wphi = rng.standard_normal(n)
    lam_ref = lam0.copy()
    dphi_ref, dbg_ref = O.step_adjoint_sc(g, f0, lam_ref, dt, ah, af, phi0.astype(np.float64), bg, 1.0,
                                          lam_phi_next=wphi, flags=FLAGS)
    dev = "cuda"
    f = torch.from_numpy(f0).to(dev)
    v = B.Vlasov(torch.empty_like(f), V=V)
    rec = [torch.empty_like(f) for _ in range(8)]
    phi_t = torch.from_numpy(phi0).to(dev)
    phi1 = torch.empty_like(phi_t)
    bg_t = torch.from_numpy(bg).to(dev)
    v.step_record_sc(f, rec, dt, ah, af, phi_t, phi1, rho_bg=bg_t)
    # phi^{n+1} as the oracle computes it (FP32-rounded)
    rho5, _ = O.moment(g, rec[5].cpu().numpy())
    phi1_ref = O.poisson(g, rho5 + bg, af, 1.0).astype(np.float32)
    assert np.allclose(phi1.cpu().numpy(), phi1_ref, rtol=1.2e-7, atol=0)  # within one FP32 rounding
    lam = torch.from_numpy(lam0).to(dev)
    dphi = torch.zeros(n, dtype=torch.float64, device=dev)
    dbg = torch.zeros(n, dtype=torch.float64, device=dev)
    v.step_adjoint_recorded_sc(f, rec, lam, dt, ah, af, phi_t, phi1, 1.0,
                               lam_phi_next=torch.from_numpy(wphi).to(dev), dLdphi_n=dphi, dLdrho_bg=dbg)
    v.status()
    e = (_rel(lam.cpu().numpy(), lam_ref), _rel(dphi.cpu().numpy(), dphi_ref), _rel(dbg.cpu().numpy(), dbg_ref))
    print("lambda %.2e  dL/dphi_n %.2e  dL/drho_bg %.2e" % e)
    assert max(e) <= 1e-10
    v.close()


@pytest.mark.parametrize("tape_segments", [1, "auto"])
def test_run_sc_gradient_matches_oracle_chain(tape_segments):
    A, B = _mods()
    n, nu = (6, 6, 6), (8, 8, 8)
    g, f0, bg, phi0 = _setup(n, nu, np.float64)
    dt, n_steps, K = 0.004, 5, 2
    ah = [0.50 + 0.01 * k for k in range(n_steps)]
    af = [0.505 + 0.01 * k for k in range(n_steps)]
    w = np.random.default_rng(6).standard_normal(n)
    # oracle: states (f_k, phi_k), L = sum w rho(f_N), then the step adjoints last to first
    fs, phis = [f0.copy()], [phi0.astype(np.float64)]
    for k in range(n_steps):
        f = fs[-1].copy()
        p1, _ = O.step(g, f, dt, ah[k], af[k], phis[-1], rho_bg=bg, self_consistent=True, flags=FLAGS)
        fs.append(f)
        phis.append(p1)
    rho_ref, _ = O.moment(g, fs[-1])
    du3 = (2 * V / nu[0]) ** 3
    lam = np.broadcast_to((du3 * w)[..., None, None, None], f0.shape).copy()
    lam_phi, dbg_ref = None, np.zeros(n)
    for k in reversed(range(n_steps)):
        dphi, dbg = O.step_adjoint_sc(g, fs[k], lam, dt, ah[k], af[k], phis[k], bg, 1.0, lam_phi_next=lam_phi,
                                      flags=FLAGS)
        lam_phi = dphi
        dbg_ref += dbg

    # one taped segment (the backward runs the others again) or all of them (nothing again)
    run = A.Run(f0.shape, torch.float64, L=1.0, V=V, tape_segments=tape_segments)
    ft = torch.from_numpy(f0).cuda().requires_grad_()
    pt = torch.from_numpy(phi0).cuda().requires_grad_()
    bt = torch.from_numpy(bg).cuda().requires_grad_()
    rho = A.run_rho_sc(ft, pt, bt, run, dt, ah, af, n_steps, K)
    assert _rel(rho.detach().cpu().numpy(), rho_ref) <= 1e-12
    (rho * torch.from_numpy(w).cuda()).sum().backward()
    run.v.status()
    e = (_rel(ft.grad.cpu().numpy(), lam), _rel(pt.grad.cpu().numpy(), lam_phi), _rel(bt.grad.cpu().numpy(), dbg_ref))
    print("dL/df0 %.2e  dL/dphi0 %.2e (FP32)  dL/drho_bg %.2e" % e)
    assert e[0] <= 1e-10 and e[1] <= 1e-6 and e[2] <= 1e-10
    run.close()
