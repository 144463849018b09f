"""Reverse mode of a run of Eq. (5) steps (``VlasovRun``: checkpoints every K steps,
segments re-recorded out of place, recorded step adjoints in reverse) on the GPU.

Pins: (1) against the oracle's chain of step adjoints (FP64 storage, gradients to
1e-10 of their largest entry, dL/dphi returned in FP32 to 1e-6); (2) against
differences of the GPU forward itself, for f0 and for phi.  The loss is piecewise
linear in f0 with very many switching surfaces (about half of all faces are limited),
so a perturbation of 1e-6 relative already crosses enough of them to move a central
difference by 0.5 %; the differences are one-sided with h = 1e-8, and at least one side
(one that stays on one linear piece) must match.  phi, which the library takes in FP32,
is moved by one unit in the last place of each value, and the derivative is taken along
the exact FP32 difference.
"""
import numpy as np
import pytest

import oracle as O
from paper_2110_15867_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

V = 5.0


def _setup(n, nu, dtype, seed=1):
    Fu = I.fermi_dirac(nu, V)
    delta = I.gaussian_field(n, 0.05, seed=seed)
    f0 = I.initial_f(delta, Fu, dtype)
    phi = I.fourier_potential(n, seed=seed + 10).astype(np.float32)
    return f0, phi


def _dt(g, phi, cfl, a=1.0):
    m = max([O.max_abs_nu(g, ax, 0.5, a, phi.astype(np.float64)) for ax in (3, 4, 5)] +
            [O.max_abs_nu(g, ax, 1.0, a, phi.astype(np.float64)) for ax in (0, 1, 2)])
    return cfl / m


def _mods():
    from paper_2110_15867_gb300 import autograd as A
    from paper_2110_15867_gb300 import binding as B
    B.load()
    return A, B


@pytest.mark.parametrize("n_steps,K", [(5, 2), (3, 4)])
def test_run_gradient_matches_oracle_chain(n_steps, K):
    A, _ = _mods()
    n, nu = (8, 8, 8), (8, 8, 8)
    f0, phi = _setup(n, nu, np.float64)
    g = O.grid(n, nu, V=V)
    dt, a = _dt(g, phi, 0.7), 1.0
    w = np.random.default_rng(5).standard_normal(n)
    # oracle: the states, L = sum_x w(x) rho(x), then the step adjoints last to first
    states = [f0.copy()]
    for _ in range(n_steps):
        f = states[-1].copy()
        O.step(g, f, dt, a, a, phi.astype(np.float64))
        states.append(f)
    rho_ref, _ = O.moment(g, states[-1])
    du3 = (2 * V / nu[0]) * (2 * V / nu[1]) * (2 * V / nu[2])
    lam = np.broadcast_to((du3 * w)[..., None, None, None], f0.shape).copy()
    dphi_ref = np.zeros(n)
    for k in reversed(range(n_steps)):
        dphi_ref += O.step_adjoint(g, states[k], lam, dt, a, phi.astype(np.float64))

    run = A.Run(f0.shape, torch.float64, L=1.0, V=V)
    ft = torch.from_numpy(f0).cuda().requires_grad_()
    pt = torch.from_numpy(phi).cuda().requires_grad_()
    rho = A.run_rho(ft, pt, run, dt, a, n_steps, K)
    run.v.status()
    rho_h = rho.detach().cpu().numpy()
    assert np.abs(rho_h - rho_ref).max() <= 1e-12 * np.abs(rho_ref).max()
    (rho * torch.from_numpy(w).cuda()).sum().backward()
    run.v.status()
    gf = ft.grad.cpu().numpy()
    gp = pt.grad.cpu().numpy().astype(np.float64)
    ef = np.abs(gf - lam).max() / np.abs(lam).max()
    ep = np.abs(gp - dphi_ref).max() / np.abs(dphi_ref).max()
    print("dL/df0 rel Linf %.2e  dL/dphi rel Linf %.2e" % (ef, ep))
    assert ef <= 1e-10 and ep <= 1e-6
    run.close()


def test_run_gradient_matches_differences():
    A, _ = _mods()
    n, nu = (8, 8, 8), (8, 8, 8)
    f0, phi = _setup(n, nu, np.float64, seed=3)
    g = O.grid(n, nu, V=V)
    dt, a, n_steps, K = _dt(g, phi, 0.7), 1.0, 4, 2
    rng = np.random.default_rng(7)
    w = torch.from_numpy(rng.standard_normal(n)).cuda()
    run = A.Run(f0.shape, torch.float64, L=1.0, V=V)

    def loss(f, p):
        with torch.no_grad():
            return float((A.run_rho(torch.from_numpy(f).cuda(), torch.from_numpy(p).cuda(), run, dt, a,
                                    n_steps, K) * w).sum())

    ft = torch.from_numpy(f0).cuda().requires_grad_()
    pt = torch.from_numpy(phi).cuda().requires_grad_()
    (A.run_rho(ft, pt, run, dt, a, n_steps, K) * w).sum().backward()
    gf = ft.grad.cpu().numpy()
    gp = pt.grad.cpu().numpy().astype(np.float64)

    # f0 along a smooth relative perturbation
    e = f0 * rng.standard_normal(n)[..., None, None, None]
    h = 1e-8
    L0 = loss(f0, phi)
    an = float((gf * e).sum())
    fw = (loss(f0 + h * e, phi) - L0) / h
    bw = (L0 - loss(f0 - h * e, phi)) / h
    print("f0: one-sided differences %.10e %.10e  adjoint %.10e" % (fw, bw, an))
    assert min(abs(fw - an), abs(bw - an)) <= 2e-5 * abs(an)

    # phi: every value moved by one unit in the last place (FP32), up and down
    d = np.sign(rng.standard_normal(n))
    pp = (phi.astype(np.float64) * (1 + 2.0 ** -23 * d)).astype(np.float32)
    pm = (phi.astype(np.float64) * (1 - 2.0 ** -23 * d)).astype(np.float32)
    fw = loss(f0, pp) - L0
    bw = L0 - loss(f0, pm)
    afw = float((gp * (pp.astype(np.float64) - phi)).sum())
    abw = float((gp * (phi - pm.astype(np.float64))).sum())
    print("phi: one-sided differences %.10e %.10e  adjoint %.10e %.10e" % (fw, bw, afw, abw))
    assert min(abs(fw - afw) / abs(afw), abs(bw - abw) / abs(abw)) <= 1e-4
    run.close()


def test_run_fp32_gradient_close_to_fp64():
    # FP32 against FP64 storage, pinned to the conditioning of the gradient: at most 3x
    # the spread of the FP64 gradients when f0 is perturbed by 4 FP32 roundings.
    A, _ = _mods()
    n, nu = (16, 16, 16), (16, 16, 16)
    f0, phi = _setup(n, nu, np.float64, seed=2)
    g = O.grid(n, nu, V=V)
    dt, a, n_steps, K = _dt(g, phi, 0.7), 1.0, 8, 4
    w = torch.from_numpy(np.random.default_rng(9).standard_normal(n)).cuda()
    fpert = f0 * (1 + 4 * 2.0 ** -24 * np.random.default_rng(11).uniform(-1, 1, f0.shape))

    def grads(f, dtype):
        run = A.Run(f.shape, dtype, L=1.0, V=V)
        ft = torch.from_numpy(f).to(dtype).cuda().requires_grad_()
        pt = torch.from_numpy(phi).cuda().requires_grad_()
        (A.run_rho(ft, pt, run, dt, a, n_steps, K) * w).sum().backward()
        run.v.status()
        out = (ft.grad.double().cpu().numpy(), pt.grad.double().cpu().numpy())
        run.close()
        return out

    g64, g64p, g32 = grads(f0, torch.float64), grads(fpert, torch.float64), grads(f0, torch.float32)
    for k, name in ((0, "dL/df0"), (1, "dL/dphi")):
        y = g64[k]
        sens = np.linalg.norm(g64p[k] - y) / np.linalg.norm(y)
        rel = np.linalg.norm(g32[k] - y) / np.linalg.norm(y)
        print("%s FP32 vs FP64 rel L2 %.2e (FP64 spread %.2e)" % (name, rel, sens))
        assert np.isfinite(g32[k]).all() and rel <= 3 * sens + 1e-6


@pytest.mark.parametrize("tape_segments", [2, 3, "auto"])
def test_more_taped_segments_give_the_same_gradients(tape_segments):
    # the forward records the last tape_segments segments directly ("auto": as many as half the
    # free memory holds, here all 4); the backward runs the others again: the same sweeps on
    # the same inputs, so lambda is bit for bit and
    # dL/dphi (per-cell sums by FP64 atomics at this velocity size) agrees to rounding
    A, _ = _mods()
    n, nu = (8, 8, 8), (8, 8, 8)
    f0, phi = _setup(n, nu, np.float64, seed=4)
    g = O.grid(n, nu, V=V)
    dt, a, n_steps, K = _dt(g, phi, 0.7), 1.0, 7, 2
    w = torch.from_numpy(np.random.default_rng(12).standard_normal(n)).cuda()
    out = {}
    for ts in (1, tape_segments):
        run = A.Run(f0.shape, torch.float64, L=1.0, V=V, tape_segments=ts)
        ft = torch.from_numpy(f0).cuda().requires_grad_()
        pt = torch.from_numpy(phi).cuda().requires_grad_()
        rho = A.run_rho(ft, pt, run, dt, a, n_steps, K)
        (rho * w).sum().backward()
        run.v.status()
        out[ts] = (rho.detach().cpu().numpy(), ft.grad.cpu().numpy(), pt.grad.double().cpu().numpy())
        run.close()
    assert np.array_equal(out[1][0], out[tape_segments][0])
    assert np.array_equal(out[1][1], out[tape_segments][1])
    assert np.abs(out[1][2] - out[tape_segments][2]).max() <= 1e-6 * np.abs(out[1][2]).max()
