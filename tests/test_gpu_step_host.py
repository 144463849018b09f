"""vlasov_step_host (one Eq. (5) step of a host buffer, its x-slabs copied in and out on a
second stream behind the cell-local sweeps) against upload + vlasov_step + download: the
same kernels on the same tiles, so the same f, rho and phi^{n+1} bit for bit, for a
self-consistent step (Poisson between the kicks) with the one-pass kick, the fused kick
tail (on u_z line tiles, or on staged planes for 48^3 velocity cubes) and the separate
sweeps, the fused moment on and off, on 16 and on 8 slabs of one x-plane, and for a step
that falls back to the three calls in sequence (a whole-cell shift in D_y / D_z)."""
import numpy as np
import pytest

import oracle as O
from paper_2110_15867_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lib():
    from paper_2110_15867_gb300 import binding as B
    B.load()
    return B


def _run(B, f0, phi0, bg, dt, a_half, host, fused):
    V = 5.0
    n = f0.shape[:3]
    f = torch.from_numpy(f0).cuda()
    v = B.Vlasov(f, V=V)
    v.set_fused_kick(int(fused))
    v.set_fused_moment(bool(fused))
    phi = torch.from_numpy(phi0).cuda()
    phi1 = torch.empty_like(phi)
    rho = torch.empty(n, dtype=torch.float64, device="cuda")
    fh = torch.from_numpy(f0.copy()).pin_memory()
    bgt = torch.from_numpy(bg).cuda()
    f.zero_()  # the step must read the host buffer, not the device array
    v.enable_timers(True)
    if host:
        v.step_host(fh, dt, a_half, 0.6, phi, rho_bg=bgt, phi_next=phi1, rho_nu=rho)
    else:
        v.upload(fh)
        v.step(dt, a_half, 0.6, phi, rho_bg=bgt, phi_next=phi1, rho_nu=rho)
        v.download(fh)
    v.status()
    _, launches = v.read_timers()
    out = (fh.numpy().copy(), rho.cpu().numpy(), phi1.cpu().numpy())
    v.close()
    return out, launches["sweep_ux"] + launches["kick"]


@pytest.mark.parametrize("n,nu,a_half", [((16, 8, 8), (16, 16, 16), 0.55), ((8, 4, 4), (32, 32, 32), 0.55),
                                         ((16, 8, 8), (16, 16, 16), 0.12), ((8, 4, 4), (48, 48, 48), 0.55)])
@pytest.mark.parametrize("fused", [2, 1, 0])
def test_step_host_is_upload_step_download(n, nu, a_half, fused):
    B = _lib()
    V = 5.0
    f0 = I.initial_f(I.gaussian_field(n, 0.05, seed=7), I.fermi_dirac(nu, V), np.float32)
    phi0 = I.fourier_potential(n, seed=17).astype(np.float32)
    bg = 3.0 * (1.0 + I.gaussian_field(n, 0.5, seed=8))
    g = O.grid(n, nu, V=V)
    p64 = phi0.astype(np.float64)
    # CFL 0.7 for the kicks (dt / 2 each) and the drift at a = 0.55; a_half = 0.12 then
    # makes D_x, D_y, D_z shift whole cells
    dt = min([1.4 / O.max_abs_nu(g, ax, 1.0, 1.0, p64) for ax in (3, 4, 5)] +
             [0.7 / O.max_abs_nu(g, ax, 1.0, 0.55, p64) for ax in (0, 1, 2)])
    ref, _ = _run(B, f0, phi0, bg, dt, a_half, False, fused)
    got, ux_launches = _run(B, f0, phi0, bg, dt, a_half, True, fused)
    for r, o in zip(ref, got):
        assert np.array_equal(r, o)
    # up to 16 slabs (one per x-plane here): each kick runs u_x (or the one-pass kick) once per
    # slab; the fallback once
    assert ux_launches == (2 if a_half < 0.5 else 2 * min(16, n[0]))


def test_step_host_fp64_falls_back_to_the_three_calls():
    # FP64 storage has no line kernel to split per slab: the same result as upload + step
    # + download, through the sequential path
    B = _lib()
    V = 5.0
    n, nu = (8, 8, 8), (8, 8, 8)
    f0 = I.initial_f(I.gaussian_field(n, 0.05, seed=9), I.fermi_dirac(nu, V), np.float64)
    phi0 = I.fourier_potential(n, seed=19).astype(np.float32)
    bg = 3.0 * (1.0 + I.gaussian_field(n, 0.5, seed=10))
    g = O.grid(n, nu, V=V)
    p64 = phi0.astype(np.float64)
    dt = min([1.4 / O.max_abs_nu(g, ax, 1.0, 1.0, p64) for ax in (3, 4, 5)] +
             [0.7 / O.max_abs_nu(g, ax, 1.0, 0.55, p64) for ax in (0, 1, 2)])
    ref, _ = _run(B, f0, phi0, bg, dt, 0.55, False, True)
    got, ux_launches = _run(B, f0, phi0, bg, dt, 0.55, True, True)
    for r, o in zip(ref, got):
        assert np.array_equal(r, o)
    assert ux_launches == 2


def _steps(B, f0, phi0, bg, dt, plan):
    """Run `plan` (a sequence of "host", "host2" (a second host buffer holding the same
    state), "moment" (a library call between steps) and "dev" (upload, vlasov_step,
    download)) on a fresh context; returns the host state, rho and phi after the last step."""
    V = 5.0
    n = f0.shape[:3]
    f = torch.zeros(f0.shape, dtype=torch.float32, device="cuda")
    v = B.Vlasov(f, V=V)
    phi = [torch.from_numpy(phi0).cuda(), torch.empty(n, dtype=torch.float32, device="cuda")]
    rho = torch.empty(n, dtype=torch.float64, device="cuda")
    bgt = torch.from_numpy(bg).cuda()
    fh = torch.from_numpy(f0.copy()).pin_memory()
    fh2 = torch.empty_like(fh).pin_memory()
    cur = fh
    for k, what in enumerate(plan):
        p_n, p_next = phi[k % 2], phi[(k + 1) % 2]
        if what == "host2":
            v.host_wait()
            torch.cuda.synchronize()
            other = fh2 if cur is fh else fh
            other.copy_(cur)
            cur = other
        if what in ("host", "host2"):
            v.step_host(cur, dt, 0.55, 0.6, p_n, rho_bg=bgt, phi_next=p_next, rho_nu=rho)
        elif what == "moment":
            v.step_host(cur, dt, 0.55, 0.6, p_n, rho_bg=bgt, phi_next=p_next, rho_nu=rho)
            v.moment(torch.empty(n, dtype=torch.float64, device="cuda"))
        else:
            v.upload(cur)
            v.step(dt, 0.55, 0.6, p_n, rho_bg=bgt, phi_next=p_next, rho_nu=rho)
            v.download(cur)
    v.host_wait()
    v.status()
    out = (cur.numpy().copy(), rho.cpu().numpy(), phi[len(plan) % 2].cpu().numpy())
    v.close()
    return out


@pytest.mark.parametrize("plan", [("host", "host", "host", "host"), ("host", "moment", "host", "host"),
                                  ("host", "host2", "host", "dev", "host")])
def test_consecutive_step_host_calls(plan):
    # Back-to-back vlasov_step_host calls start each slab's upload once the previous call's
    # download of that slab is done (the downloads run on a stream of their own); another
    # library call between two of them, a second host buffer, or device steps in between
    # must see the finished downloads.  Every plan equals the same number of device steps.
    B = _lib()
    V = 5.0
    n, nu = (16, 8, 8), (16, 16, 16)
    f0 = I.initial_f(I.gaussian_field(n, 0.05, seed=27), I.fermi_dirac(nu, V), np.float32)
    phi0 = I.fourier_potential(n, seed=37).astype(np.float32)
    bg = 3.0 * (1.0 + I.gaussian_field(n, 0.5, seed=28))
    g = O.grid(n, nu, V=V)
    p64 = phi0.astype(np.float64)
    dt = min([1.4 / O.max_abs_nu(g, ax, 1.0, 1.0, p64) for ax in (3, 4, 5)] +
             [0.7 / O.max_abs_nu(g, ax, 1.0, 0.55, p64) for ax in (0, 1, 2)])
    ref = _steps(B, f0, phi0, bg, dt, ("dev",) * len(plan))
    got = _steps(B, f0, phi0, bg, dt, plan)
    for r, o in zip(ref, got):
        assert np.array_equal(r, o)
