"""The fused kick tail (D_uy and D_uz in one pass of the u_z line kernel) against the
separate sweeps: the same arithmetic, so whole steps must agree bit for bit, with both
orientations of the Courant number present (the potential's gradient changes sign across
the box), for n_u = 16 and 32.  The oracle comparison of the step itself is
tests/test_gpu_parity.py::test_step_fixed_potential_fp32, which runs the fused path."""
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


@pytest.mark.parametrize("n,nu", [((8, 8, 8), (16, 16, 16)), ((4, 6, 4), (32, 32, 32)), ((6, 4, 4), (8, 32, 32))])
def test_fused_kick_is_bitwise_the_separate_sweeps(n, nu):
    B = _lib()
    V = 5.0
    f0 = I.initial_f(I.gaussian_field(n, 0.05, seed=4), I.fermi_dirac(nu, V), np.float32)
    phi_np = I.fourier_potential(n, seed=14).astype(np.float32)
    g = O.grid(n, nu, V=V)
    m = max([O.max_abs_nu(g, ax, 0.5, 1.0, phi_np.astype(np.float64)) for ax in (3, 4, 5)] +
            [O.max_abs_nu(g, ax, 1.0, 1.0, phi_np.astype(np.float64)) for ax in (0, 1, 2)])
    dt = 0.8 / m
    phi = torch.from_numpy(phi_np).cuda()
    out = {}
    for fused in (True, False):
        f = torch.from_numpy(f0).cuda()
        v = B.Vlasov(f, V=V)
        v.set_fused_kick(fused)
        v.enable_timers(True)
        for _ in range(3):
            v.step(dt, 1.0, 1.0, phi)
        v.status()
        _, launches = v.read_timers()
        out[fused] = (f.cpu().numpy(), launches)
        v.close()
    assert np.array_equal(out[True][0], out[False][0])
    fused_launches = out[True][1]["sweep_uyuz"]
    print("fused kick-tail launches:", fused_launches)
    if nu[1] == nu[2]:
        assert fused_launches == 6 and out[True][1]["sweep_uy"] == 0 and out[True][1]["sweep_uz"] == 0
    else:
        assert fused_launches == 0
    assert out[False][1]["sweep_uyuz"] == 0


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
@pytest.mark.parametrize("nu", [16, 32])
def test_fused_kick_16bit_against_the_oracle(fmt, nu):
    # 16-bit storage: the fused pass keeps D_uy's result in FP32 and encodes only after
    # D_uz, so it is not the separate sweeps bit for bit (those encode twice); both are
    # held to the codec bound of the parity tests per encode against the FP64 oracle's
    # kick (D_ux, D_uy, D_uz) of the same decoded input: relative L1 <= k 2^-8 (BF16) or
    # k 2^-11 (FP16) + 1e-6 with k the number of encodes (fused 2, separate 3)
    B = _lib()
    V = 5.0
    bound = {"bf16": 2.0 ** -8, "f16": 2.0 ** -11}[fmt]
    tdt = {"bf16": torch.bfloat16, "f16": torch.float16}[fmt]
    n = (8, 8, 8) if nu == 16 else (4, 4, 4)
    f0 = I.initial_f(I.gaussian_field(n, 0.05, seed=6), I.fermi_dirac(nu, V), np.float64)
    phi_np = I.fourier_potential(n, seed=16).astype(np.float32)
    g = O.grid(n, nu, V=V)
    dt = 0.8 / max(O.max_abs_nu(g, ax, 1.0, 1.0, phi_np.astype(np.float64)) for ax in (3, 4, 5))
    phi = torch.from_numpy(phi_np).cuda()
    codes0, scale0 = B.encode_lines(torch.from_numpy(f0).cuda(), tdt)
    ref = B.decode_lines(codes0, scale0).cpu().numpy()
    for ax in (3, 4, 5):
        O.sweep(g, ref, ax, dt, 1.0, phi_np.astype(np.float64))
    err = {}
    for fused in (True, False):
        codes, scale = codes0.clone(), scale0.clone()
        v = B.Vlasov(codes, V=V, scale=scale)
        v.set_fused_kick(fused)
        v.enable_timers(True)
        v.kick(dt, phi)  # D_ux, then D_uy and D_uz (one pass when fused)
        v.status()
        _, launches = v.read_timers()
        out = B.decode_lines(codes, scale).cpu().numpy()
        err[fused] = np.abs(out - ref).sum() / np.abs(ref).sum()
        assert launches["sweep_uyuz"] == (1 if fused else 0)
        v.close()
    print("%s n_u %d kick rel L1: fused %.2e, separate %.2e" % (fmt, nu, err[True], err[False]))
    assert err[True] <= 2 * bound + 1e-6 and err[False] <= 3 * bound + 1e-6
