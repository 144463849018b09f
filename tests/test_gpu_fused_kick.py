"""The fused kicks against the separate sweeps.  Mode 2 runs the whole kick D_uz D_uy D_ux
in one pass over each velocity cube (n_ux = n_uy = n_uz = 16 or 32), mode 1 runs D_ux and
then D_uy D_uz in one pass (of the u_z line kernel for n_uz = 16, 32; over staged (cell,
j_x) planes for n_uy = n_uz = 48), mode 0 three separate sweeps.  The
arithmetic of every line is the same, so whole FP32 steps must agree bit for bit, with both
orientations of the Courant number present (the potential's gradient changes sign across
the box), for n_u = 16 and 32 and a velocity grid the one-pass kick does not take.  16-bit
storage: the one-pass kick keeps the rounding points and random streams of mode 1, so the
two agree bit for bit (codes and scales), and both are held to the codec bound against
the oracle (for n_u = 48, where mode 2 falls back to mode 1, the staged-plane tail).  The oracle comparison of the FP32 step itself is
tests/test_gpu_parity.py::test_step_fixed_potential_fp32, which runs the default mode."""
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


@pytest.mark.parametrize("n,nu", [((8, 8, 8), (16, 16, 16)), ((4, 6, 4), (32, 32, 32)), ((6, 4, 4), (8, 32, 32)),
                                  ((5, 4, 7), (32, 32, 32)), ((4, 5, 4), (48, 48, 48)), ((4, 4, 4), (8, 48, 48))])
def test_fused_kicks_are_bitwise_the_separate_sweeps(n, nu):
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
    for mode in (2, 1, 0):
        f = torch.from_numpy(f0).cuda()
        v = B.Vlasov(f, V=V)
        v.set_fused_kick(mode)
        v.enable_timers(True)
        for _ in range(3):
            v.step(dt, 1.0, 1.0, phi)
        v.status()
        _, launches = v.read_timers()
        out[mode] = (f.cpu().numpy(), launches)
        v.close()
    assert np.array_equal(out[2][0], out[0][0])
    assert np.array_equal(out[1][0], out[0][0])
    cube = nu[0] == nu[1] == nu[2] and nu[2] in (16, 32)  # the one-pass kick
    tail = nu[1] == nu[2]  # the fused tail: u_z lines of a TMA tile (16, 32) or staged planes (48)
    print("one-pass kick launches:", out[2][1]["kick"], "fused tail launches:", out[1][1]["sweep_uyuz"])
    assert out[2][1]["kick"] == (6 if cube else 0)
    if cube:
        assert out[2][1]["sweep_ux"] == 0 and out[2][1]["sweep_uyuz"] == 0
    assert out[1][1]["kick"] == 0 and out[1][1]["sweep_uyuz"] == (6 if tail else 0)
    if tail:
        assert out[1][1]["sweep_uy"] == 0 and out[1][1]["sweep_uz"] == 0
    assert out[0][1]["sweep_uyuz"] == 0 and out[0][1]["kick"] == 0


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
@pytest.mark.parametrize("nu", [16, 32, 48])
def test_fused_kicks_16bit(fmt, nu):
    # 16-bit storage: the fused tail (mode 1) keeps D_uy's result in FP32 and encodes only
    # after D_uz, so it is not the separate sweeps (mode 0, which encode three times) bit
    # for bit; the one-pass kick (mode 2) encodes at the same points with the same random
    # streams as mode 1 and must equal it bit for bit.  All are held to the codec bound of
    # the parity tests per encode against the FP64 oracle's kick (D_ux, D_uy, D_uz) of the
    # same decoded input: relative L1 <= k 2^-8 (BF16) or k 2^-11 (FP16) + 1e-6 with k the
    # number of encodes (modes 2 and 1: 2, mode 0: 3)
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
    for _ in range(2):
        for ax in (3, 4, 5):
            O.sweep(g, ref, ax, dt / 2, 1.0, phi_np.astype(np.float64))
    err, res = {}, {}
    for mode in (2, 1, 0):
        codes, scale = codes0.clone(), scale0.clone()
        v = B.Vlasov(codes, V=V, scale=scale)
        v.set_fused_kick(mode)
        v.enable_timers(True)
        for _ in range(2):
            v.kick(dt / 2, phi)  # twice, so that the second kick reads what the first encoded
        v.status()
        _, launches = v.read_timers()
        res[mode] = (codes.view(torch.int16).cpu().numpy(), scale.cpu().numpy())
        if mode == 2 and nu in (16, 32):
            assert launches["kick"] == 2 and launches["sweep_ux"] == 0 and launches["sweep_uyuz"] == 0
        else:  # n_u = 48: mode 2 is mode 1
            assert launches["kick"] == 0 and launches["sweep_uyuz"] == (2 if mode >= 1 else 0)
        out = B.decode_lines(codes, scale).cpu().numpy()
        err[mode] = np.abs(out - ref).sum() / np.abs(ref).sum()
        v.close()
    print("%s n_u %d two half kicks, rel L1: one pass %.2e, fused tail %.2e, separate %.2e" %
          (fmt, nu, err[2], err[1], err[0]))
    assert np.array_equal(res[2][0], res[1][0]) and np.array_equal(res[2][1], res[1][1])
    assert err[2] <= 4 * bound + 1e-6 and err[1] <= 4 * bound + 1e-6 and err[0] <= 6 * bound + 1e-6
