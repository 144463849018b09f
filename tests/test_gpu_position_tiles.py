"""Position sweeps with whole lines staged per tile against the streamed sweep.

Both march every line of Eq. (3) with the same SL-MPP5 code (the streamed kernel walks
a negative Courant number with the mirrored stencil in memory order, the tile kernel
walks the line from its far end: the same operations), so single FP32 sweeps and whole
Eq. (5) steps must agree bit for bit, the moment the tile x sweep sums must equal the
streamed one's, and the launch counters must show which kernel ran.  Shapes: line
lengths 16, 24, 32, 48 and 64, n_uz = 32 (the z sweep's sign-grouped warps) and 16.
The u_x sweep of Eq. (4) with lines of 48 (zero-flux, the Courant number of each cell)
runs on the same tiles of [cell][u_x][u_y u_z]: bit for bit the streamed sweep in FP32,
within the codec bound of the oracle in BF16 / FP16.
"""
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


SHAPES = [((16, 16, 16), (16, 16, 16)), ((24, 16, 32), (8, 16, 32)), ((32, 4, 16), (16, 8, 32)),
          ((4, 48, 8), (8, 8, 16)), ((64, 8, 4), (8, 16, 32))]


@pytest.mark.parametrize("n,nu", SHAPES)
def test_tile_sweeps_are_bitwise_the_streamed_sweeps(n, nu):
    B = _lib()
    V = 5.0
    f0 = I.initial_f(I.gaussian_field(n, 0.05, seed=5), I.fermi_dirac(nu, V), np.float32)
    g = O.grid(n, nu, V=V)
    for ax in range(3):
        dt = 0.8 / O.max_abs_nu(g, ax, 1.0, 0.9)
        out = {}
        for tiles in (True, False):
            f = torch.from_numpy(f0).cuda()
            v = B.Vlasov(f, V=V)
            v.set_position_tiles(tiles)
            v.sweep(ax, dt, 0.9)
            v.sweep(ax, -0.6 * dt, 0.9)
            v.status()
            out[tiles] = f.cpu().numpy()
            v.close()
        assert np.array_equal(out[True], out[False]), ax


@pytest.mark.parametrize("n,nu", [((16, 16, 16), (16, 16, 16)), ((32, 4, 16), (16, 8, 32))])
def test_tile_step_and_fused_moment_are_bitwise_the_streamed_ones(n, nu):
    B = _lib()
    V = 5.0
    f0 = I.initial_f(I.gaussian_field(n, 0.05, seed=6), I.fermi_dirac(nu, V), np.float32)
    phi_np = I.fourier_potential(n, seed=16).astype(np.float32)
    g = O.grid(n, nu, V=V)
    p64 = phi_np.astype(np.float64)
    dt = min([1.4 / O.max_abs_nu(g, ax, 1.0, 1.0, p64) for ax in (3, 4, 5)] +
             [0.8 / O.max_abs_nu(g, ax, 1.0, 1.0, p64) for ax in (0, 1, 2)])
    phi = torch.from_numpy(phi_np).cuda()
    out = {}
    for tiles in (True, False):
        f = torch.from_numpy(f0).cuda()
        v = B.Vlasov(f, V=V)
        v.set_position_tiles(tiles)
        rho = torch.empty(n, dtype=torch.float64, device="cuda")
        v.enable_timers(True)
        for _ in range(2):
            v.step(dt, 1.0, 1.0, phi, rho_nu=rho)
        v.status()
        _, launches = v.read_timers()
        out[tiles] = (f.cpu().numpy(), rho.cpu().numpy(), launches)
        v.close()
    assert np.array_equal(out[True][0], out[False][0])
    assert np.array_equal(out[True][1], out[False][1])
    for k in ("sweep_x", "sweep_y", "sweep_z"):
        assert out[True][2][k] == 2 and out[False][2][k] == 2
    assert out[True][2]["moment"] == 2  # the partial sums of the tile x sweep, added per cell


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_16bit_tile_sweeps_against_the_oracle(fmt):
    # BF16 / FP16 storage with n_uz = 32 runs the staged tiles too (decode, FP32 march,
    # stochastic-rounding encode per value with the kept line scales).  Its random streams
    # differ from the streamed sweep's, so both are held to the codec bound of the parity
    # tests against the FP64 oracle's sweep of the same decoded input: relative L1 <=
    # 2^-8 (BF16) / 2^-11 (FP16) + 1e-6, L_inf <= 1.5 x twice that, per sweep and axis.
    B = _lib()
    V = 5.0
    bound = {"bf16": 2.0 ** -8, "f16": 2.0 ** -11}[fmt]
    tdt = {"bf16": torch.bfloat16, "f16": torch.float16}[fmt]
    n, nu = (32, 16, 16), (16, 16, 32)
    f0 = I.initial_f(I.gaussian_field(n, 0.05, seed=8), I.fermi_dirac(nu, V), np.float64)
    g = O.grid(n, nu, V=V)
    codes0, scale0 = B.encode_lines(torch.from_numpy(f0).cuda(), tdt)
    for ax in range(3):
        dt = 0.8 / O.max_abs_nu(g, ax, 1.0, 0.9)
        ref = B.decode_lines(codes0, scale0).cpu().numpy()
        O.sweep(g, ref, ax, dt, 0.9)
        for tiles in (True, False):
            codes, scale = codes0.clone(), scale0.clone()
            v = B.Vlasov(codes, V=V, scale=scale)
            v.set_position_tiles(tiles)
            v.sweep(ax, dt, 0.9)
            v.status()
            out = B.decode_lines(codes, scale).cpu().numpy()
            v.close()
            err = np.abs(out - ref)
            rl1 = err.sum() / np.abs(ref).sum()
            rinf = err.max() / np.abs(ref).max()
            print("%s axis %d %s: rel L1 %.2e, rel Linf %.2e" % (fmt, ax, "tiles" if tiles else "streamed", rl1, rinf))
            assert rl1 <= bound + 1e-6 and rinf <= 1.5 * (2 * bound + 1e-6)
            assert torch.equal(scale, scale0)  # a position sweep keeps the line scales


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_16bit_tile_sweeps_with_48_cell_lines(fmt):
    # n_uz = 48: a tile's 256 columns fall on 6 or 7 u_z lines, starting inside one, so each
    # column finds its own line's scale in a box of 12 read from the line index rounded down
    # to a multiple of 4; a warp's 32 columns span one or two lines.  One 48-cell position
    # axis at a time (the staged tiles take L = 48), against the FP64 oracle with the codec
    # bound, tiles and streamed sweep alike.
    B = _lib()
    V = 5.0
    bound = {"bf16": 2.0 ** -8, "f16": 2.0 ** -11}[fmt]
    tdt = {"bf16": torch.bfloat16, "f16": torch.float16}[fmt]
    nu = (8, 8, 48)
    for ax in range(3):
        n = tuple(48 if k == ax else 4 for k in range(3))
        f0 = I.initial_f(I.gaussian_field(n, 0.05, seed=9 + ax), I.fermi_dirac(nu, V), np.float64)
        g = O.grid(n, nu, V=V)
        codes0, scale0 = B.encode_lines(torch.from_numpy(f0).cuda(), tdt)
        dt = 0.8 / O.max_abs_nu(g, ax, 1.0, 0.9)
        ref = B.decode_lines(codes0, scale0).cpu().numpy()
        O.sweep(g, ref, ax, dt, 0.9)
        for tiles in (True, False):
            codes, scale = codes0.clone(), scale0.clone()
            v = B.Vlasov(codes, V=V, scale=scale)
            v.set_position_tiles(tiles)
            v.sweep(ax, dt, 0.9)
            v.status()
            out = B.decode_lines(codes, scale).cpu().numpy()
            v.close()
            err = np.abs(out - ref)
            rl1 = err.sum() / np.abs(ref).sum()
            rinf = err.max() / np.abs(ref).max()
            print("%s n_uz 48 axis %d %s: rel L1 %.2e, rel Linf %.2e" % (fmt, ax, "tiles" if tiles else "streamed", rl1, rinf))
            assert rl1 <= bound + 1e-6 and rinf <= 1.5 * (2 * bound + 1e-6)
            assert torch.equal(scale, scale0)


@pytest.mark.parametrize("n,nu", [((4, 4, 4), (48, 48, 48)), ((4, 5, 4), (48, 8, 32))])
def test_ux_tile_sweep_is_bitwise_the_streamed_sweep(n, nu):
    B = _lib()
    V = 5.0
    f0 = I.initial_f(I.gaussian_field(n, 0.05, seed=11), I.fermi_dirac(nu, V), np.float32)
    phi_np = I.fourier_potential(n, seed=12)
    g = O.grid(n, nu, V=V)
    dt = 0.8 / O.max_abs_nu(g, 3, 1.0, 1.0, phi_np)
    phi = torch.from_numpy(phi_np.astype(np.float32)).cuda()
    out = {}
    for tiles in (True, False):
        f = torch.from_numpy(f0).cuda()
        v = B.Vlasov(f, V=V)
        v.set_position_tiles(tiles)
        v.sweep(3, dt, 1.0, phi)
        v.sweep(3, -0.6 * dt, 1.0, phi)
        v.status()
        out[tiles] = f.cpu().numpy()
        v.close()
    assert np.array_equal(out[True], out[False])


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_16bit_ux_tile_sweep_against_the_oracle(fmt):
    # n_ux = n_uz = 48: the u_x tiles take each column's own u_z line scale per row, as
    # the position tiles do; held to the codec bound against the FP64 oracle's sweep of
    # the decoded input, like the register-line sweep (whose random streams differ: the
    # codes of the two must not be equal, which shows that two kernels ran)
    B = _lib()
    V = 5.0
    bound = {"bf16": 2.0 ** -8, "f16": 2.0 ** -11}[fmt]
    tdt = {"bf16": torch.bfloat16, "f16": torch.float16}[fmt]
    n, nu = (4, 4, 4), (48, 16, 48)
    f0 = I.initial_f(I.gaussian_field(n, 0.05, seed=13), I.fermi_dirac(nu, V), np.float64)
    phi_np = I.fourier_potential(n, seed=14)
    g = O.grid(n, nu, V=V)
    dt = 0.8 / O.max_abs_nu(g, 3, 1.0, 1.0, phi_np)
    phi = torch.from_numpy(phi_np.astype(np.float32)).cuda()
    codes0, scale0 = B.encode_lines(torch.from_numpy(f0).cuda(), tdt)
    ref = B.decode_lines(codes0, scale0).cpu().numpy()
    O.sweep(g, ref, 3, dt, 1.0, phi_np)
    got = {}
    for tiles in (True, False):
        codes, scale = codes0.clone(), scale0.clone()
        v = B.Vlasov(codes, V=V, scale=scale)
        v.set_position_tiles(tiles)
        v.sweep(3, dt, 1.0, phi)
        v.status()
        out = B.decode_lines(codes, scale).cpu().numpy()
        v.close()
        err = np.abs(out - ref)
        rl1 = err.sum() / np.abs(ref).sum()
        rinf = err.max() / np.abs(ref).max()
        print("%s u_x %s: rel L1 %.2e, rel Linf %.2e" % (fmt, "tiles" if tiles else "lines", rl1, rinf))
        assert rl1 <= bound + 1e-6 and rinf <= 1.5 * (2 * bound + 1e-6)
        assert torch.equal(scale, scale0)  # the u_x sweep keeps the line scales
        got[tiles] = codes
    assert not torch.equal(got[True], got[False])
