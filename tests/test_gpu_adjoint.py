"""Parity of the CUDA adjoint (reverse mode of the sweeps and of one Eq. (5) step,
through the C ABI) with the oracle's adjoint, itself pinned by finite differences and
the dot-product identity (tests/test_oracle_adjoint.py).

Tolerances.  FP64 storage: the GPU takes the oracle's limiter branches (ties need a
difference below 1e-16 relative), so lambda agrees to rounding: relative L1 <= 1e-12,
L_inf <= 1e-10 of max |lambda|, dL/dg and dL/dphi to 1e-10 of their largest entry.
FP32 storage: arithmetic in FP32 against the FP64 oracle on the same FP32 input.
Where the forward sits within FP32 rounding of a limiter switch the two sides may take
different branches (and over a step the FP32 forward states drift from the FP64 ones
by rounding, so more faces sit near a switch); each such face moves a few entries by
O(|lambda|).  For one sweep at most 2e-4 of the entries may be off by more than 1e-3
of max |lambda| and the others, leaving out the cells within 3 of an off entry along
the swept axis (the stencil of the flipped face), must agree to FP32 rounding (relative
L1 <= 1e-6 over them).  Over a step the later adjoint sweeps spread each flip over its neighbours, so
there the bound is at most 2e-4 of the entries off by 1e-3 and relative L1 <= 1e-3
overall.  The measured values are printed.
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


def _setup(n, nu, V=5.0, seed=1, rms=0.01, dtype=np.float32):
    Fu = I.fermi_dirac(nu, V)
    delta = I.gaussian_field(n, rms, seed=seed)
    f0 = I.initial_f(delta, Fu, dtype)
    phi = I.fourier_potential(n, seed=seed + 10).astype(np.float32)
    lam = np.random.default_rng(seed + 20).standard_normal(f0.shape).astype(dtype)
    return f0, phi, lam


def _dt_for(g, axis, phi, cfl, a=1.0):
    return cfl / O.max_abs_nu(g, axis, 1.0, a, phi.astype(np.float64))


def _dt_step(g, phi, cfl, a=1.0):
    # kicks advance dt / 2, the drift dt
    m = max([O.max_abs_nu(g, ax, 0.5, a, phi.astype(np.float64)) for ax in (3, 4, 5)] +
            [O.max_abs_nu(g, ax, 1.0, a, phi.astype(np.float64)) for ax in (0, 1, 2)])
    return cfl / m


def _compare(gpu, ref, fp64, what="", step=False, axis=None):
    gpu = np.asarray(gpu, dtype=np.float64)
    err = np.abs(gpu - ref)
    scale = np.abs(ref).max()
    rl1 = err.sum() / np.abs(ref).sum()
    rinf = err.max() / scale
    off = err > 1e-3 * scale
    bad = np.count_nonzero(off) / err.size
    # a limiter branch that flips at one face moves the adjoint of the cells of that
    # face's stencil (up to 3 cells away along the swept axis) by amounts that can stay
    # below the off-branch threshold: the on-branch set leaves those cells out
    near = off.copy()
    if axis is not None:
        for k in range(1, 4):
            near |= np.roll(off, k, axis) | np.roll(off, -k, axis)
    rl1_on = err[~near].sum() / np.abs(ref[~near]).sum()
    print("%s rel L1 %.2e  rel Linf %.2e  off-branch fraction %.2e  rel L1 on-branch %.2e"
          % (what, rl1, rinf, bad, rl1_on))
    if fp64:
        assert rl1 <= 1e-12 and rinf <= 1e-10, (rl1, rinf)
    elif step:
        assert bad <= 2e-4 and rl1 <= 1e-3, (rl1, rinf, bad, rl1_on)
    else:
        assert bad <= 2e-4 and rl1_on <= 1e-6, (rl1, rinf, bad, rl1_on)


def _compare_field(gpu, ref, fp64, what=""):
    gpu = np.asarray(gpu, dtype=np.float64)
    rel = np.abs(gpu - ref).max() / np.abs(ref).max()
    rl2 = np.linalg.norm(gpu - ref) / np.linalg.norm(ref)
    print("%s rel Linf %.2e  rel L2 %.2e" % (what, rel, rl2))
    if fp64:
        assert rel <= 1e-10, rel
    else:
        assert rl2 <= 1e-3, rl2


SHAPES = [
    ((16, 16, 16), (16, 16, 16)),   # u_z lines of 16 in registers
    ((6, 5, 7), (8, 20, 12)),       # ragged; u_z lines of 12 through the column march
    ((4, 5, 8), (4, 8, 32)),        # periodic lines of 4 and 5; u_x lines of 4; u_z rows of 32
    ((32, 32, 16), (8, 8, 8)),      # FP32 position lines of 32 and 16 through staged tiles
]


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("n,nu", SHAPES)
@pytest.mark.parametrize("axis", [0, 1, 2, 3, 4, 5])
def test_sweep_adjoint(n, nu, axis, dtype):
    B = _lib()
    f0, phi, lam0 = _setup(n, nu, dtype=dtype)
    g = O.grid(n, nu, V=5.0)
    a = 1.0
    dt = _dt_for(g, axis, phi, 0.8, a)
    lam_ref = lam0.astype(np.float64)
    dLdg_ref = O.sweep_adjoint(g, f0.astype(np.float64), lam_ref, axis, dt, a, phi.astype(np.float64))
    dev = torch.device("cuda")
    f_in = torch.from_numpy(f0).to(dev)
    lam = torch.from_numpy(lam0).to(dev)
    own = torch.zeros_like(f_in)
    v = B.Vlasov(own, L=1.0, V=5.0)
    dLdg = torch.zeros(n, dtype=torch.float64, device=dev) if axis >= 3 else None
    v.sweep_adjoint(f_in, lam, axis, dt, a, torch.from_numpy(phi).to(dev), dLdg)
    v.status()
    fp64 = dtype == np.float64
    _compare(lam.cpu().numpy(), lam_ref, fp64, "axis %d lambda" % axis, axis=axis)
    if axis >= 3:
        _compare_field(dLdg.cpu().numpy(), dLdg_ref, fp64, "axis %d dL/dg" % axis)
    assert torch.equal(f_in.cpu(), torch.from_numpy(f0))  # the sweep input is read only
    v.close()


def _rough_velocity_f(n, nu, dtype, seed=7):
    # the Fermi-Dirac profile times positive white noise, with a tenth of the cells
    # nearly emptied: velocity lines whose constraint acts at many faces (and whose
    # positivity clamp acts on the nearly empty donors), unlike the smooth profiles.
    # No exact zeros: equal neighbours would tie the limiter's selections, where the
    # oracle's min / max and the kernel may credit different (equal) arguments
    rng = np.random.default_rng(seed)
    f = I.initial_f(I.gaussian_field(n, 0.01, seed=seed), I.fermi_dirac(nu, 5.0), np.float64)
    f *= 0.2 + rng.random(f.shape)
    f[rng.random(f.shape) < 0.1] *= 1e-3
    return f.astype(dtype)


def _general_path_fraction(f, axis, s):
    # share of the faces of the velocity lines along `axis` (fractional Courant number
    # s, flow toward +index) where fbar is not between c0 and f_MP = median(c0, cp1,
    # f_UL), i.e. where the adjoint cannot take the plain-face path
    c = np.moveaxis(f.astype(np.float64), axis, -1)
    pad = np.zeros(c.shape[:-1] + (3,))
    e = np.concatenate([pad, c, pad], -1)
    m = c.shape[-1]
    cm2, cm1, c0, cp1, cp2 = (e[..., 3 + o:3 + o + m] for o in (-2, -1, 0, 1, 2))
    # weights of the mean flux over the departure interval, in powers of s
    W = np.array([[2, -13, 47, 27, -3]]) / 60.0
    w = (W[0] + np.array([0, -1 / 24, 5 / 8, -5 / 8, 1 / 24]) * s + np.array([-1 / 24, 1 / 4, -1 / 3, 1 / 12, 1 / 24]) * s ** 2
         + np.array([0, 1 / 24, -1 / 8, 1 / 8, -1 / 24]) * s ** 3 + np.array([1 / 120, -1 / 30, 1 / 20, -1 / 30, 1 / 120]) * s ** 4)
    fbar = w[0] * cm2 + w[1] * cm1 + w[2] * c0 + w[3] * cp1 + w[4] * cp2
    ful = c0 + (1 - s) / s * (c0 - cm1)
    fmp = np.median(np.stack([c0, cp1, ful]), axis=0)
    between = (fbar >= np.minimum(c0, fmp)) & (fbar <= np.maximum(c0, fmp))
    return 1.0 - between[..., :m - 1].mean()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("n,nu", [((4, 4, 4), (16, 16, 16)), ((4, 5, 6), (8, 20, 32))])
@pytest.mark.parametrize("axis", [3, 4, 5])
def test_sweep_adjoint_rough_velocity_lines(n, nu, axis, dtype):
    # On smooth velocity profiles every face of a velocity adjoint is plain (fbar kept,
    # no curvature adjoint pending); rough lines run its general path at many faces and
    # the hand-over between the two, which must agree with the oracle as well
    B = _lib()
    f0 = _rough_velocity_f(n, nu, dtype)
    phi = I.fourier_potential(n, seed=11).astype(np.float32)
    lam0 = np.random.default_rng(21).standard_normal(f0.shape).astype(dtype)
    assert _general_path_fraction(f0, axis, 0.5) > 0.5  # (smooth profiles: about 0.13)
    g = O.grid(n, nu, V=5.0)
    dt = _dt_for(g, axis, phi, 0.8)
    lam_ref = lam0.astype(np.float64)
    dLdg_ref = O.sweep_adjoint(g, f0.astype(np.float64), lam_ref, axis, dt, 1.0, phi.astype(np.float64))
    dev = torch.device("cuda")
    lam = torch.from_numpy(lam0).to(dev)
    dLdg = torch.zeros(n, dtype=torch.float64, device=dev)
    v = B.Vlasov(torch.zeros(f0.shape, dtype=lam.dtype, device=dev), L=1.0, V=5.0)
    v.sweep_adjoint(torch.from_numpy(f0).to(dev), lam, axis, dt, 1.0, torch.from_numpy(phi).to(dev), dLdg)
    v.status()
    fp64 = dtype == np.float64
    _compare(lam.cpu().numpy(), lam_ref, fp64, "rough axis %d lambda" % axis, axis=axis)
    _compare_field(dLdg.cpu().numpy(), dLdg_ref, fp64, "rough axis %d dL/dg" % axis)
    v.close()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_sweep_adjoint_whole_cell_shift(axis, dtype):
    # |nu| up to 2.6: the forward shifts whole cells after the fractional update
    B = _lib()
    n, nu = (8, 6, 10), (8, 8, 12)
    f0, phi, lam0 = _setup(n, nu, dtype=dtype)
    g = O.grid(n, nu, V=5.0)
    dt = _dt_for(g, axis, phi, 2.6)
    lam_ref = lam0.astype(np.float64)
    O.sweep_adjoint(g, f0.astype(np.float64), lam_ref, axis, dt, 1.0)
    f_in = torch.from_numpy(f0).cuda()
    lam = torch.from_numpy(lam0).cuda()
    v = B.Vlasov(torch.zeros_like(f_in), V=5.0)
    v.sweep_adjoint(f_in, lam, axis, dt, 1.0)
    v.status()
    _compare(lam.cpu().numpy(), lam_ref, dtype == np.float64, "axis %d shift lambda" % axis, axis=axis)
    v.close()


@pytest.mark.parametrize("n,nu", [((8, 8, 8), (8, 8, 8)), ((4, 6, 5), (12, 8, 16))])
def test_step_adjoint_fp64(n, nu):
    B = _lib()
    f0, phi, lam0 = _setup(n, nu, dtype=np.float64)
    g = O.grid(n, nu, V=5.0)
    dt = _dt_step(g, phi, 0.8)
    a_half = 1.0
    lam_ref = lam0.copy()
    dphi_ref = O.step_adjoint(g, f0, lam_ref, dt, a_half, phi.astype(np.float64))
    f_n = torch.from_numpy(f0).cuda()
    lam = torch.from_numpy(lam0).cuda()
    own = torch.from_numpy(f0 * 0.5).cuda()
    own_before = own.clone()
    v = B.Vlasov(own, V=5.0)
    dphi = torch.zeros(n, dtype=torch.float64, device="cuda")
    v.step_adjoint(f_n, lam, dt, a_half, torch.from_numpy(phi).cuda(), dphi)
    v.status()
    _compare(lam.cpu().numpy(), lam_ref, True, "step lambda")
    _compare_field(dphi.cpu().numpy(), dphi_ref, True, "step dL/dphi")
    assert torch.equal(own, own_before)  # the context's own f is untouched
    # a second call reuses the scratch and accumulates into dL/dphi
    lam2 = torch.from_numpy(lam0).cuda()
    v.step_adjoint(f_n, lam2, dt, a_half, torch.from_numpy(phi).cuda(), dphi)
    v.status()
    assert torch.equal(lam2, lam)
    _compare_field(dphi.cpu().numpy(), 2 * dphi_ref, True, "step dL/dphi twice")
    v.close()


def _rel(x, y, order=1):
    return np.linalg.norm((x - y).ravel(), order) / np.linalg.norm(y.ravel(), order)


def test_step_adjoint_fp32():
    # The adjoint of the limited step is piecewise: near a limiter switch a rounding-
    # level change of the state moves lambda and dL/dphi by O(1) locally (in the f_UL
    # branch dF/ds carries d alpha/ds = -(1 + alpha)^2).  The FP32 result is pinned to
    # that conditioning: its distance from the FP64 oracle is at most 3x the oracle's
    # own spread when its input is perturbed by 4 FP32 roundings (4 * 2^-24 relative).
    B = _lib()
    n, nu = (16, 16, 16), (16, 16, 16)
    f0, phi, lam0 = _setup(n, nu)
    g = O.grid(n, nu, V=5.0)
    dt = _dt_step(g, phi, 0.8)
    f64, phi64 = f0.astype(np.float64), phi.astype(np.float64)
    lam_ref = lam0.astype(np.float64)
    dphi_ref = O.step_adjoint(g, f64, lam_ref, dt, 1.0, phi64)
    fp = f64 * (1 + 4 * 2.0 ** -24 * np.random.default_rng(99).uniform(-1, 1, f64.shape))
    lam_p = lam0.astype(np.float64)
    dphi_p = O.step_adjoint(g, fp, lam_p, dt, 1.0, phi64)
    sens_l, sens_p = _rel(lam_p, lam_ref), _rel(dphi_p, dphi_ref, 2)

    f_n = torch.from_numpy(f0).cuda()
    lam = torch.from_numpy(lam0).cuda()
    v = B.Vlasov(torch.zeros_like(f_n), V=5.0)
    dphi = torch.zeros(n, dtype=torch.float64, device="cuda")
    v.step_adjoint(f_n, lam, dt, 1.0, torch.from_numpy(phi).cuda(), dphi)
    v.status()
    err_l = _rel(lam.cpu().numpy().astype(np.float64), lam_ref)
    err_p = _rel(dphi.cpu().numpy(), dphi_ref, 2)
    print("step lambda rel L1 %.2e (oracle spread %.2e); dL/dphi rel L2 %.2e (oracle spread %.2e)"
          % (err_l, sens_l, err_p, sens_p))
    assert err_l <= 3 * sens_l + 1e-6 and err_p <= 3 * sens_p + 1e-6
    v.close()


def test_adjoint_argument_errors():
    B = _lib()
    n, nu = (8, 8, 8), (16, 16, 16)
    f0, phi, lam0 = _setup(n, nu)
    f = torch.from_numpy(f0).cuda()
    v = B.Vlasov(f, V=5.0)
    with pytest.raises(B.VlasovError) as e:
        v.sweep_adjoint(f, f, 0, 0.01)        # lambda aliases the input
    assert e.value.code == B.EINVAL
    with pytest.raises(B.VlasovError) as e:
        v.sweep_adjoint(f, torch.from_numpy(lam0).cuda(), 3, 0.01)  # velocity sweep without phi
    assert e.value.code == B.EINVAL
    v.close()
    codes, scale = B.encode_lines(f, torch.bfloat16)
    vb = B.Vlasov(codes, V=5.0, scale=scale)
    with pytest.raises(B.VlasovError) as e:
        vb.sweep_adjoint(codes, codes.clone(), 0, 0.01)  # 16-bit storage has no adjoint
    assert e.value.code == B.EINVAL
    vb.close()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("cfl", [0.8, 1.7])
def test_step_adjoint_low_memory_is_the_same(dtype, cfl):
    # four scratch arrays (inputs of sweeps 3 and 6 kept, the rest rebuilt) against eight
    # (every input recorded): the same kernels on the same inputs, so lambda is bit for bit;
    # dL/dphi sums the lines of each cell with FP64 atomics, whose order varies from run to
    # run, so it agrees to 1e-12 of its largest entry; cfl 1.7 includes whole-cell shifts
    B = _lib()
    n, nu = (8, 6, 8), (8, 12, 16)
    f0, phi, lam0 = _setup(n, nu, dtype=dtype)
    g = O.grid(n, nu, V=5.0)
    m = max([O.max_abs_nu(g, ax, 1.0, 1.0, phi.astype(np.float64)) for ax in (0, 1, 2)])
    mv = max([O.max_abs_nu(g, ax, 0.5, 1.0, phi.astype(np.float64)) for ax in (3, 4, 5)])
    dt = min(cfl / m, 0.8 / mv)
    out = {}
    for arrays in (8, 4):
        v = B.Vlasov(torch.from_numpy(f0).cuda(), V=5.0)
        v.set_adjoint_arrays(arrays)
        lam = torch.from_numpy(lam0).cuda()
        dphi = torch.zeros(n, dtype=torch.float64, device="cuda")
        v.step_adjoint(torch.from_numpy(f0).cuda(), lam, dt, 1.0, torch.from_numpy(phi).cuda(), dphi)
        v.status()
        out[arrays] = (lam.cpu().numpy(), dphi.cpu().numpy())
        v.close()
    assert np.array_equal(out[4][0], out[8][0])
    assert np.abs(out[4][1] - out[8][1]).max() <= 1e-12 * np.abs(out[8][1]).max()
    if dtype == np.float64:
        lam_ref = lam0.copy()
        dphi_ref = O.step_adjoint(g, f0, lam_ref, dt, 1.0, phi.astype(np.float64))
        _compare(out[4][0], lam_ref, True, "low-memory step lambda")
        _compare_field(out[4][1], dphi_ref, True, "low-memory step dL/dphi")


def test_dLdphi_is_reproducible_when_cells_fill_blocks():
    # n_u = 16: every velocity line set of a cell (256 lines) fills whole 256-thread blocks,
    # so dL/dg is summed per cell in a fixed order: two runs agree bit for bit
    B = _lib()
    n, nu = (6, 8, 4), (16, 16, 16)
    f0, phi, lam0 = _setup(n, nu)
    g = O.grid(n, nu, V=5.0)
    dt = _dt_step(g, phi, 0.8)
    runs = []
    for _ in range(2):
        v = B.Vlasov(torch.from_numpy(f0).cuda(), V=5.0)
        lam = torch.from_numpy(lam0).cuda()
        dphi = torch.zeros(n, dtype=torch.float64, device="cuda")
        v.step_adjoint(torch.from_numpy(f0).cuda(), lam, dt, 1.0, torch.from_numpy(phi).cuda(), dphi)
        v.status()
        runs.append((lam.cpu().numpy(), dphi.cpu().numpy()))
        v.close()
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])


def test_step_record_with_48_cell_velocity_lines():
    # n_u = 48: the recorded step runs D_ux on the staged tiles of [cell][u_x][u_y u_z] out
    # of place (each sweep reads one array and writes the next); its result equals the
    # in-place step (which takes the fused staged-plane tail) bit for bit, and the recorded
    # adjoint of that step runs on the recorded inputs (finite, and the same as the
    # adjoint that records into the library's own arrays)
    B = _lib()
    n, nu = (4, 4, 4), (48, 48, 48)
    f0, phi, lam0 = _setup(n, nu)
    g = O.grid(n, nu, V=5.0)
    dt = _dt_step(g, phi, 0.8)
    phi_t = torch.from_numpy(phi).cuda()
    f = torch.from_numpy(f0).cuda()
    v = B.Vlasov(f, V=5.0)
    f_n = f.clone()
    rec = [torch.empty_like(f) for _ in range(8)]
    f_next = torch.empty_like(f)
    v.step_record(f_n, rec, dt, 1.0, phi_t, f_next)
    v.step(dt, 1.0, 1.0, phi_t)
    v.status()
    assert torch.equal(f_next, f)
    lam = torch.from_numpy(lam0).cuda()
    dphi = torch.zeros(n, dtype=torch.float64, device="cuda")
    v.step_adjoint_recorded(f_n, rec, lam, dt, 1.0, phi_t, dphi)
    lam2 = torch.from_numpy(lam0).cuda()
    dphi2 = torch.zeros(n, dtype=torch.float64, device="cuda")
    v.step_adjoint(f_n, lam2, dt, 1.0, phi_t, dphi2)
    v.status()
    assert torch.isfinite(lam).all() and torch.isfinite(dphi).all()
    assert torch.equal(lam, lam2)
    assert (dphi - dphi2).abs().max() <= 1e-12 * dphi.abs().max()
    v.close()
