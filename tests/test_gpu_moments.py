"""Velocity moments on the GPU (density, mean velocity, dispersion tensor; Sec. 4.1.3)
against the oracle (pinned in tests/test_oracle_moments.py) on the same stored values.

Tolerances: per-thread FP32 compensated sums of FP32 products (each product rounded
once, 6e-8 relative) combined in FP64: rho to 1e-6 of its largest value, umean to
1e-6 V (the mean is a difference of nearly cancelling sums), sigma2 to 1e-5 of its
largest entry.  FP64 storage: 1e-12."""
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


def _field(n, nu, dtype, seed=5):
    f = I.initial_f(I.gaussian_field(n, 0.3, seed=seed), I.fermi_dirac(nu, V), np.float64)
    # break the velocity symmetry so the mean velocity and off-diagonal terms are not zero
    rng = np.random.default_rng(seed)
    tilt = 1 + 0.2 * rng.standard_normal(n + (1, 1, 1)) * np.linspace(-1, 1, nu[0])[:, None, None]
    return (f * tilt).clip(0).astype(dtype)


def _check(gpu, ref, fp64):
    rho, um, s2 = [x.cpu().numpy() for x in gpu]
    rr, ur, sr = ref
    e_rho = np.abs(rho - rr).max() / np.abs(rr).max()
    e_um = np.abs(um - ur).max() / V
    e_s2 = np.abs(s2 - sr).max() / np.abs(sr).max()
    print("rho %.2e  umean %.2e (of V)  sigma2 %.2e" % (e_rho, e_um, e_s2))
    tol = (1e-12, 1e-12, 1e-12) if fp64 else (1e-6, 1e-6, 1e-5)
    assert e_rho <= tol[0] and e_um <= tol[1] and e_s2 <= tol[2]


@pytest.mark.parametrize("n,nu", [((16, 16, 16), (16, 16, 16)), ((6, 5, 7), (8, 20, 12)), ((4, 4, 4), (32, 32, 32))])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_moments_match_oracle(n, nu, dtype):
    B = _lib()
    f = _field(n, nu, dtype)
    g = O.grid(n, nu, V=V)
    ref = O.moments(g, f.astype(np.float64))
    ft = torch.from_numpy(f).cuda()
    v = B.Vlasov(ft, V=V)
    out = v.moments()
    v.status()
    _check(out, ref, dtype == np.float64)
    # the density agrees with the density kernel
    rho1 = v.moment().cpu().numpy()
    assert np.abs(out[0].cpu().numpy() - rho1).max() <= (1e-13 if dtype == np.float64 else 1e-6) * rho1.max()
    v.close()


@pytest.mark.parametrize("tdt", ["bfloat16", "float16"])
def test_moments_of_16bit_codes(tdt):
    B = _lib()
    n, nu = (6, 4, 4), (16, 16, 16)
    f = _field(n, nu, np.float32)
    codes, scale = B.encode_lines(torch.from_numpy(f).cuda(), getattr(torch, tdt))
    vals = B.decode_lines(codes, scale).cpu().numpy()
    g = O.grid(n, nu, V=V)
    ref = O.moments(g, vals)
    v = B.Vlasov(codes, V=V, scale=scale)
    out = v.moments()
    v.status()
    _check(out, ref, False)
    v.close()
