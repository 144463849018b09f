"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds none of the method's arithmetic: it only draws the initial
distribution function, the density perturbation, the external potential and the
CDM background, all on the host in FP64 with ``numpy.random.default_rng``.  Both
the FP64 oracle and the CUDA path take their inputs from here.

Recipe (the paper's cosmological initial conditions, Planck-2015 runs at 0.4 eV,
Sec. 5.1, are not reproduced; these fields stand in for them):

* velocity distribution: relativistic Fermi-Dirac shape
  F(u) = 1 / (exp(|u| / u_T) + 1) at velocity cell centres, -V <= u < V
  (the relic-neutrino distribution of Sec. 2);
* density perturbation delta(x): white noise whose Fourier amplitude is scaled
  by |k|^-1 (power spectrum P ~ k^-2), k = 0 removed, rescaled to a given rms;
* initial f0(x, u) = (1 + delta(x)) F(u), rounded once to the storage type;
* external potential phi(x) = sum over 8 modes of 0.1 cos(2 pi n.x / L + theta)
  with integer n in [-3, 3]^3 minus the origin and theta uniform in [0, 2 pi);
* CDM density contrast delta_c: the delta(x) recipe with seed + 1.
"""
from __future__ import annotations

import numpy as np


def velocity_centres(nu: int, V: float) -> np.ndarray:
    """u_j = -V + (j + 1/2) du, du = 2V / nu."""
    du = 2.0 * V / nu
    return -V + (np.arange(nu) + 0.5) * du


def spatial_centres(n: int, L: float = 1.0) -> np.ndarray:
    return (np.arange(n) + 0.5) * (L / n)


def fermi_dirac(nu, V: float, uT: float = 1.0) -> np.ndarray:
    """F(u) = 1/(exp(|u|/u_T)+1) on the nu_x x nu_y x nu_z velocity grid (FP64)."""
    if isinstance(nu, int):
        nu = (nu, nu, nu)
    ux = velocity_centres(nu[0], V)[:, None, None]
    uy = velocity_centres(nu[1], V)[None, :, None]
    uz = velocity_centres(nu[2], V)[None, None, :]
    umag = np.sqrt(ux * ux + uy * uy + uz * uz)
    return 1.0 / (np.exp(umag / uT) + 1.0)


def gaussian_field(n, rms: float, seed: int, slope: float = -2.0) -> np.ndarray:
    """Gaussian random field with power spectrum P(k) ~ k^slope, zero mean, given rms."""
    if isinstance(n, int):
        n = (n, n, n)
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(n)
    wk = np.fft.fftn(w)
    k = np.sqrt(sum(np.meshgrid(*[np.fft.fftfreq(m) * m for m in n], indexing="ij")[i] ** 2
                    for i in range(3)))
    amp = np.zeros_like(k)
    nz = k > 0
    amp[nz] = k[nz] ** (slope / 2.0)
    d = np.real(np.fft.ifftn(wk * amp))
    d -= d.mean()
    s = d.std()
    return d * (rms / s) if s > 0 else d


def fourier_potential(n, seed: int, n_modes: int = 8, amp: float = 0.1,
                      L: float = 1.0) -> np.ndarray:
    """phi(x) = sum_m amp cos(2 pi n_m . x / L + theta_m) at spatial cell centres."""
    if isinstance(n, int):
        n = (n, n, n)
    rng = np.random.default_rng(seed)
    x = [spatial_centres(m, L) for m in n]
    X = np.meshgrid(*x, indexing="ij")
    phi = np.zeros(n)
    count = 0
    while count < n_modes:
        nm = rng.integers(-3, 4, size=3)
        th = rng.uniform(0.0, 2.0 * np.pi)
        if not nm.any():
            continue
        phi += amp * np.cos(2.0 * np.pi * (nm[0] * X[0] + nm[1] * X[1] + nm[2] * X[2]) / L + th)
        count += 1
    return phi


def initial_f(delta: np.ndarray, F: np.ndarray, dtype=np.float32) -> np.ndarray:
    """f0 = (1 + delta(x)) F(u), formed in FP64 and rounded once to dtype; shape 6D."""
    f = (1.0 + delta)[:, :, :, None, None, None] * F[None, None, None, :, :, :]
    return f.astype(dtype)


# Workload recipes (sizes, precisions and schedules of the five benchmarked setups).
CONFIGS = {
    "parity16": dict(n=16, nu=16, V=5.0, delta_rms=0.01, seed=1, cfl=0.7, a=1.0,
                     dtype="f32"),
    "fp32_64x32": dict(n=64, nu=32, V=5.0, delta_rms=0.05, cdm_rms=1.0, seed=2, steps=10,
                       a0=0.5, a1=0.6, cfl=(0.5, 0.9), dtype="f32"),
    "lowprec_96x32": dict(n=96, nu=32, V=5.0, delta_rms=0.01, seed=1, steps=20, cfl=0.7,
                          a=1.0, dtype="bf16", sub_n=24, sub_nu=16),
    "adjoint_32x16": dict(n=32, nu=16, V=5.0, delta_rms=0.01, seed=1, steps=16, cfl=0.7,
                          a=1.0, checkpoint=4, fd_n=8, fd_nu=8),
    "large_48x48": dict(n=48, nu=48, V=8.0, delta_rms=0.1, cdm_rms=3.0, seed=5, steps=50,
                        a0=0.2, a1=1.0, cfl=0.9, dtype="f32"),
}
