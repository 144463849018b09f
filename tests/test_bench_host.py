"""Host-side arithmetic of bench.py, on the CPU:

- the Courant numbers it picks dt from (courant_per_dt: |u| / (a^2 dx) per position axis,
  |g_i| / du per velocity axis with the periodic 4th-order gradient) equal the oracle's
  largest Courant number of each axis (Eq. 3 and Eq. 4);
- drift_dt makes the largest position Courant number at a_half exactly the step's CFL;
- the a(t) schedule runs linearly from a0 to a1 once over the steps of a run, with a_half
  the midpoint and every step's CFL inside the configured range;
- the source hash behind the traffic record ignores comments and blank lines, and changes
  with the code.
"""
import os
import sys

import numpy as np
import pytest

import oracle as O
from paper_2110_15867_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("n,nu,V", [((8, 6, 5), 16, 5.0), ((6, 6, 6), 12, 8.0)])
def test_courant_per_dt_matches_the_oracle(n, nu, V):
    phi = I.fourier_potential(n, seed=21)
    c = bench.courant_per_dt(phi, n, nu, V)
    g = O.grid(n, (nu, nu, nu), V=V)
    for ax in range(6):
        ref = O.max_abs_nu(g, ax, 1.0, 1.0, phi.astype(np.float64))
        assert c[ax] == pytest.approx(ref, rel=1e-12), ax


def test_drift_dt_puts_the_largest_position_courant_number_at_cfl():
    w = bench.WORKLOAD
    g = O.grid(w["n"], w["nu"], V=w["V"])
    for k in range(3):
        _, a_h, _, cfl = bench.schedule(k, 3)
        dt = bench.drift_dt(cfl, a_h, w["n"], w["nu"], w["V"], w["L"])
        for ax in range(3):
            assert O.max_abs_nu(g, ax, dt, a_h, None) == pytest.approx(cfl, rel=1e-12)


@pytest.mark.parametrize("nsteps", [10, 20, 3])
def test_schedule_runs_a_linearly_with_midpoint_drift(nsteps):
    w = bench.WORKLOAD
    prev_end = None
    for k in range(nsteps):
        a_s, a_h, a_e, cfl = bench.schedule(k, nsteps)
        assert a_s < a_h < a_e and a_h == pytest.approx(0.5 * (a_s + a_e))
        assert w["cfl"][0] <= cfl <= w["cfl"][1]
        if prev_end is not None:
            assert a_s == pytest.approx(prev_end)
        prev_end = a_e
    assert bench.schedule(0, nsteps)[0] == pytest.approx(w["a0"])
    assert prev_end == pytest.approx(w["a1"])


def test_source_hash_ignores_comments_only():
    code = "int f(int a) {\n    return a + 1; // one more\n}\n"
    commented = "/* header\n   comment */\n" + code.replace("// one more", "// changed") + "\n\n// trailing\n"
    changed = code.replace("a + 1", "a + 2")
    assert bench._code_only(code) == bench._code_only(commented)
    assert bench._code_only(code) != bench._code_only(changed)
    for kind in bench.KERNEL_SOURCES:
        h = bench.kernel_source_hash(kind)
        assert isinstance(h, str) and len(h) == 16
    assert bench.kernel_source_hash("no_such_kernel") is None


def test_step_bandwidth_counts_one_pass_per_sweep_launch():
    # two one-pass kicks and three position sweeps per step: five passes of 8 B per cell,
    # whatever the updates a pass makes
    kind_n = {"kick": 6, "sweep_x": 3, "sweep_y": 3, "sweep_z": 3, "moment": 3, "poisson": 27}
    kinds = ["kick", "sweep_x", "sweep_y", "sweep_z"]
    r = bench.step_bandwidth(kind_n, kinds, cells=1000, steps=3, ms_per_step=1.0, hbm_peak=100.0)
    assert r["passes_per_step"] == 5
    assert r["bytes_per_step"] == 5 * bench.BYTES_PER_UPDATE * 1000
    assert abs(r["GBs"] - 5 * 8 * 1000 / 1e-3 / 1e9) < 1e-12
    assert abs(r["frac_of_measured"] - r["GBs"] / 100.0) < 1e-15
