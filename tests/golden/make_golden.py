"""Write the golden line fixtures of tests/golden/ from the FP64 oracle alone.

    python tests/golden/make_golden.py

sweep_lines_fp64.json holds one 16-cell line profile (smooth, with a top hat and two
near-empty cells) and its SL-MPP5 sweep (Eq. 3 / Eq. 4; Sec. 4.2: semi-Lagrangian flux,
MP constraint, positivity clamp) at given Courant numbers: periodic lines (position
axes, whole-cell shifts included) and zero-flux lines (velocity axes, |nu| < 1).  The
"position_x" block is the x sweep of a (16, 4, 4) x (8, 4, 4) grid whose x lines all hold
the profile: its Courant numbers are those of the eight u_x columns, formed as the library
forms them, nu_j = u_j dt / (a^2 dx) with u_j = -V + (j + 1/2) du.  Nothing here calls
the CUDA path; the values are the oracle's.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402

PROFILE = [1.0 + 0.5 * np.sin(2 * np.pi * i / 16) for i in range(16)]
PROFILE[5] += 2.0
PROFILE[6] += 2.0
PROFILE[7] += 2.0
PROFILE[12] = 1e-6
PROFILE[13] = 2e-6

# x sweep of the (16, 4, 4) x (8, 4, 4) grid: L = 1, V = 5, a = 1, dt with max |nu| = 2.4
GRID = {"n": [16, 4, 4], "nu": [8, 4, 4], "L": 1.0, "V": 5.0, "a": 1.0}


def position_nus(dt):
    n, nvel, V, L, a = GRID["n"][0], GRID["nu"][0], GRID["V"], GRID["L"], GRID["a"]
    du = 2.0 * V / nvel
    dx = L / n
    return [(-V + (j + 0.5) * du) * dt / (a * a * dx) for j in range(nvel)]


def build():
    n, nvel, V, L = GRID["n"][0], GRID["nu"][0], GRID["V"], GRID["L"]
    umax = -V + (nvel - 0.5) * (2.0 * V / nvel)
    dt = 2.4 * (L / n) / umax
    nus = position_nus(dt)
    c = np.array(PROFILE)
    out = {
        "citation": "Eq. (3) and Eq. (4): one directionally split SL-MPP5 sweep of a line "
                    "(Sec. 4.2: fractional flux of the departure interval, MP constraint, positivity "
                    "clamp; position axes periodic, velocity axes zero-flux); values from the FP64 "
                    "oracle (oracle/vlasov_oracle.c) through tests/golden/make_golden.py",
        "profile": PROFILE,
        "position_x": {"grid": GRID, "dt": dt, "nu": nus,
                       "lines": [O.sweep_line(c, nu, periodic=True).tolist() for nu in nus]},
        "periodic": [{"nu": nu, "line": O.sweep_line(c, nu, periodic=True).tolist()}
                     for nu in (0.0, 0.37, -0.81, 1.0, 2.55, -3.2)],
        "zero_flux": [{"nu": nu, "line": O.sweep_line(c, nu, periodic=False).tolist()}
                      for nu in (0.0, 0.25, -0.5, 0.93, -0.99)],
    }
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "sweep_lines_fp64.json"), "w") as fh:
        json.dump(build(), fh, indent=1)
        fh.write("\n")
