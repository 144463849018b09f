"""The CUDA x sweep against the golden lines of tests/golden/sweep_lines_fp64.json (values of
the FP64 oracle, Eq. 3): a (16, 4, 4) x (8, 4, 4) grid whose x lines all hold the fixture's
profile, swept once at Courant numbers up to 2.4 (whole-cell shifts and both signs); every
x line of u_x column j must equal the stored line j: FP64 storage to rounding, FP32 storage
to the per-sweep tolerance (relative L1 <= 1e-6, L_inf <= 1e-4 of the largest value)."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sweep_lines_fp64.json")


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_x_sweep_matches_the_golden_lines(dtype):
    from paper_2110_15867_gb300 import binding as B
    B.load()
    with open(GOLDEN) as fh:
        d = json.load(fh)
    px = d["position_x"]
    g = px["grid"]
    n, nu = tuple(g["n"]), tuple(g["nu"])
    c = np.array(d["profile"])
    f0 = np.broadcast_to(c[:, None, None, None, None, None], n + nu).astype(dtype).copy()
    f = torch.from_numpy(f0).cuda()
    v = B.Vlasov(f, L=g["L"], V=g["V"])
    v.sweep(0, px["dt"], g["a"])
    v.status()
    out = f.cpu().numpy().astype(np.float64)
    v.close()
    for j, line in enumerate(px["lines"]):
        ref = np.array(line)
        got = out[:, :, :, j, :, :].reshape(n[0], -1)
        err = np.abs(got - ref[:, None])
        rl1 = err.sum() / (np.abs(ref).sum() * got.shape[1])
        rinf = err.max() / np.abs(ref).max()
        if dtype == np.float64:
            assert rl1 <= 1e-13 and rinf <= 1e-12, (j, px["nu"][j], rl1, rinf)
        else:
            assert rl1 <= 1e-6 and rinf <= 1e-4, (j, px["nu"][j], rl1, rinf)
