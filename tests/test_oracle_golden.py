"""The golden line fixtures (tests/golden/sweep_lines_fp64.json, written from the oracle by
tests/golden/make_golden.py): the oracle still produces them, and they hold what the
mathematics fixes for a conservative, positivity-preserving SL sweep (Eq. 3 / Eq. 4,
Sec. 4.2): the line sum is conserved (periodic lines; zero-flux lines lose nothing at
their closed ends), nu = 0 is the identity, an integer Courant number on a periodic line
is an exact shift, and no value is negative."""
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "sweep_lines_fp64.json")


def _load():
    with open(GOLDEN) as fh:
        return json.load(fh)


def test_the_oracle_reproduces_the_golden_lines():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    now, stored = mg.build(), _load()
    assert now["position_x"]["nu"] == stored["position_x"]["nu"]
    pairs = list(zip(now["position_x"]["lines"], stored["position_x"]["lines"]))
    pairs += [(a["line"], b["line"]) for a, b in zip(now["periodic"], stored["periodic"])]
    pairs += [(a["line"], b["line"]) for a, b in zip(now["zero_flux"], stored["zero_flux"])]
    for a, b in pairs:
        np.testing.assert_allclose(a, b, rtol=1e-14, atol=1e-16)


def test_golden_lines_conserve_mass_and_stay_positive():
    d = _load()
    c = np.array(d["profile"])
    lines = [np.array(x) for x in d["position_x"]["lines"]]
    lines += [np.array(e["line"]) for e in d["periodic"]] + [np.array(e["line"]) for e in d["zero_flux"]]
    for line in lines:
        assert abs(line.sum() - c.sum()) <= 1e-14 * c.sum()
        assert (line >= 0).all()


@pytest.mark.parametrize("block", ["periodic", "zero_flux"])
def test_golden_identity_and_integer_shift(block):
    d = _load()
    c = np.array(d["profile"])
    for e in d[block]:
        line = np.array(e["line"])
        if e["nu"] == 0.0:
            assert np.array_equal(line, c)
        if block == "periodic" and float(e["nu"]).is_integer():
            assert np.array_equal(line, np.roll(c, int(e["nu"])))
