"""Failure detection on the GPU without a fault: the bounded device wait (the one every
TMA kernel uses for a copy or a peer) runs out on an mbarrier phase that nothing
completes; the kernel records the timeout and returns, vlasov_status reports
VLASOV_ETIMEOUT once, and the same context then runs a sweep and reports success."""
import time

import numpy as np
import pytest

from paper_2110_15867_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_a_bounded_wait_that_runs_out_is_reported_and_the_context_stays_usable():
    from paper_2110_15867_gb300 import binding as B
    B.load()
    n, nu, V = (8, 8, 8), (8, 8, 8), 5.0
    f0 = I.initial_f(I.gaussian_field(n, 0.01, seed=3), I.fermi_dirac(nu, V), np.float32)
    f = torch.from_numpy(f0).cuda()
    v = B.Vlasov(f, V=V)
    t0 = time.perf_counter()
    v.selftest_wait()
    with pytest.raises(B.VlasovError) as e:
        v.status()
    waited = time.perf_counter() - t0
    assert e.value.code == B.ETIMEOUT
    assert 1.0 < waited < 30.0  # the wait's limit is 2 s of device time
    v.status()  # the error word was cleared
    before = f.clone()
    v.sweep(0, 0.001, 1.0)
    v.status()
    assert not torch.equal(before, f) and torch.isfinite(f).all()
    v.close()
