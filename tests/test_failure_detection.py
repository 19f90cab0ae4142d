"""Failure detection on the GPU without a fault: a bounded wait that runs out is reported, not hung.

dc_selftest_wait runs the Fermi kernel's grid barrier on a launch one block short of what the barrier
expects, so the wait cannot complete.  The library must come back with DC_ERR_TIMEOUT well inside the
poll bound, clear its device flags, and keep the context working: the core weights computed afterwards
equal those computed before bit for bit, and mu and the density agree within the Fermi solve's
stopping rule (it starts from the previous mu, so repeated solves may differ in the last bits; a
Newton correction below 1e-14 Ha and |df/dmu| <= 1/(4 kT) bound the density change far below 1e-10).
"""
import time

import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DC_ERR_TIMEOUT = -5  # include/dcdft.h


def test_grid_barrier_timeout_is_reported_and_the_context_survives():
    from paper_2606_21125_b300 import DCSolver, _stream
    cfg = workloads.small_config(n=(12, 12, 12), L=(7.2, 7.2, 7.2), bc="periodic", natom=4, precision="fp64",
                                 n_warmup=2)
    with DCSolver(cfg) as s:
        s.warmup()
        rho0, q0, mu0 = (t.clone() for t in s.density())
        torch.cuda.synchronize()
        for _ in range(2):
            t0 = time.perf_counter()
            st = s.lib.dc_selftest_wait(s.ctx, _stream())
            dt = time.perf_counter() - t0
            assert st == DC_ERR_TIMEOUT
            assert b"bounded device wait" in s.lib.dc_last_error()
            assert dt < 30.0
        rho1, q1, mu1 = s.density()
        torch.cuda.synchronize()
        assert torch.equal(q0, q1)
        assert abs(float(mu1.item()) - float(mu0.item())) < 1e-11
        assert float(torch.max(torch.abs(rho1 - rho0))) <= 1e-10 * float(torch.max(torch.abs(rho0)))
    from paper_2606_21125_b300 import load
    assert load().dc_selftest_wait(None, None) == -1
