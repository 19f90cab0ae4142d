"""The allocation-free chemical-potential entry point against the context's own Fermi-level solve.

The file name sorts last, so pytest collects it after every other test file; it also passes alone.
Tolerances: mu within 1e-11 Ha (both solves stop at a Newton correction below 1e-14 Ha or a
bracket below 1e-13 Ha), occupations within 1e-9 (|df/dmu| <= 1/(4 kT) = 25 Ha^-1 at kT = 0.01),
electron count within 1e-9.
"""
import numpy as np
import pytest

import workloads
from oracle import fermi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DC_ERR_ARG = -1  # include/dcdft.h


def _ne(cfg):
    return float(np.sum(cfg["spec"]["Z"][cfg["species"]]))


@pytest.fixture(scope="module")
def si8():
    from paper_2606_21125_b300 import DCSolver
    cfg = workloads.make_config("si8", precision="fp64")
    s = DCSolver(cfg)
    s.warmup()
    rho, q, mu = s.density()
    _, eps = s.get_state()
    torch.cuda.synchronize()
    return cfg, eps, q, float(mu.item())


def test_matches_context_fermi_level_on_two_calls_in_a_row(si8):
    from paper_2606_21125_b300 import fermi_level_noalloc
    cfg, eps, q, mu_ctx = si8
    kT = cfg["kT"]
    mu = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    occ = torch.empty_like(eps)
    for call in range(2):
        occ.fill_(-1.0)
        fermi_level_noalloc(eps, q, _ne(cfg), kT, mu, occ)
        got = float(mu.item())
        assert abs(got - mu_ctx) < 1e-11, (call, got, mu_ctx)
        ref_occ = 0.5 * (1.0 - torch.tanh(0.5 * (eps - mu_ctx) / kT))
        assert torch.max(torch.abs(occ - ref_occ)).item() < 1e-9
        assert abs(float(torch.sum(2.0 * occ * q).item()) - _ne(cfg)) < 1e-9
        mu.fill_(0.0 if call == 0 else float("nan"))  # second call starts from another guess


def test_many_blocks_against_the_oracle():
    """300,000 states (more blocks than SMs need to stride over) against the FP64 oracle's bisection."""
    from paper_2606_21125_b300 import fermi_level_noalloc
    r = np.random.default_rng(20260603)
    n = 300_000
    eps_h = np.sort(r.normal(0.0, 0.3, n))
    q_h = r.uniform(0.0, 1.0, n)
    ne = float(np.sum(q_h))  # half filling
    kT = 0.01
    mu_ref = fermi.find_mu(eps_h, q_h, ne, kT)
    eps = torch.from_numpy(eps_h).cuda()
    q = torch.from_numpy(q_h).cuda()
    mu = torch.zeros(1, dtype=torch.float64, device="cuda")
    occ = torch.empty_like(eps)
    for _ in range(2):
        fermi_level_noalloc(eps, q, ne, kT, mu, occ)
        assert abs(float(mu.item()) - mu_ref) < 1e-11
        assert abs(float(torch.sum(2.0 * occ * q).item()) - ne) < 1e-7 * ne


def test_solves_allocate_nothing(si8):
    """After the setup call, repeated solves change neither the device's free memory (any cudaMalloc
    would take at least one 2 MB page) nor the number of torch allocations."""
    from paper_2606_21125_b300 import fermi_level_noalloc, load
    cfg, eps, q, _ = si8
    assert load().dc_fermi_level_noalloc(None, None, 0, 0.0, 0.01, None, None, None) == 0
    mu = torch.zeros(1, dtype=torch.float64, device="cuda")
    occ = torch.empty_like(eps)
    fermi_level_noalloc(eps, q, _ne(cfg), cfg["kT"], mu, occ)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    n0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for _ in range(5):
        fermi_level_noalloc(eps, q, _ne(cfg), cfg["kT"], mu, occ)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    n1 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    assert free1 == free0
    assert n1 == n0


def test_wrapper_rejects_mismatched_tensors(si8):
    from paper_2606_21125_b300 import fermi_level_noalloc
    cfg, eps, q, _ = si8
    mu = torch.zeros(1, dtype=torch.float64, device="cuda")
    occ = torch.empty_like(eps)
    with pytest.raises(ValueError):
        fermi_level_noalloc(eps, q[:-1], _ne(cfg), cfg["kT"], mu, occ)
    with pytest.raises(ValueError):
        fermi_level_noalloc(eps, q.float(), _ne(cfg), cfg["kT"], mu, occ)
    with pytest.raises(ValueError):
        fermi_level_noalloc(eps, q, _ne(cfg), cfg["kT"], mu[:0], occ)
    with pytest.raises(ValueError):
        fermi_level_noalloc(eps.cpu(), q, _ne(cfg), cfg["kT"], mu, occ)


def test_setup_call_and_oversize_rejection():
    from paper_2606_21125_b300 import _lib, load
    lib = load()
    assert lib.dc_fermi_level_noalloc(None, None, 0, 0.0, 0.01, None, None, None) == _lib.DC_OK
    d = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = d.data_ptr()
    st = lib.dc_fermi_level_noalloc(p, p, 2**31, 1.0, 0.01, p, p, None)
    assert st == DC_ERR_ARG
    assert b"nstates" in lib.dc_last_error()
    st = lib.dc_fermi_level_noalloc(p, p, 4, 1.0, 0.0, p, p, None)
    assert st == DC_ERR_ARG
    assert torch.all(d == 0.0)  # rejected calls write nothing
