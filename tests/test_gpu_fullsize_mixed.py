"""The mixed-precision path at the benchmark's own sizes against the FP64 oracle (Sec. 2.2, Eqs. 1-4).

Mixed precision: FP32 stencil (orbital-pair kernel), 3xBF16 Gram on tensor cores at n = 48 with
4096-point items on persistent CTAs, the FP32/mixed subspace solve (FP32 Jacobi, FP64 Newton-Schulz,
no FP64 finishing sweeps), FP32 rotation, then core weights, the Fermi level and the density.

Input: the oracle warms each fragment up (Rayleigh-Ritz of the SplitMix64 start, then CheFSI passes in
the starting potential), rounds the orbitals to FP32 and hands them, with their Ritz values, to the
library (set_state); both sides then run one CheFSI pass and the density stage from that same
FP32-rounded state.  Tolerances are the method's accuracy budget: 1e-5 Ha for eigenvalues and mu,
1e-5 relative (L1) for the density; core weights within 1e-5 of the largest, per state where the state
is separated from its neighbours by more than 1e-2 Ha and summed over each cluster of nearly
degenerate states otherwise (their eigenvectors, hence their individual weights, are not unique), and
each fragment's occupation-weighted core charge within 1e-5 relative.
"""
import numpy as np
import pytest

import workloads
from oracle import fermi
from oracle.pool import FragmentPool
from tests.oracle_pack import oracle_state, pack, unpack_states

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WARM = 4  # oracle warm-up passes


def _gpu_pass(cfg, psi_fp32, eps, V, env=None):
    import os
    from paper_2606_21125_b300 import DCSolver
    old = {k: os.environ.get(k) for k in (env or {})}
    os.environ.update(env or {})
    try:
        s = DCSolver(cfg)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    with s:
        s.set_potential(torch.tensor(V.reshape(-1), dtype=torch.float64, device="cuda"))
        s.set_tuning("fp32", 4, 256, 1)
        s.set_state(torch.from_numpy(psi_fp32).cuda(), torch.from_numpy(eps).cuda())
        s.chefsi(1)
        _, e1 = s.get_state()
        rho, q, mu = s.density()
        torch.cuda.synchronize()
        return s.layout, e1.cpu().numpy(), q.cpu().numpy(), float(mu.item()), rho.cpu().numpy()


def _clusters(eps, gap):
    """Runs of consecutive (ascending) eigenvalues closer than ``gap``: their eigenvectors, and so their
    individual core weights, are not determined by the Hamiltonian, only the cluster's span is."""
    out, start = [], 0
    for i in range(1, len(eps) + 1):
        if i == len(eps) or eps[i] - eps[i - 1] > gap:
            out.append((start, i))
            start = i
    return out


def _assert_core_weights(st, e1, q, ref_e, ref_q, mu, gap=1e-2, frags=None):
    """Core weights (Eq. 3 projection of each state onto its fragment's core).  A single state's weight
    moves by about (error of H) / (gap to its nearest neighbour), so per state it is compared where the
    state is separated from its neighbours by more than ``gap`` Ha and summed over each cluster of
    nearly degenerate states otherwise (a sum invariant under rotations inside the cluster), within 1e-5
    of the largest weight; the occupation-weighted core charge of every fragment, sum_i 2 f_i q_i, which
    is what the Fermi level and the density use, within 1e-5 relative."""
    eps_f, q_f = unpack_states(st, ref_e), unpack_states(st, ref_q)
    got_f = unpack_states(st, q)
    tol = 1e-5 * np.max(ref_q)
    for f in (range(st.frags.nfrag) if frags is None else frags):
        for a, b in _clusters(eps_f[f], gap):
            assert abs(np.sum(got_f[f][a:b]) - np.sum(q_f[f][a:b])) < tol * (b - a), (f, a, b)
        occ = 2.0 * fermi.occupation(eps_f[f], mu, st.kT)
        ref_charge = float(np.sum(occ * q_f[f]))
        assert abs(float(np.sum(occ * got_f[f])) - ref_charge) < 1e-5 * max(ref_charge, 1e-3), f


def test_mixed_pass_and_density_si_weak64_whole():
    """All 64 fragments of the 64-atom weak-scaling cell (22^3 fragments, 48 orbitals), 4096-point Gram
    items: every eigenvalue, core weight, mu and the whole density against the oracle."""
    cfg = workloads.make_config("si_weak64", precision="mixed")
    st = oracle_state(cfg, subset=[])
    V = st.veff(st.rho_in)
    nf = st.frags.nfrag
    pool = FragmentPool(cfg, list(range(nf)))
    try:
        warm = pool.warm(V, WARM, round_fp32=True)
        res = pool.solve(V, 1)
        sq = pool.core_squares()
    finally:
        pool.close()
    psi = pack(st, {f: warm[f][0] for f in range(nf)}).astype(np.float32)
    eps0 = pack(st, {f: warm[f][1] for f in range(nf)})
    lay, e1, q, mu, rho = _gpu_pass(cfg, psi, eps0, V, env={"DC_GRAM_CHUNK": "4096"})
    ref_e = pack(st, {f: res[f][0] for f in range(nf)})
    ref_q = pack(st, {f: res[f][1] for f in range(nf)})
    assert np.max(np.abs(e1 - ref_e)) < 1e-5
    ref_mu = fermi.find_mu(ref_e, ref_q, st.ne, st.kT)
    assert abs(mu - ref_mu) < 1e-5
    _assert_core_weights(st, e1, q, ref_e, ref_q, ref_mu)
    ref_rho = np.zeros(st.grid.npts)
    ref_eps = unpack_states(st, ref_e)
    for f in range(nf):
        occ = fermi.occupation(ref_eps[f], ref_mu, st.kT)
        ref_rho[sq[f][1]] = np.einsum("i,ip->p", 2.0 * occ, sq[f][0])
    assert np.sum(np.abs(rho - ref_rho)) < 1e-5 * np.sum(np.abs(ref_rho))


def test_mixed_pass_si512_sampled_fragments():
    """The Si512 cell (512 fragments, 1536 Gram items of 4096 points over the persistent CTAs): the
    eigenvalues and core weights of sampled fragments against the oracle; the electron count of the
    whole-cell Fermi level and density as properties."""
    from paper_2606_21125_b300 import DCSolver
    cfg = workloads.make_config("si512", precision="mixed")
    sample = [0, 219, 511]
    st = oracle_state(cfg, subset=sample)
    V = st.veff(st.rho_in)
    st.initial_rr(V)
    st.solve(V, WARM)
    for f in sample:
        st.psi[f] = st.psi[f].astype(np.float32).astype(np.float64)
    with DCSolver(cfg) as s:
        s.set_tuning("fp32", 4, 256, 1)
        s.warmup()  # every fragment gets a warm state; the sampled ones are replaced below
        s.set_potential(torch.tensor(V.reshape(-1), dtype=torch.float64, device="cuda"))
        psi, eps = s.get_state()
        fr = s.maps()["frag"]
        per = [int(np.prod(fr[f, 3:6])) * int(fr[f, 9]) for f in range(fr.shape[0])]
        poff = np.concatenate([[0], np.cumsum(per)])
        soff = np.concatenate([[0], np.cumsum(fr[:, 9])])
        for f in sample:
            psi[poff[f]:poff[f + 1]] = torch.from_numpy(st.psi[f].reshape(-1).astype(np.float32)).cuda()
            eps[soff[f]:soff[f + 1]] = torch.from_numpy(st.eps[f]).cuda()
        s.set_state(psi, eps)
        s.chefsi(1)
        _, e1 = s.get_state()
        rho, q, mu = s.density()
        e1, q, mu, rho = e1.cpu().numpy(), q.cpu().numpy(), float(mu.item()), rho.cpu().numpy()
    from oracle import density
    st.solve(V, 1)
    for f in sample:
        a, b = soff[f], soff[f + 1]
        assert np.max(np.abs(e1[a:b] - st.eps[f])) < 1e-5, f
        ref_q = density.core_weights(st.frags, f, st.psi[f], st.grid.dV)
        tol = 1e-5 * np.max(ref_q)
        for ca, cb in _clusters(st.eps[f], 1e-2):
            assert abs(np.sum(q[a + ca:a + cb]) - np.sum(ref_q[ca:cb])) < tol * (cb - ca), (f, ca, cb)
    # the chemical potential fixes the electron count (Eq. 4) and the density integrates to it
    assert abs(float(np.sum(2.0 * fermi.occupation(e1, mu, st.kT) * q)) - st.ne) < 1e-8 * st.ne
    assert np.min(rho) >= 0.0
    assert abs(st.grid.dV * float(np.sum(rho)) - st.ne) < 1e-8 * st.ne
