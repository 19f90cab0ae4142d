"""The fragment-sharded SCF step (Sec. 2.2; Sec. 2.5 distributes fragments over processes) on CPU.

Two gloo ranks drive ``paper_2606_21125_b300.sharded.ShardedStep`` (the product's exchange protocol:
all-reduce sums of the zero-padded (eps, q) arrays and of the per-rank core densities) with the FP64
oracle as the per-rank fragment solver.  Every step's chemical potential, rho_out, energy and mixed
density must equal the single-process oracle step bit for bit, and the shard boundaries must follow
the partition rule.  The native library's side of the same protocol runs on one GPU in
``tests/test_gpu_sharded.py``.
"""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")

STEPS = 2


def _cfg():
    import workloads
    return workloads.small_config(n=(14, 12, 12), L=(8.0, 7.0, 7.0), num_fragment=(3, 2, 2), buffer=(2, 2, 2),
                                  nstate=6, natom=4, seed=9, n_warmup=2, cheb_degree=6, kerker_q0=0.8)


class OracleShard:
    """The three per-rank calls of the sharded step, computed by the FP64 oracle on fragments [lo, hi)."""

    def __init__(self, cfg, lo, hi):
        from oracle import scf
        self.st = scf.DCState(cfg, fragments_subset=list(range(lo, hi)))
        self.st.warmup()
        self.off = np.concatenate([[0], np.cumsum(self.st.norb)]).astype(np.int64)

    def step_local(self, rho_in, eps, q):
        from oracle import density
        st = self.st
        self.V = st.veff(rho_in.numpy().reshape(st.grid.shape()))
        st.solve(self.V, int(st.cfg["n_pass"]))
        eps.zero_()
        q.zero_()
        for f in st.active:
            a, b = self.off[f], self.off[f + 1]
            eps[a:b] = torch.from_numpy(st.eps[f])
            q[a:b] = torch.from_numpy(density.core_weights(st.frags, f, st.psi[f], st.grid.dV))

    def step_density(self, eps, q, rho_part, mu):
        from oracle import density, fermi
        st = self.st
        self.eps_all, self.q_all = eps.numpy().copy(), q.numpy().copy()
        self.mu = fermi.find_mu(self.eps_all, self.q_all, st.ne, st.kT)
        mu[0] = self.mu
        rho = np.zeros(st.grid.npts)
        for f in st.active:
            occ = fermi.occupation(st.eps[f], self.mu, st.kT)
            g, vals = density.core_density(st.frags, f, st.psi[f], occ)
            rho[g] = vals
        rho_part.copy_(torch.from_numpy(rho))

    def step_finish(self, rho_in, rho_out):
        from oracle import energy, fermi
        st = self.st
        rin = rho_in.numpy().reshape(st.grid.shape()).copy()
        rout = rho_out.numpy().reshape(st.grid.shape()).copy()
        occ_all = fermi.occupation(self.eps_all, self.mu, st.kT)
        eband = energy.band_sum(self.eps_all, self.q_all, occ_all)
        E = energy.total_energy(st.grid, st.hxc, eband, self.V, rout, st.rhoiG)
        S = fermi.entropy(self.eps_all, self.q_all, self.mu, st.kT)
        new = energy.mix(rin, rout, st.alpha, st.grid, float(st.cfg.get("kerker_q0", 0.0)))
        rho_in.copy_(torch.from_numpy(new.reshape(-1)))
        return dict(E=E, F=E - st.kT * S, mu=self.mu, drho=energy.residual(st.grid, rout, rin, st.ne))


def _rank(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2606_21125_b300.sharded import ShardedStep, shard_range
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        cfg = _cfg()
        from oracle import scf
        probe = scf.DCState(cfg, fragments_subset=[])
        ext = probe.frags.extent
        cost = [int(np.prod(ext[f])) * int(probe.norb[f]) for f in range(probe.frags.nfrag)]
        lo, hi = shard_range(cost, rank, ws)
        local = OracleShard(cfg, lo, hi)
        nst = int(np.sum(probe.norb))
        drv = ShardedStep(local, lambda t: dist.all_reduce(t, op=dist.ReduceOp.SUM), nst, probe.grid.npts,
                          lambda n: torch.zeros(n, dtype=torch.float64))
        rho = torch.from_numpy(probe.rho_in.reshape(-1).copy())
        res = []
        for _ in range(STEPS):
            s = drv.step(rho)
            res.append((s["E"], s["F"], s["mu"], s["drho"], drv.rho_part.numpy().copy(), rho.numpy().copy()))
        out.put((rank, (lo, hi), res))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_sharded_step_equals_single_process_step():
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    from oracle import scf
    cfg = _cfg()
    ref = scf.DCState(cfg)
    ref.warmup()
    want = [ref.scf_step() for _ in range(STEPS)]
    want_rho_in = ref.rho_in.reshape(-1)

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29700 + os.getpid() % 1000
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = [q.get(timeout=600) for _ in ps]
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    got.sort()
    (r0, rng0, res0), (r1, rng1, res1) = got
    assert rng0[0] == 0 and rng0[1] == rng1[0] and rng1[1] == 12 and rng0[1] > 0
    for res in (res0, res1):
        for k, (E, F, mu, drho, rho_out, rho_in) in enumerate(res):
            assert E == want[k]["E"] and F == want[k]["F"] and mu == want[k]["mu"] and drho == want[k]["drho"], k
            assert np.array_equal(rho_out, want[k]["rho_out"].reshape(-1)), k
        assert np.array_equal(res[-1][5], want_rho_in)


def test_shard_range_rule():
    from paper_2606_21125_b300.sharded import shard_range
    cost = [5, 5, 5, 5]
    assert [shard_range(cost, r, 2) for r in range(2)] == [(0, 2), (2, 4)]
    assert [shard_range(cost, r, 4) for r in range(4)] == [(0, 1), (1, 2), (2, 3), (3, 4)]
    # a dominant fragment still leaves every rank one fragment
    cost = [1, 100, 1]
    assert [shard_range(cost, r, 3) for r in range(3)] == [(0, 1), (1, 2), (2, 3)]
    # balance by work: the heavy tail goes to its own rank
    cost = [1] * 8 + [8]
    assert [shard_range(cost, r, 2) for r in range(2)] == [(0, 8), (8, 9)]
    r = np.random.default_rng(1)
    for _ in range(200):
        F = int(r.integers(1, 40))
        n = int(r.integers(1, F + 1))
        cost = [int(c) for c in r.integers(0, 60, F)]
        parts = [shard_range(cost, k, n) for k in range(n)]
        assert parts[0][0] == 0 and parts[-1][1] == F
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
        assert all(hi > lo for lo, hi in parts)
    with pytest.raises(ValueError):
        shard_range([1, 1], 0, 3)
