"""The library's side of the fragment-sharded SCF step (Sec. 2.5), on one GPU.

Two contexts own the two fragment shards of one system (rank 0 and 1 of 2).  They run one after the
other on the same GPU: no kernel of one waits for the other, and the two exchanges of the step (sums of
the zero-padded (eps, q) arrays and of the per-rank core densities) are plain tensor additions in
between, standing in for the all-reduce.  Every step must equal the single-context ``dc_scf_step`` bit
for bit, and the shard ranges must follow ``sharded.shard_range``.
"""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cfg(precision):
    return workloads.small_config(n=(21, 13, 16), L=(11.0, 7.0, 8.5), num_fragment=(2, 3, 2), buffer=(3, 2, 2),
                                  nstate=8, natom=6, seed=3, n_warmup=3, precision=precision, kerker_q0=0.8)


class _Emulated:
    """The per-rank calls of every shard, with the exchanges done as tensor sums."""

    def __init__(self, shards):
        self.shards = shards

    def step(self, rho_in):
        lay = self.shards[0].layout
        parts = [dict(eps=torch.empty(lay.nstates, dtype=torch.float64, device="cuda"),
                      q=torch.empty(lay.nstates, dtype=torch.float64, device="cuda"),
                      rho=torch.empty(lay.npts, dtype=torch.float64, device="cuda"),
                      rin=rho_in.clone()) for _ in self.shards]
        for s, p in zip(self.shards, parts):
            s.step_local(p["rin"], p["eps"], p["q"])
        eps = sum(p["eps"] for p in parts)
        q = sum(p["q"] for p in parts)
        for s, p in zip(self.shards, parts):
            s.step_density(eps, q, p["rho"])
        rho_out = sum(p["rho"] for p in parts)
        stats = [s.step_finish(p["rin"], rho_out) for s, p in zip(self.shards, parts)]
        for p in parts[1:]:
            assert torch.equal(p["rin"], parts[0]["rin"])
        rho_in.copy_(parts[0]["rin"])
        return stats, rho_out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_two_shards_equal_one_context(precision):
    from paper_2606_21125_b300 import DCSolver
    from paper_2606_21125_b300.sharded import fragment_costs, shard_range
    cfg = _cfg(precision)
    shape = (0, 256, 1) if precision == "fp64" else (1, 256, 1)
    dt = "fp64" if precision == "fp64" else "fp32"
    with DCSolver(cfg) as one:
        one.set_tuning(dt, *shape)
        one.set_tuning("fp64", 0, 256, 1)
        costs = fragment_costs(one.maps()["frag"])
        shards = [DCSolver(dict(cfg, rank=r, nranks=2)) for r in range(2)]
        try:
            for r, s in enumerate(shards):
                assert (s.layout.frag_lo, s.layout.frag_hi) == shard_range(costs, r, 2)
                s.set_tuning(dt, *shape)
                s.set_tuning("fp64", 0, 256, 1)
                s.warmup()
            one.warmup()
            _, rho1 = one.initial()
            rho1 = rho1.clone()
            rho2 = rho1.clone()
            emu = _Emulated(shards)
            for k in range(3):
                want = one.scf_step(rho1)
                got, rho_out = emu.step(rho2)
                for g in got:
                    for key in ("E", "F", "mu", "drho", "ne"):
                        assert g[key] == want[key], (k, key, g[key], want[key])
                assert torch.equal(rho_out, one.rho_out()), k
                assert torch.equal(rho2, rho1), k
        finally:
            for s in shards:
                s.close()


def test_shard_refuses_whole_system_calls():
    from paper_2606_21125_b300 import DCError, DCSolver
    cfg = _cfg("fp64")
    with DCSolver(dict(cfg, rank=1, nranks=2)) as s:
        s.warmup()
        _, rho = s.initial()
        with pytest.raises(DCError):
            s.scf_step(rho.clone())
    with pytest.raises(DCError):
        DCSolver(dict(cfg, rank=2, nranks=2))
