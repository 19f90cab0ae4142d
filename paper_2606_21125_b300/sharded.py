"""Fragment-sharded DC-DFT SCF step over several ranks (Sec. 2.2; Sec. 2.5 distributes fragments over
processes).

Fragments are independent inside an SCF iteration; they couple only through the global chemical
potential (the electron count sums over every fragment's core weights) and through the global density,
from which every rank rebuilds the same potential.  Each rank therefore owns a contiguous range of
fragment ids (z-major slabs of the fragment grid), balanced by the stencil work P_f n_f, and a step has
exactly two exchanges:

1. the (eps, q) pairs of all states: each rank fills its own states and leaves zeros elsewhere, so an
   all-reduce sum assembles the global arrays bit for bit; every rank then runs the same Fermi solve;
2. the density: each rank writes rho_out on its own cores (zeros elsewhere; the cores partition the
   cell), so a second all-reduce sum gives the global rho_out; every rank then runs the same energy,
   residual and mixing.

With one rank the step equals the single-context step bit for bit.  ``ShardedStep`` is written against
two small interfaces so that the same driver runs the native library on GPUs (``DCSolver`` and NCCL
all-reduce) and any other implementation of the three per-rank calls.
"""
from __future__ import annotations


def shard_range(cost, rank, nranks):
    """Fragment range [lo, hi) of ``rank`` of ``nranks`` for per-fragment costs ``cost`` (integers).

    Boundary b_r (0 < r < nranks) is the first fragment f whose cost prefix sum_{f' < f} cost satisfies
    prefix * nranks >= r * total, clamped to at least b_{r-1} + 1 and at most F - (nranks - r), so every
    rank owns at least one fragment.  The native library applies the same integer rule.
    """
    F = len(cost)
    if not 1 <= nranks <= F or not 0 <= rank < nranks:
        raise ValueError("need 0 <= rank < nranks <= number of fragments")
    total = sum(int(c) for c in cost)
    bounds = [0]
    f, prefix = 0, 0
    for r in range(1, nranks):
        while f < F and prefix * nranks < r * total:
            prefix += int(cost[f])
            f += 1
        b = max(f, bounds[-1] + 1)
        b = min(b, F - (nranks - r))
        bounds.append(b)
    bounds.append(F)
    return bounds[rank], bounds[rank + 1]


class ShardedStep:
    """One rank's side of the sharded SCF step.

    ``local`` provides the three per-rank calls of the native library (``DCSolver`` does):
      step_local(rho_in, eps, q)              -- potential, own fragments' CheFSI passes and core weights;
                                                eps/q filled for own states, zero elsewhere
      step_density(eps, q, rho_part, mu)      -- mu from all states, rho_out on own cores, zero elsewhere
      step_finish(rho_in, rho_out) -> stats   -- energies, residual, mixing of rho_in in place
    ``allreduce_sum(t)`` sums tensor ``t`` over all ranks in place.  ``zeros(n)`` returns a float64
    tensor of n zeros on the ranks' device.
    """

    def __init__(self, local, allreduce_sum, nstates, npts, zeros):
        self.local = local
        self.allreduce_sum = allreduce_sum
        self.eps = zeros(nstates)
        self.q = zeros(nstates)
        self.rho_part = zeros(npts)
        self.mu = zeros(1)

    def step(self, rho_in):
        """One SCF step; ``rho_in`` (global, identical on every rank) is mixed in place.  Returns the
        step statistics (identical on every rank) and leaves the global rho_out in ``self.rho_part``."""
        self.local.step_local(rho_in, self.eps, self.q)
        self.allreduce_sum(self.eps)
        self.allreduce_sum(self.q)
        self.local.step_density(self.eps, self.q, self.rho_part, self.mu)
        self.allreduce_sum(self.rho_part)
        return self.local.step_finish(rho_in, self.rho_part)


def fragment_costs(layout_frag):
    """P_f n_f per fragment from the ``frag`` table of ``DCSolver.maps()`` (extents in columns 3-5,
    orbital count in column 9)."""
    return [int(r[3]) * int(r[4]) * int(r[5]) * int(r[9]) for r in layout_frag]


class ShardedSolver:
    """A ``DCSolver`` that owns this rank's fragment shard, stepped with NCCL (or any torch.distributed
    backend) all-reduce sums.  ``cfg`` as for ``DCSolver``; rank and world size come from
    ``torch.distributed`` (initialised by the caller)."""

    def __init__(self, cfg, group=None):
        import torch
        import torch.distributed as dist

        from . import DCSolver
        self.rank = dist.get_rank(group)
        self.nranks = dist.get_world_size(group)
        self.solver = DCSolver(dict(cfg, rank=self.rank, nranks=self.nranks))
        dev = torch.device("cuda", torch.cuda.current_device())
        lay = self.solver.layout

        def allreduce(t):
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)

        self.step_driver = ShardedStep(self.solver, allreduce, int(lay.nstates), int(lay.npts),
                                       lambda n: torch.zeros(n, dtype=torch.float64, device=dev))

    @property
    def fragments(self):
        lay = self.solver.layout
        return int(lay.frag_lo), int(lay.frag_hi)

    def warmup(self):
        self.solver.warmup()

    def scf_step(self, rho_in):
        return self.step_driver.step(rho_in)

    def close(self):
        self.solver.close()
