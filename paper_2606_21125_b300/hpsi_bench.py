"""H-apply micro-benchmark: dc_hpsi on every fragment and orbital of a workload.

Reports the achieved bandwidth of the stencil kernel as algorithmic bytes (read psi, write H psi,
read V_f once per fragment point) over CUDA-event time, with a buffer larger than L2 written
between repetitions.  The potential is a seeded synthetic one (no SCF needed).

    python -m paper_2606_21125_b300.hpsi_bench --workload si_weak64 --dtype fp32 --reps 20
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--workload", default="si_weak64")
    p.add_argument("--dtype", default="fp32", choices=["fp32", "fp64"])
    p.add_argument("--reps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--all-shapes", action="store_true", help="one line per launch shape that fits")
    args = p.parse_args()

    import numpy as np
    import torch

    import workloads
    from paper_2606_21125_b300 import DCSolver

    cfg = workloads.make_config(args.workload, precision=args.dtype)
    s = DCSolver(cfg)
    n = cfg["n"]
    g = np.random.default_rng(5)
    z, y, x = np.meshgrid(*[np.arange(n[d]) / n[d] for d in (2, 1, 0)], indexing="ij")
    V = -0.5 + 0.3 * np.cos(2 * np.pi * (x + 2 * y + z)) + 0.2 * np.sin(2 * np.pi * (3 * x - y))
    s.set_potential(torch.tensor(V.reshape(-1), dtype=torch.float64, device="cuda"))
    dt = torch.float64 if args.dtype == "fp64" else torch.float32
    psi = torch.tensor(g.standard_normal(s.layout.psi_elems), dtype=dt, device="cuda")
    out = torch.empty_like(psi)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    shapes = [None]
    if args.all_shapes:
        shapes = [(0, 128, 1), (0, 128, 2), (0, 256, 1), (0, 256, 2), (0, 512, 1), (0, 512, 2), (0, 512, 4),
                  (1, 128, 1), (1, 256, 1), (1, 512, 1), (1, 1024, 1), (1, 256, 2), (1, 512, 2), (2, 128, 1),
                  (2, 256, 1), (3, 256, 1)]
    for shape in shapes:
        if shape is not None and not s.set_tuning(args.dtype, *shape):
            continue
        for _ in range(args.warmup):
            s.hpsi(psi, out)
        torch.cuda.synchronize()
        s.profile(True)
        for _ in range(args.reps):
            flush.fill_(1.0)
            s.hpsi(psi, out)
        torch.cuda.synchronize()
        prof = s.profile_read()
        s.profile(False)
        h, pj = prof["hpsi"], prof["project"]
        res = dict(workload=args.workload, dtype=args.dtype, reps=args.reps, shape=shape,
                   point_orbitals=int(s.layout.psi_elems), hpsi_ms=h["ms"] / args.reps,
                   hpsi_gbs=h["bytes"] / (h["ms"] * 1e-3) / 1e9, project_ms=pj["ms"] / args.reps,
                   total_gbs=(h["bytes"] + pj["bytes"]) / ((h["ms"] + pj["ms"]) * 1e-3) / 1e9)
        print(json.dumps(res), flush=True)
    s.close()


if __name__ == "__main__":
    main()
