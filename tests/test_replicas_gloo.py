"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas, no data-path collective).

bench.py runs one independent replica per GPU; the only cross-rank work is a barrier and the max of
each rank's timed region, from which rank 0 reports ws * steps / max.  Here two CPU processes take
that reduction through gloo with different per-rank times, and the reference arm, launched by
torchrun with two ranks, prints exactly one JSON line (rank 0's).
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _rank(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        secs = [0.25, 0.75][rank]
        slowest, value = bench.whole_job(secs, ws, 10, dist, "cpu")
        dist.barrier()
        out.put((rank, slowest, value))
    finally:
        dist.destroy_process_group()


def test_whole_job_takes_the_slowest_rank_over_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, value in res:
        assert slowest == 0.75
        assert value == pytest.approx(2 * 10 / 0.75)


def test_whole_job_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job(0.5, 1, 4, None, "cpu") == (0.5, 8.0)


def test_reference_arm_under_torchrun_prints_once():
    port = 30500 + os.getpid() % 1000
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--workload", "si8", "--steps", "1", "--warmup", "0",
           "--sample-frags", "1"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2
