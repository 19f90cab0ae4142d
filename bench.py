"""Benchmark of one DC-DFT SCF step (the whole batched fragment Kohn-Sham solve) on one B300.

A step is one pass of every stage of the path over the Si512 workload (80^3 grid, 8^3 fragments of
10^3 core + 6-point buffers = 22^3 points, 48 orbitals each, 512 atoms): potential (Poisson +
exchange), gather, Chebyshev filter (degree 10) with the fused stencil H-apply, Gram and
Rayleigh-Ritz, FP64 subspace solves, rotation, core weights, Fermi level, density, energies and
mixing.  The orbital block (1.05 GB in FP32) is larger than L2, so no L2 flush is needed between
steps.

Output: one JSON line (rank 0).  ``value`` is SCF steps per second summed over ranks (each rank runs
its own replica: weak scaling, no collective on the data path), timed with CUDA events over K steps
with no per-stage events; a second pass of K steps with per-stage events gives the stage split and the
stencil's launch durations for the roofline.  ``--impl reference`` times the FP64 CPU oracle on the
host's cores (fragments in parallel processes) on a bounded, stride-chosen sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SCF-step time and Hψ HBM GB/s vs peak, mixed vs FP64 at ≤1e-6 Ha/atom"
WORKLOAD_TEXT = {
    "si512": "Si512 a-Si-like (4^3 diamond supercell, a=41.04 bohr, N(0,0.3) displacements), 80^3 grid, "
             "8^3 fragments of 10^3 core + 6-point buffer (22^3), 48 orbitals each",
    "si64": "Si64 (2^3 supercell), 40^3 grid, 4^3 fragments of 10^3 core + 5 (20^3), 32 orbitals",
    "si8": "Si8 diamond cell, 20^3 grid, 2^3 fragments of 10^3 core + 4 (18^3), 24 orbitals",
    "si_weak64": "Si64 weak-scaling cell (2^3 supercell, N(0,0.3)), 40^3 grid, 4^3 fragments of 10^3 core + 6 "
                 "(22^3), 48 orbitals",
    "si_weak4096": "Si4096 weak-scaling cell (8^3 supercell, N(0,0.3)), 160^3 grid, 16^3 fragments of 10^3 core + 6 "
                   "(22^3), 48 orbitals",
    "water": "water-like liquid, 1378 rigid H2O at 1 g/cm^3 (random sequential addition, O-O >= 2.5 A) in a 65.6 "
             "bohr box, 192^3 grid, 12^3 fragments of 16^3 core + 8 (32^3), orbitals from each fragment's electrons",
}


def _metric():
    """The benchmark's metric: SCF-step time and the stencil's HBM bandwidth against the measured peak,
    mixed precision against FP64 at an energy difference of at most 1e-6 Ha/atom."""
    return METRIC


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=40)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="si512", choices=sorted(WORKLOAD_TEXT))
    p.add_argument("--precision", default="mixed", choices=["fp32", "fp64", "mixed"],
                   help="mixed (default): FP32 stencil, 3xBF16 tensor-core Gram, FP64 subspace and Fermi level")
    p.add_argument("--sample-frags", type=int, default=0,
                   help="fragments in the oracle's timed sample (0: every fragment for cpu_baseline up to 512 "
                        "fragments, two per host process for --impl reference)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-compare", action="store_true", help="skip the FP64 comparison run")
    p.add_argument("--shape", default=None,
                   help="pin the FP32 stencil launch shape 'kind,threads,pairs' instead of autotuning")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.file,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and "Active" in r[5 + k] and "Not" not in r[5 + k]:
                    reasons.add(nm)
        if not sm:
            return None
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), samples=len(sm), reasons=sorted(reasons))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return dict(hbm_gbs=6400.0, bf16_tflops=1800.0, bf16_tflops_sustained=1400.0), "fallback"


def kernel_traffic(kernel_file, point_orbitals, extent):
    """DRAM traffic per launch of the dominant kernel from a committed ncu capture, scaled to this
    workload's point-orbitals when its fragments have the captured extent; None (with the reason) when
    the kernel source changed since the capture or the fragment shape differs."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)[kernel_file]
        src = open(os.path.join(ROOT, "paper_2606_21125_b300", "csrc", kernel_file), "rb").read()
        if rec.get("sha256") != hashlib.sha256(src).hexdigest():
            return None, "kernel changed since the ncu capture"
        if int(rec["fragment_extent"]) != int(extent):
            return None, f"captured on {rec['fragment_extent']}^3 fragments, not {extent}^3"
        scale = point_orbitals / float(rec["point_orbitals_per_launch"])
        return rec["bytes_per_launch"] * scale, (f"ncu DRAM bytes of one launch on {rec['workload']} "
                                                 f"({rec['profile']}), scaled x{scale:g} by point-orbitals")
    except (OSError, KeyError, ValueError, TypeError):
        return None, "no ncu capture"


# ------------------------------------------------------------------------------------------------
# CPU oracle on a bounded sample (cpu_baseline and --impl reference)
# ------------------------------------------------------------------------------------------------
class OracleRun:
    """The FP64 oracle's SCF step on the host's cores.

    Fragments are solved by ``oracle.pool.FragmentPool`` (one spawn process per core, one BLAS thread
    each); the global stages (V_eff by FFT Poisson + exchange, Fermi level, energy, residual, mixing) run
    in this process.  ``sample=None`` runs every fragment; otherwise ``sample`` stride-chosen fragments
    run and the fragment-parallel part of the step is scaled by F / sample (labelled extrapolated).
    The starting Rayleigh-Ritz of each fragment is set-up, not timed.
    """

    def __init__(self, cfg, sample=None, nproc=None):
        from oracle import scf
        from oracle.pool import FragmentPool
        self.cfg = cfg
        nf = int(cfg["num_fragment"][0] * cfg["num_fragment"][1] * cfg["num_fragment"][2])
        self.nf = nf
        if sample is None or sample >= nf:
            self.frags = list(range(nf))
        else:
            k = max(1, int(sample))
            self.frags = sorted(set(int(round(i * nf / k)) % nf for i in range(k)))
        self.scale = nf / len(self.frags)
        self.st = scf.DCState(cfg, fragments_subset=[])  # global arrays only
        self.ne = self.st.ne / self.scale  # electrons of the sampled fragments, so that mu stays in range
        self.pool = FragmentPool(cfg, self.frags, nproc)
        self.pool.initial_rr(self.st.veff(self.st.rho_in))

    def step(self):
        import numpy as np
        from oracle import energy, fermi
        st = self.st
        t0 = time.perf_counter()
        V = st.veff(st.rho_in)
        t1 = time.perf_counter()
        res = self.pool.solve(V, int(self.cfg["n_pass"]))
        t2 = time.perf_counter()
        eps_all = np.concatenate([res[f][0] for f in self.frags])
        q_all = np.concatenate([res[f][1] for f in self.frags])
        mu = fermi.find_mu(eps_all, q_all, self.ne, st.kT)
        t3 = time.perf_counter()
        dens = self.pool.core_density(mu)
        t4 = time.perf_counter()
        rho = np.zeros(st.grid.npts)
        for f in self.frags:
            rho[dens[f][0]] = dens[f][1]
        rho = rho.reshape(st.grid.shape())
        occ_all = fermi.occupation(eps_all, mu, st.kT)
        eb = energy.band_sum(eps_all, q_all, occ_all)
        energy.total_energy(st.grid, st.hxc, eb, V, rho, st.rhoiG)
        fermi.entropy(eps_all, q_all, mu, st.kT)
        energy.residual(st.grid, rho, st.rho_in, st.ne)
        energy.mix(st.rho_in, rho, 0.0)  # alpha 0: the timed input stays the same from step to step
        t5 = time.perf_counter()
        return (t1 - t0) + (t3 - t2) + (t5 - t4) + ((t2 - t1) + (t4 - t3)) * self.scale

    @property
    def cores(self):
        return self.pool.nproc

    def describe(self):
        base = (f"FP64 oracle on {self.pool.nproc} host processes (one BLAS thread each; host has {os.cpu_count()} "
                f"cores): fragments solved in parallel, global stages (Poisson/exchange, Fermi, density assembly, "
                f"energy, mixing) in the parent")
        if self.scale == 1.0:
            return base + f"; whole workload, all {self.nf} fragments"
        return (base + f"; extrapolated: {len(self.frags)} of {self.nf} fragments (stride-chosen), the fragment-"
                f"parallel part scaled x{self.scale:g}")

    def close(self):
        self.pool.close()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import workloads
    cfg = workloads.make_config(args.workload, precision="fp64")
    nproc = os.cpu_count() or 1
    # a bounded sample per step (about two fragments per process) keeps K + W steps within minutes
    samp = OracleRun(cfg, sample=args.sample_frags or 2 * nproc, nproc=nproc)
    for _ in range(args.warmup):
        samp.step()
    ts = [samp.step() for _ in range(args.steps)]
    samp.close()
    sec = sum(ts) / len(ts)
    val = 1.0 / sec
    line = dict(impl="reference", metric=_metric(), value=val, unit="SCF steps/s", n_gpus=args.gpus,
                steps=args.steps, warmup=args.warmup, ms_per_step=sec * 1e3, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=WORKLOAD_TEXT[args.workload], precision="fp64 (oracle)"),
                cpu_baseline=dict(value=val, unit="SCF steps/s", cores=samp.cores, host_cores=os.cpu_count(),
                                  kind="oracle", sample=samp.describe()),
                e2e=dict(value=val, unit="SCF steps/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------------
def whole_job(seconds, ws, steps, dist, device):
    """Replicas timing: the slowest rank's time for the timed steps (max over ranks) and the whole-job
    throughput ws * steps / that time.  dist is torch.distributed (or None for one rank); the
    reduction tensor lives on `device` ("cuda" under NCCL, "cpu" under gloo)."""
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    slowest = float(t.item())
    return slowest, ws * steps / slowest


HARTREE_EV = 27.211386245988  # eV per hartree (CODATA 2018)
FP64_NOMINAL_TFLOPS = 1.25    # B300 FP64 dense, nominal; bench replaces it with the measured FMA rate


def lcfo_measure(solver, mu, stream, reps=5):
    """Time dc_lcfo_basis on the solver's current orbitals with eps_cut = mu + 0.1 eV and
    lambda_cut = 1e-7 (the paper's validation values) and count its FP64 FMAs exactly:
    per fragment n_sel (n_sel + 1) / 2 |core| for the overlap and m n_sel |core| for the basis."""
    import numpy as np
    import torch
    psi, eps = solver.get_state()
    ecut = mu + 0.1 / HARTREE_EV
    res = solver.lcfo_basis(psi, eps, ecut, 1e-7)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        res = solver.lcfo_basis(psi, eps, ecut, 1e-7)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    fr = solver.maps()["frag"]
    eps_h = eps.cpu().numpy()
    nb = res[1].cpu().numpy()
    fma, so = 0, 0
    for f in range(fr.shape[0]):
        n, ncore = int(fr[f, 9]), int(np.prod(fr[f, 6:9]))
        nsel = int(np.count_nonzero(eps_h[so:so + n] < ecut))
        fma += (nsel * (nsel + 1) // 2 + int(nb[f]) * nsel) * ncore
        so += n
    tflops = 2.0 * fma / (ms * 1e-3) / 1e12
    return dict(ms=ms, eps_cut_minus_mu_eV=0.1, lambda_cut=1e-7, nbasis_total=int(nb.sum()),
                nbasis_per_fragment=[int(nb.min()), int(nb.max())],
                roofline=dict(bound="alu", achieved=tflops, peak=FP64_NOMINAL_TFLOPS, unit="TFLOP/s (FP64)",
                              frac=tflops / FP64_NOMINAL_TFLOPS, peak_kind="nominal FP64 (no measured FP64 peak)",
                              fp64_fma_per_launch=fma))


def fp64_peak(stream, reps=3):
    """Measured FP64 FMA rate of this device (TFLOP/s, 2 flops per FMA): the library's FMA-chain probe,
    one full wave of CTAs, timed with CUDA events on the launching stream (best of ``reps``)."""
    import ctypes as C

    import torch

    from paper_2606_21125_b300 import _lib, load
    lib = load()
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    fmas = C.c_int64(0)
    iters = 1 << 16
    best = float("inf")
    sptr = C.c_void_p(stream.cuda_stream)
    _lib.check("dc_fp64_fma_probe", lib.dc_fp64_fma_probe(iters // 16, C.c_void_p(sink.data_ptr()),
                                                          C.byref(fmas), sptr))
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _lib.check("dc_fp64_fma_probe", lib.dc_fp64_fma_probe(iters, C.c_void_p(sink.data_ptr()), C.byref(fmas),
                                                              sptr))
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return 2.0 * fmas.value / (best * 1e-3) / 1e12


def hpsi_measure(solver, stream, reps=10):
    """dc_hpsi alone (the H-apply of every fragment and orbital of the state block: projections
    <p|psi>, then the stencil + local + nonlocal kernel), timed with CUDA events over ``reps`` calls.
    Algorithmic bytes per call: the projection pass reads the block once; the H-apply reads the block
    and V_f and writes H psi.  The block (1.05 GB on Si512) exceeds L2, so no flush is needed."""
    import torch
    psi, _ = solver.get_state()
    out = torch.empty_like(psi)
    solver.hpsi(psi, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        solver.hpsi(psi, out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    es = psi.element_size()
    lay = solver.layout
    by = es * (3.0 * lay.psi_elems + lay.frag_points)
    return dict(ms=ms, bytes=by, gbs=by / (ms * 1e-3) / 1e9,
                note="read psi (projections) + read psi, V_f and write H psi (stencil), per call")


def run_ours(args):
    import numpy as np
    import torch

    import workloads
    from paper_2606_21125_b300 import DCSolver

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    cfg = workloads.make_config(args.workload, precision=args.precision)
    solver = DCSolver(cfg)
    if args.shape:
        kind, threads, pairs = (int(v) for v in args.shape.split(","))
        if not solver.set_tuning("fp64" if args.precision == "fp64" else "fp32", kind, threads, pairs):
            raise SystemExit(f"--shape {args.shape} does not fit this workload")
    t0 = time.perf_counter()
    solver.warmup()
    torch.cuda.synchronize()
    init_s = time.perf_counter() - t0
    _, rho0 = solver.initial()
    rho = rho0.clone()
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        solver.scf_step(rho)
    torch.cuda.synchronize()

    # ---- timed region: K SCF steps with inputs resident in HBM, no stage events ----
    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stats = None
    for _ in range(args.steps):
        stats = solver.scf_step(rho)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    ms_max, value = whole_job(ms * 1e-3, ws, args.steps, dist, "cuda")
    ms_max *= 1e3
    ms_step = ms_max / args.steps

    # ---- the same K steps again with CUDA events around every stage (stage split and the stencil's
    # launch durations for the roofline); this pass is not the headline ----
    solver.profile(True)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    pstats = None
    for _ in range(args.steps):
        pstats = solver.scf_step(rho)
    p1.record(stream)
    torch.cuda.synchronize()
    prof = solver.profile_read()
    solver.profile(False)
    prof_ms_step = p0.elapsed_time(p1) / args.steps
    steps_done = args.warmup + 2 * args.steps

    # ---- the same steps in plain FP64: step time and energy difference per atom ----
    compare = None
    if args.precision != "fp64" and not args.no_compare:
        ref = DCSolver(workloads.make_config(args.workload, precision="fp64"))
        ref.warmup()
        _, r64 = ref.initial()
        r64 = r64.clone()
        for _ in range(args.warmup + args.steps):
            ref.scf_step(r64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s64 = None
        for _ in range(args.steps):
            s64 = ref.scf_step(r64)
        e1.record(stream)
        torch.cuda.synchronize()
        natom = len(cfg["pos"])
        compare = dict(precision="fp64", ms_per_step=e0.elapsed_time(e1) / args.steps,
                       speedup=(e0.elapsed_time(e1) / args.steps) / ms_step,
                       dE_per_atom=abs(pstats["E"] - s64["E"]) / natom, dmu=abs(pstats["mu"] - s64["mu"]),
                       steps_compared=steps_done)
        ref.close()

    # ---- end to end through the public API with host buffers (H2D rho_in, D2H rho + stats) ----
    host = torch.empty(solver.layout.npts, dtype=torch.float64, pin_memory=True)
    host.copy_(rho.cpu())
    hnp = host.numpy()
    solver.scf_step(hnp)
    barrier()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(args.steps):
        solver.scf_step(hnp)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - w0
    _, e2e_val = whole_job(e2e_s, ws, args.steps, dist, "cuda")
    nb = 8 * solver.layout.npts

    # ---- H psi alone, the DC-LCFO basis step, the measured FP64 rate (after the timed region) ----
    hpsi_line = hpsi_measure(solver, stream)
    lcfo_line = lcfo_measure(solver, stats["mu"], stream)
    fp64 = fp64_peak(stream)
    lcfo_line["roofline"].update(peak=fp64, frac=lcfo_line["roofline"]["achieved"] / fp64,
                                 peak_kind="measured FP64 FMA rate (dc_fp64_fma_probe, CUDA events)")

    # ---- roofline of the dominant kernel (stencil H-apply, its launches in the profiled pass) ----
    peaks, peak_kind = measured_peaks()
    tun = solver.tuning()["fp64" if args.precision == "fp64" else "fp32"]
    stencil_name = STENCIL_KINDS.get(tun["kind"], f"kind {tun['kind']}")
    stencil_name += f", {tun['threads']} threads x {tun['pairs']} point pairs"
    h = prof["hpsi"]
    achieved = h["bytes"] / (h["ms"] * 1e-3) / 1e9 if h["ms"] > 0 else 0.0
    fr = solver.maps()["frag"]
    extent = int(fr[0, 3]) if (fr[:, 3:6] == fr[0, 3]).all() else -1
    traffic, traffic_note = kernel_traffic("k_cheb.cu" if tun["kind"] == 4 else "k_hamiltonian.cu",
                                           float(solver.layout.psi_elems), extent)
    per_launch_bytes = h["bytes"] / max(1, h["launches"])
    launches = sum(v["launches"] for v in prof.values())

    line = dict(metric=_metric(), value=value, unit="SCF steps/s", n_gpus=ws, steps=args.steps,
                warmup=args.warmup, ms_per_step=ms_step, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype={"fp32": "f32", "fp64": "f64", "mixed": "f32+bf16x3"}[args.precision],
                data="synthetic",
                config=dict(workload=WORKLOAD_TEXT[args.workload], precision=args.precision,
                            subspace_dtype="f64", cheb_degree=cfg["cheb_degree"], n_pass=cfg["n_pass"],
                            l2="orbital block larger than L2 (no flush needed)",
                            parallelism=f"replicas x{ws}" if ws > 1 else "single GPU"),
                roofline=dict(kernel=stencil_name,
                              bound="hbm", achieved=achieved, peak=peaks["hbm_gbs"], unit="GB/s",
                              frac=achieved / peaks["hbm_gbs"], peak_kind=peak_kind + " (hbm_gbs)",
                              traffic=traffic, traffic_note=traffic_note,
                              algorithmic_bytes_per_launch=per_launch_bytes, launches=h["launches"],
                              avg_launch_ms=h["ms"] / max(1, h["launches"]),
                              timing="CUDA events around each stencil launch in a second pass of the same K "
                                     "steps (the headline pass runs without events)"),
                stages_ms_per_step={k: v["ms"] / args.steps for k, v in prof.items()},
                profiled_pass_ms_per_step=prof_ms_step,
                hpsi=hpsi_line,
                e2e=dict(value=e2e_val, unit="SCF steps/s", h2d_bytes_per_step=nb, d2h_bytes_per_step=nb + 8 * 16),
                gpu_launches=launches, launches_counted="this library's kernels per profiled pass of K steps",
                init_s=init_s, fp64_compare=compare, lcfo=lcfo_line,
                fp64_measured_tflops=fp64,
                last_step=dict(E_per_atom=stats["E"] / len(cfg["pos"]), mu=stats["mu"], drho=stats["drho"]),
                clocks=clocks)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        ocfg = workloads.make_config(args.workload, precision="fp64")
        nf = int(np.prod(ocfg["num_fragment"]))
        nproc = os.cpu_count() or 1
        sample = args.sample_frags or (None if nf <= 512 else 16 * nproc)
        samp = OracleRun(ocfg, sample=sample, nproc=nproc)
        sec = samp.step()
        line["cpu_baseline"] = dict(value=1.0 / sec, unit="SCF steps/s", cores=samp.cores,
                                    host_cores=os.cpu_count(), kind="oracle", sample=samp.describe(),
                                    seconds_per_step=sec)
        samp.close()
    solver.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


STENCIL_KINDS = {
    0: "k_hstep (stencil + local + nonlocal H-apply, fused Chebyshev step)",
    1: "k_hpair (orbital-pair FP32 stencil + local + nonlocal H-apply, fused Chebyshev step)",
    2: "k_hpair (orbital-pair FP32 stencil, fused Chebyshev step), register-capped",
    3: "k_hpair (orbital-pair FP32 stencil, fused Chebyshev step), every projector record of a fragment staged once",
    4: "k_cheb (orbital-pair FP32 stencil compiled for one cubic fragment extent, planes streamed through a "
       "shared-memory ring by bulk async copies, fused Chebyshev step)",
}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
