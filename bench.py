"""Benchmark: HDCG time-to-solution on one GB300 against plain red-black CG,
with the fine Mpc^dag Mpc hop kernels' achieved bandwidth against the HBM roofline.

One step = one full HDCG solve of H x = b to a true FP64 residual of ``tol``
(a Gaussian source; ``--nrhs`` of them together), inputs resident in HBM.  The
default workload is the physical-point-like lattice: 32^3 x 64, Ls 16 Moebius
(b 1.5, c 0.5), M5 1.8, m 0.001, links exp(i 0.45 H); three levels (4^4
blocks with Nvec 40, then 2^4 blocks of the coarse lattice with Nvec 24);
FP16 storage of the sloppy fine operator and the subspace, FP32 little Dirac
operator, FP32 outer operator, double-float (FP64-accurate) true residuals.
After the timed steps the workload's 12 spin-colour point sources are solved
once as a batch (``batched``: time per right-hand side against the single
solve).  The subspaces and coarse operators are built once before the timed
region (the paper reports set-up separately).  Inputs are larger than L2 (a
3.2 GB field per right-hand side) and L2 is flushed (a 512 MiB write) before
every timed step anyway.

Timed steps run with the library's event profiling off; the per-kernel
profile (hop launch times and bytes, solve phases) comes from one extra
solve after the timed region.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload NAME]
Under torchrun (N > 1) every rank solves its own replica (independent seed);
the timing is the max over ranks.  ``--impl reference`` times the FP64 CPU
oracle on the host cores (bounded sample, see ``cpu_sample_desc``).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic as sy  # noqa: E402

METRIC = "HDCG solve seconds vs plain CG at 1e-8 (1 GB300); fine Mpc†Mpc GB/s, %HBM peak"
DEFAULT_WORKLOAD = "cfg5_32x32x32x64_ls16_mobius_3lvl"
PREC = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3}

# Fine H applies (outer + preconditioner + FP64 residual) per right-hand side
# of one HDCG solve, from the GPU arm's solve statistics on each workload (a
# property of the algorithm on that input).  The reference arm, which runs no
# GPU code, scales the oracle's per-apply time by it; the GPU arm reports its
# measured count beside this figure (``h_applies_per_rhs``).
H_APPLIES_PER_RHS = {DEFAULT_WORKLOAD: 824, "cfg2_16x16x16x16_ls16_shamir": 140}

# DRAM bytes (read + write) per hop_kernel launch of the outer precision from
# one ncu capture of the current kernel, per workload; None once the kernel
# changes (the counters then no longer describe it).
HOP_TRAFFIC = {
    # ncu (dram__bytes_read.sum + dram__bytes_write.sum) of the four FP16 passes
    # of one H at this size (bench.py --apply-only 3, no fused CG epilogue),
    # averaged per launch: 2.19, 3.32, 2.14 and 3.33 GB for passes A-D
    DEFAULT_WORKLOAD: 2.745e9,
}


def hop_flops_per_site(w) -> int:
    """Floating-point operations of one H = Mpc^dag Mpc per 5D site (four hop
    passes), counted from the operator's structure: each pass does 8 hops of
    (spin projection 12 + two 3x3 complex matrix-vector products 144 +
    reconstruction 24) = 1440; M_ee^-1 by log2(Ls) shift-and-add steps is
    48 log2(Ls) + 24; K = b + c P_s is 72 for Moebius and 24 (a scale) for
    Shamir, and Moebius applies it to each of the 8 neighbours in pass A;
    the M_oo terms of passes B and D are 72 + 48, with 24 more for the output
    scale of pass D."""
    lg = (w.Ls - 1).bit_length()
    minv = 48 * lg + 24
    mob = w.c != 0.0
    k = 72 if mob else 24
    pass_a = 1440 + (8 * 72 if mob else 0) + minv + k
    pass_b = 1440 + 72 + 48
    pass_c = 1440 + k + minv
    pass_d = 1440 + k + 72 + 48 + 24
    return pass_a + pass_b + pass_c + pass_d


def operator_bytes_per_site(w, bytes_per_real: int) -> float:
    """Algorithmic bytes of one H per 5D site: four passes each read their input
    (24 reals) and write their output (24), read the links once per 4D site
    (8 x 18 reals shared by Ls sites), and passes B and D re-read psi for the
    M_oo term (24 each): (240 + 576 / Ls) reals."""
    return (240.0 + 576.0 / w.Ls) * bytes_per_real


def replica_seeds(w, rank: int) -> dict:
    """Seeds of rank `rank`'s replica: every rank solves its own independent
    problem of the workload (weak scaling, no data-path collective); rank 0
    uses the workload's own seeds."""
    return {"gauge": w.gauge_seed + 100 * rank, "source": w.source_seed + rank,
            "subspace": w.subspace_seed + rank, "ldop": w.subspace_seed + 7 + rank}


def max_over_ranks(value: float, world: int, device) -> float:
    """The largest per-rank value: the job's time per step when every rank
    solves its own replica (one all-reduce on the timing, outside the timed work)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def host_info():
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "cpu": model}


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline and --impl reference)
# ----------------------------------------------------------------------------
SAMPLE_DIMS = (8, 8, 8, 8)


def oracle_h_seconds_per_site(w, reps=1):
    """Seconds per 5D odd site of one FP64 oracle H = Mpc^dag Mpc apply, timed on
    an 8^4 lattice with the workload's Ls and action (the oracle's cost is
    linear in the volume)."""
    from oracle.dwf import DWF
    dims = SAMPLE_DIMS
    U = sy.gauge_field(dims, w.eps, w.gauge_seed)
    d = DWF(dims, w.Ls, w.M5, w.b, w.c, w.mass, U)
    psi = sy.gaussian_fermion(dims, w.Ls, w.source_seed)
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        d.mdagm(psi)
        ts.append(time.perf_counter() - t0)
    return min(ts) / (int(np.prod(dims)) // 2 * w.Ls)


def n5_of(w) -> int:
    return int(np.prod(w.dims)) // 2 * w.Ls


def cpu_sample_desc(w, n_h_per_rhs, nrhs):
    return (f"one FP64 oracle H apply on an {'x'.join(map(str, SAMPLE_DIMS))}x{w.Ls} lattice (same action), "
            f"scaled per 5D site to the {'x'.join(map(str, w.dims))}x{w.Ls} lattice and by the {n_h_per_rhs} fine H "
            f"applies per right-hand side of one HDCG solve, times {nrhs} right-hand sides; the oracle's "
            "coarse-grid work is not included")


def oracle_cg_solve_cfg1():
    """The oracle's own FP64 solve of the 8^4 x 8 Shamir workload (CG to its
    tolerance 1e-10): a complete oracle solve timed on the host cores."""
    from oracle.dwf import DWF
    from oracle.solvers import cg
    w = sy.WORKLOADS["cfg1_8x8x8x8_ls8_shamir"]
    d = DWF(w.dims, w.Ls, w.M5, w.b, w.c, w.mass, sy.gauge_field(w.dims, w.eps, w.gauge_seed))
    b = sy.gaussian_fermion(w.dims, w.Ls, w.source_seed)
    t0 = time.perf_counter()
    _, it = cg(d.mdagm, b, w.tol)
    return {"workload": w.name, "algorithm": "CG", "tol": w.tol, "iterations": int(it),
            "seconds": time.perf_counter() - t0, "cores": 1}


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(k, "1")
    nrhs = args.nrhs
    n_h = H_APPLIES_PER_RHS.get(w.name, 140)
    for _ in range(args.warmup):
        oracle_h_seconds_per_site(w)
    ts = [oracle_h_seconds_per_site(w) for _ in range(args.steps)]
    per_site = statistics.mean(ts)
    value = per_site * n5_of(w) * n_h * nrhs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "lattice": list(w.dims), "Ls": w.Ls, "tol": w.tol, "rhs_per_gpu": nrhs},
            "cpu_baseline": {"value": value, "unit": "s", "cores": 1, "kind": "oracle",
                             "sample": cpu_sample_desc(w, n_h, nrhs), **host_info()},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def build_levels(h, w, seeds, args):
    """Subspaces and coarse operators (timed separately, outside the solves)."""
    prec = PREC[w.prec]
    sub_prec = prec if prec in (0, 1) else 2
    cp = args.coarse_prec or w.coarse_prec
    coarse_prec = PREC[cp] if cp else (0 if prec == 0 else (1 if prec == 1 else 2))
    out = {}
    t0 = time.perf_counter()
    h.build_subspace(w.block, w.nvec, sub_prec, inv_steps=w.inv_steps, inv_shift=0.0, inv_tol=w.inv_tol,
                     inv_maxiter=w.inv_maxiter, seed=seeds["subspace"])
    out["subspace"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    h.build_coarse(coarse_prec)
    out["coarse_operator"] = time.perf_counter() - t0
    if w.block2 and not args.two_level:
        t0 = time.perf_counter()
        h.build_subspace(w.block2, w.nvec2, 1, inv_steps=w.inv2_steps, inv_shift=0.0, inv_tol=w.inv2_tol,
                         inv_maxiter=w.inv2_maxiter, seed=seeds["subspace"] + 11, level=2)
        out["level2_subspace"] = time.perf_counter() - t0
        t0 = time.perf_counter()
        h.build_coarse(1, level=2)
        out["level2_operator"] = time.perf_counter() - t0
        if w.qtrunc_order:
            t0 = time.perf_counter()
            lo, hi = h.set_coarse_preconditioner(w.qtrunc_order)
            out["qtrunc_chebyshev"] = {"seconds": time.perf_counter() - t0, "order": w.qtrunc_order,
                                       "interval": [lo, hi]}
    ldop = args.ldop_nvec if args.ldop_nvec is not None else w.ldop_nvec
    if ldop and (not w.block2 or args.two_level):
        t0 = time.perf_counter()
        h.build_coarse_deflation(ldop, inv_steps=3, shift=-1e-3, tol=1e-5, maxiter=20000, seed=seeds["ldop"])
        out["ldop_deflation"] = time.perf_counter() - t0
    return out


def run_ours(args, w):
    import torch
    import torch.distributed as dist

    from paper_1402_2585_gb300 import ALG_ADEF2, ALG_CG, Hdcg, HdcgError

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # the library runs on its own (non-legacy) stream, so its coarse loops can replay CUDA graphs
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    prec = PREC[w.prec]
    outer = 0 if prec == 0 else 1
    nrhs = args.nrhs
    batch_rhs = w.nrhs if args.batch_rhs is None else args.batch_rhs
    # the oracle's complete FP64 solve of the 8^4 x 8 workload runs on one host
    # core in a child process while the GPU works (about 1.5 minutes)
    oracle_proc = None
    if world == 1 and rank == 0 and not args.no_cpu_baseline:
        oracle_proc = subprocess.Popen(
            [sys.executable, "-c", "import json, bench; print(json.dumps(bench.oracle_cg_solve_cfg1()))"],
            cwd=ROOT, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True,
            env=dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1"))
    t_setup0 = time.perf_counter()
    seeds = replica_seeds(w, rank)
    U = sy.gauge_field(w.dims, w.eps, seeds["gauge"])
    h = Hdcg(w.dims, w.Ls, antiperiodic_t=w.antiperiodic_t, stream=stream.cuda_stream)
    h.set_dwf(w.M5, w.b, w.c, w.mass)
    h.set_gauge(torch.from_numpy(U).to(dev))
    del U
    setup = build_levels(h, w, seeds, args)
    setup["total"] = time.perf_counter() - t_setup0

    prm = Hdcg.default_params(algorithm=ALG_ADEF2, outer_prec=outer, sloppy_prec=prec, maxiter=5000,
                              reliable_delta=args.reliable_delta, batch=1, coarse_maxiter=5000)
    if nrhs == 1:
        bh = sy.gaussian_fermion(w.dims, w.Ls, seeds["source"])[None]
    else:
        bh = sy.gaussian_fermions(w.dims, w.Ls, seeds["source"], nrhs)
    # pinned host copies (the end-to-end run copies them in and out every step)
    bp = torch.empty(bh.shape, dtype=torch.complex128, pin_memory=not args.no_e2e)
    bp.numpy()[...] = bh
    del bh
    b = bp.to(dev)
    x = torch.zeros_like(b)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    try:
        for _ in range(args.warmup):
            h.solve(b, x, w.tol, prm, nrhs=nrhs)
    except HdcgError as e:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "error": str(e), "workload": w.name}), flush=True)
        raise
    barrier()

    # timed region: profiling off
    clk = ClockSampler(local)
    clk.start()
    launches0 = h.launch_count()
    times, stats = [], []
    torch.cuda.nvtx.range_push("timed")
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        st = h.solve(b, x, w.tol, prm, nrhs=nrhs)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        times.append(e0.elapsed_time(e1) / 1e3)
        stats.append(st.as_dict())
    torch.cuda.nvtx.range_pop()
    launches = h.launch_count() - launches0
    clocks = clk.stop()
    t_solve = max_over_ranks(statistics.mean(times), world, dev)
    s0 = stats[-1]

    # profile pass: one more solve with event timing of every hop launch and phase
    flush.zero_()
    torch.cuda.synchronize(dev)
    h.set_profiling(True)
    h.solve(b, x, w.tol, prm, nrhs=nrhs)
    hop_all = {}
    for pname, pc in (("f64", 0), ("f32", 1), ("f16", 2), ("bf16", 3), ("df64", 5)):
        n_p, ms_p, by_p, op_p = h.get_hop_profile(pc, operator_bytes=True)
        if n_p:
            hop_all[pname] = {"launches": n_p, "avg_launch_us": ms_p * 1e3 / n_p, "ms": ms_p, "bytes": by_p,
                              "op_bytes": op_p, "GBps": by_p / (ms_p / 1e3) / 1e9 if ms_p > 0 else None}
    phases = h.get_phase_profile()
    h.set_profiling(False)
    coarse_rl = coarse_roofline(h, w, args)

    # the solution's true residual, recomputed by the library's FP64-accurate operator
    true_res = s0["true_residual"]


    # plain red-black CG on the same GPU (FP32 with FP64 reliable updates), one
    # right-hand side, bounded by --cg-maxiter: if it has not converged by then,
    # its time is a lower bound on its time to solution
    flush.zero_()
    torch.cuda.synchronize(dev)
    prm_cg = Hdcg.default_params(algorithm=ALG_CG, outer_prec=outer, maxiter=args.cg_maxiter,
                                 reliable_delta=args.reliable_delta)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    cgs = h.solve(b[:1].contiguous(), x[:1].contiguous(), w.tol, prm_cg, nrhs=1).as_dict()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t_cg = e0.elapsed_time(e1) / 1e3
    cg_conv = cgs["status"] == 0
    t_hdcg_rhs = t_solve / nrhs
    plain_cg = {"seconds": t_cg, "iterations": cgs["iterations"], "true_residual": cgs["true_residual"],
                "converged": cg_conv, "maxiter": args.cg_maxiter, "rhs": 1,
                "note": ("converged" if cg_conv else
                         "not converged at the iteration cap: its time to solution exceeds 'seconds'")}
    speedup = {"value": t_cg / t_hdcg_rhs if t_hdcg_rhs > 0 else None,
               "kind": "per right-hand side" + ("" if cg_conv else ", lower bound (CG not converged)"),
               "hdcg_seconds_per_rhs": t_hdcg_rhs}
    del b, x
    torch.cuda.empty_cache()

    # the batch of spin-colour point sources (12 for the physical-point-like
    # workload), solved together in batches as large as the device memory takes
    batched = None
    if batch_rhs > 1:
        pb = torch.from_numpy(sy.point_sources(w.dims, w.Ls, batch_rhs)).to(dev)
        px = torch.zeros_like(pb)
        flush.zero_()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sb = h.solve(pb, px, w.tol, prm, nrhs=batch_rhs).as_dict()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        tb = e0.elapsed_time(e1) / 1e3
        # the first point source alone, for the batched-against-sequential ratio
        p1 = pb[:1].contiguous()
        x1 = torch.zeros_like(p1)
        flush.zero_()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        s1 = h.solve(p1, x1, w.tol, prm, nrhs=1).as_dict()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        t1 = e0.elapsed_time(e1) / 1e3
        batched = {"rhs": batch_rhs, "sources": "spin-colour point sources", "seconds": tb,
                   "seconds_per_rhs": tb / batch_rhs, "rhs_per_batch": sb["batch_rhs"],
                   "iterations_max": sb["iterations"], "true_residual_max": sb["true_residual"],
                   "status": sb["status"], "single_gaussian_rhs_seconds": t_solve / nrhs,
                   "first_source_alone": {"seconds": t1, "iterations": s1["iterations"],
                                          "true_residual": s1["true_residual"]},
                   "speedup_vs_sequential_estimate": batch_rhs * t1 / tb if tb > 0 else None,
                   "sequential_note": "12 sequential solves estimated as 12 x the first source alone"}
        del pb, px, p1, x1
        torch.cuda.empty_cache()

    # end to end through the public API with pinned host buffers (every step copies
    # the right-hand sides in and the solutions out)
    e2e = None
    if not args.no_e2e:
        xp = torch.zeros(bp.shape, dtype=bp.dtype, pin_memory=True)
        ts_e2e = []
        for _ in range(1):
            flush.zero_()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            h.solve(bp, xp, w.tol, prm, nrhs=nrhs)
            ts_e2e.append(time.perf_counter() - t0)
        nbytes = bp.numel() * bp.element_size()
        e2e = {"value": statistics.mean(ts_e2e), "unit": "s", "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes}
        del bp, xp

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peak, peak_kind = peaks()
    pname = {0: "f64", 1: "f32"}[outer]
    sloppy = {0: "f64", 1: "f32", 2: "f16", 3: "bf16"}[prec]
    n_h = s0["n_mdagm_outer"] + s0["n_mdagm_sloppy"] + s0["n_mdagm_f64"]
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        per_site = oracle_h_seconds_per_site(w)
        n_h_rhs = n_h / nrhs
        solve1 = None
        if oracle_proc is not None:
            try:
                out, _ = oracle_proc.communicate(timeout=900)
                solve1 = json.loads(out.strip().splitlines()[-1])
            except Exception as e:   # report, do not fail the GPU line
                oracle_proc.kill()
                solve1 = {"error": str(e)}
        cpu = {"value": per_site * n5_of(w) * n_h, "unit": "s", "cores": 1, "kind": "oracle",
               "sample": cpu_sample_desc(w, round(n_h_rhs), nrhs), **host_info(),
               "oracle_solve_cfg1": solve1}
    line = {
        "metric": METRIC, "value": t_solve, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_solve * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": f"{pname} outer, {sloppy} sloppy", "data": "synthetic",
        "config": {"workload": w.name, "lattice": list(w.dims), "Ls": w.Ls, "M5": w.M5, "b": w.b, "c": w.c,
                   "mass": w.mass, "eps": w.eps, "block": list(w.block), "nvec": w.nvec,
                   "block2": list(w.block2) if (w.block2 and not args.two_level) else None,
                   "nvec2": w.nvec2 if (w.block2 and not args.two_level) else None, "tol": w.tol,
                   "storage": w.prec, "coarse_storage": args.coarse_prec or w.coarse_prec or w.prec,
                   "rhs_per_gpu": nrhs, "sources": "gaussian",
                   "l2": "inputs larger than L2; also flushed (512 MiB write) before each step",
                   "parallelism": f"replicas x{world}"},
        "roofline": None,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches / max(1, args.steps)),
        "clocks": clocks,
        "plain_cg": plain_cg,
        "speedup_vs_plain_cg": speedup,
        "hdcg": {"iterations": s0["iterations"], "coarse_iterations": s0["coarse_iterations"],
                 "coarse_iterations_max": s0["coarse_iterations_max"],
                 "n_mdagm_outer": s0["n_mdagm_outer"], "n_mdagm_sloppy": s0["n_mdagm_sloppy"],
                 "n_mdagm_f64": s0["n_mdagm_f64"], "reliable_updates": s0["reliable_updates"],
                 "true_residual": true_res, "batch_rhs": s0["batch_rhs"],
                 "h_applies_per_rhs": n_h / nrhs,
                 "h_applies_per_rhs_reference_arm": H_APPLIES_PER_RHS.get(w.name)},
        "phases_ms_per_solve_profiled": phases,
        "coarse_roofline": coarse_rl,
        "hop_profile": hop_all,
        "batched": batched,
        "setup_seconds": setup,
        "reliable_delta": args.reliable_delta,
    }
    line["roofline"] = roofline(w, hop_all, sloppy, peak, peak_kind, nrhs)
    line["hop_flops"] = hop_flop_rate(w, hop_all, sloppy)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def coarse_roofline(h, w, args):
    """The level-1 little Dirac stencil (Sec. 5.1) on its own: the tensor-core
    apply (k_capply_tc) of the workload's coarse operator to 1 and to 12
    coarse vectors, timed by the library with CUDA events over 20 launches
    after 3 warm-ups (hdcg_time_coarse_apply).
    Algorithmic bytes per apply: the stored operator, 81 Nvec^2 complex per
    coarse site (FP16: 4 B per complex; FP32 as FP16 hi + lo: 8 B), read once
    for all right-hand sides; the vectors (16 B per complex in and out of the
    coarse layout) are a few percent on top and not counted."""
    cp = args.coarse_prec or w.coarse_prec or w.prec
    bpc = {"f16": 4, "f32": 8, "f64": 16}.get(cp)
    vc = int(np.prod([d // b for d, b in zip(w.dims, w.block)]))
    peak, peak_kind = peaks()
    out = {"kernel": "k_capply_tc (tcgen05)" if cp in ("f16", "f32") else "capply (CUDA cores)",
           "storage": cp, "coarse_sites": vc, "nvec": w.nvec, "peak": peak, "peak_kind": f"{peak_kind} HBM copy"}
    if cp not in ("f16", "f32"):
        return out
    for R in (1, 12):
        t = h.time_coarse_apply(R, 20) / 1e6
        bytes_ = vc * 81 * w.nvec ** 2 * bpc
        out[f"rhs{R}"] = {"us_per_apply": t * 1e6, "operator_bytes": bytes_,
                          "GBps": bytes_ / t / 1e9, "frac": bytes_ / t / 1e9 / peak,
                          "tflops": 8.0 * vc * 81 * w.nvec ** 2 * R / t / 1e12}
    return out


def hop_flop_rate(w, hop_all, pname):
    """Flop rate of the roofline kernel's launches: every four launches are one
    H over the lattice's odd 5D sites (the bench's solves have one right-hand
    side), at hop_flops_per_site flops per site."""
    hp = hop_all.get(pname)
    if not hp or hp["ms"] <= 0:
        return None
    flops = hp["launches"] / 4.0 * n5_of(w) * hop_flops_per_site(w)
    return {"flop_per_site_per_H": hop_flops_per_site(w), "achieved": flops / (hp["ms"] / 1e3) / 1e12,
            "unit": "TFLOP/s", "kernel": f"hop_kernel ({pname} storage), the roofline kernel's launches"}


def roofline(w, hop_all, pname, peak, peak_kind, nrhs):
    """The dominant kernel's roofline: hop_kernel passes in the sloppy storage
    precision (most of the solve's fine-operator work).  achieved = algorithmic
    bytes per launch / mean launch time (CUDA events on the library's stream,
    profiled solve), in two accountings: the operator's own bytes ((240 +
    576/Ls) reals per 5D site per H, split over its four passes) and those plus
    the bytes the launches' fused epilogues add (CG update, shifted term)."""
    hp = hop_all.get(pname)
    if not hp:
        return None
    per_launch_s = hp["ms"] / 1e3 / hp["launches"]
    b_fused = hp["bytes"] / hp["launches"]
    b_op = hp["op_bytes"] / hp["launches"]
    return {"bound": "hbm", "achieved": b_fused / per_launch_s / 1e9, "peak": peak, "unit": "GB/s",
            "frac": b_fused / per_launch_s / 1e9 / peak,
            "traffic": HOP_TRAFFIC.get(w.name) if pname == "f16" else None,
            "traffic_note": ("ncu, unfused operator passes of one H at this size, mean per launch"
                             if HOP_TRAFFIC.get(w.name) and pname == "f16" else None),
            "kernel": f"hop_kernel ({pname} storage, 4 passes per H)", "launches": hp["launches"],
            "avg_launch_us": per_launch_s * 1e6, "bytes_per_launch": b_fused,
            "achieved_operator_bytes_only": b_op / per_launch_s / 1e9,
            "frac_operator_bytes_only": b_op / per_launch_s / 1e9 / peak,
            "operator_bytes_per_launch": b_op, "peak_kind": f"{peak_kind} HBM copy"}


def run_apply_only(args, w):
    """A small case for kernel profiling: ``args.apply_only`` H applies in the
    workload's storage precision on device-resident canonical buffers (after
    two warm-up applies); prints the mean time per apply."""
    import torch

    from paper_1402_2585_gb300 import Hdcg
    prec = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3, "df64": 5}[args.apply_prec] if args.apply_prec else PREC[w.prec]
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    h = Hdcg(w.dims, w.Ls, antiperiodic_t=w.antiperiodic_t, stream=stream.cuda_stream)
    h.set_dwf(w.M5, w.b, w.c, w.mass)
    h.set_gauge(torch.from_numpy(sy.gauge_field(w.dims, w.eps, w.gauge_seed)).to(dev))
    dt = {0: torch.float64, 1: torch.float32, 2: torch.float16, 3: torch.bfloat16, 5: torch.float64}[prec]
    psi = sy.gaussian_fermion(w.dims, w.Ls, w.source_seed)
    x = torch.view_as_real(torch.from_numpy(psi)).to(dt).to(dev).contiguous()
    y = torch.empty_like(x)
    for _ in range(2):
        h.apply_mdagm(x, y, prec)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("profile")
    e0.record(stream)
    for _ in range(args.apply_only):
        h.apply_mdagm(x, y, prec)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize(dev)
    print(json.dumps({"workload": w.name, "applies": args.apply_only, "prec": prec,
                      "ms_per_apply": e0.elapsed_time(e1) / args.apply_only}), flush=True)


def run_coarse_only(args, w):
    """A small case for kernel profiling: the workload's coarse operator
    (subspace = block-orthonormalised Gaussian vectors, no inverse iteration)
    applied ``args.coarse_only`` times through hdcg_coarse_apply."""
    import torch

    from paper_1402_2585_gb300 import Hdcg
    prec = PREC[w.prec]
    sub_prec = prec if prec in (0, 1) else 2
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    h = Hdcg(w.dims, w.Ls, antiperiodic_t=w.antiperiodic_t, stream=stream.cuda_stream)
    h.set_dwf(w.M5, w.b, w.c, w.mass)
    h.set_gauge(torch.from_numpy(sy.gauge_field(w.dims, w.eps, w.gauge_seed)).to(dev))
    h.build_subspace(w.block, w.nvec, sub_prec, inv_steps=0, seed=w.subspace_seed)
    cp = args.coarse_prec or w.coarse_prec
    h.build_coarse(PREC[cp] if cp else sub_prec)
    vc = 1
    for d, b in zip(w.dims, w.block):
        vc *= d // b
    R = args.coarse_rhs
    if R:
        xs = sy.complex_normal(5, (R, vc, w.nvec))
    else:
        xs = sy.coarse_gaussian(vc, w.nvec, 5)
    x = torch.view_as_real(torch.from_numpy(xs)).to(dev).contiguous()
    y = torch.empty_like(x)

    def once():
        if R:
            h.coarse_apply_multi(x, y, R)
        else:
            h.coarse_apply(x, y)
    once()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    torch.cuda.nvtx.range_push("profile")
    e0.record(stream)
    for _ in range(args.coarse_only):
        once()
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize(dev)
    print(json.dumps({"workload": w.name, "coarse_applies": args.coarse_only, "rhs": R or 1,
                      "coarse_storage": cp or w.prec,
                      "ms_per_call_device": e0.elapsed_time(e1) / args.coarse_only,
                      "ms_per_call_host": (time.perf_counter() - t0) * 1e3 / args.coarse_only}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(sy.WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--two-level", action="store_true", help="leave out the blocked second coarsening")
    ap.add_argument("--reliable-delta", type=float, default=0.01, help="FP64 true-residual update factor")
    ap.add_argument("--cg-maxiter", type=int, default=6000,
                    help="iteration cap of the plain-CG comparison (one right-hand side)")
    ap.add_argument("--coarse-prec", choices=["f64", "f32", "f16"], default=None,
                    help="storage of the little Dirac operator (default: the workload's)")
    ap.add_argument("--nrhs", type=int, default=1,
                    help="Gaussian right-hand sides per timed solve (reported as rhs_per_gpu)")
    ap.add_argument("--batch-rhs", type=int, default=None,
                    help="point sources of the one batched solve after the timed steps (default: the workload's)")
    ap.add_argument("--ldop-nvec", type=int, default=None,
                    help="second-level global deflation vectors (two-level workloads; default: the workload's)")
    ap.add_argument("--apply-only", type=int, default=0,
                    help="profiling case: run this many H applies only (no solve)")
    ap.add_argument("--apply-prec", choices=["f64", "f32", "f16", "bf16", "df64"], default=None,
                    help="with --apply-only: operator precision (default: the workload's storage)")
    ap.add_argument("--coarse-rhs", type=int, default=0,
                    help="with --coarse-only: apply to this many right-hand sides at once (hdcg_coarse_apply_multi)")
    ap.add_argument("--coarse-only", type=int, default=0,
                    help="profiling case: build the coarse operator and apply it this many times")
    args = ap.parse_args()
    w = sy.WORKLOADS[args.workload]
    if args.coarse_only:
        run_coarse_only(args, w)
    elif args.apply_only:
        run_apply_only(args, w)
    elif args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
