"""Benchmark: HDCG time-to-solution on one GB300 against plain red-black CG,
with the fine Mpc^dag Mpc hop kernels' achieved bandwidth against the HBM roofline.

One step = one full HDCG (A-DEF2) solve of H x = b to a true FP64 residual of
``tol`` on the workload's lattice, inputs resident in HBM; subspace and coarse
operator are built once before the timed region (the paper reports setup
separately).  L2 is flushed (a 512 MiB write) before every timed step.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload NAME]
Under torchrun (N > 1) every rank solves its own replica (independent seed);
the timing is the max over ranks.  ``--impl reference`` times the FP64 CPU
oracle on the host cores (bounded sample, see ``cpu_sample``).
"""
from __future__ import annotations

import argparse
import json
import os
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
DEFAULT_WORKLOAD = "cfg2_16x16x16x16_ls16_shamir"
PREC = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3}


# DRAM bytes (read + write) per FP32 hop_kernel launch, mean of the four passes of
# one H, from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of
# the current kernel on this workload; to be reset to None whenever hop_kernel
# changes, since the counters then no longer describe it.
HOP_F32_TRAFFIC = {DEFAULT_WORKLOAD: 126.2e6}


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
def oracle_h_seconds(w, reps=1):
    """Seconds of one FP64 oracle H = Mpc^dag Mpc apply on the workload's full lattice."""
    from oracle.dwf import DWF
    U = sy.gauge_field(w.dims, w.eps, w.gauge_seed)
    d = DWF(w.dims, w.Ls, w.M5, w.b, w.c, w.mass, U)
    psi = sy.gaussian_fermion(w.dims, w.Ls, w.source_seed)
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        d.mdagm(psi)
        ts.append(time.perf_counter() - t0)
    return min(ts)


def cpu_sample_desc(w, n_h):
    return (f"one FP64 oracle H apply on the full {'x'.join(map(str, w.dims))}x{w.Ls} lattice, "
            f"scaled by the {n_h} fine H applies (outer + preconditioner + FP64 residual) of one HDCG solve "
            "of this workload; coarse-grid work of the oracle not included")


# H applies per HDCG solve of the default workload, recorded from the GPU arm's
# solve statistics (a property of the algorithm on this input); used only to
# scale the oracle's per-apply time in --impl reference, which runs no GPU code.
H_APPLIES_PER_SOLVE = {DEFAULT_WORKLOAD: 140}   # 15 outer + 120 preconditioner + 5 FP64 residual


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(k, "1")
    n_h = H_APPLIES_PER_SOLVE.get(w.name, 140)
    for _ in range(args.warmup):
        oracle_h_seconds(w)
    ts = [oracle_h_seconds(w) for _ in range(args.steps)]
    per_h = statistics.mean(ts)
    value = per_h * n_h
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_h * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "lattice": list(w.dims), "Ls": w.Ls, "tol": w.tol},
            "cpu_baseline": {"value": value, "unit": "s", "cores": 1, "kind": "oracle",
                             "sample": cpu_sample_desc(w, n_h)},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def run_ours(args, w):
    import torch
    import torch.distributed as dist

    from paper_1402_2585_gb300 import ALG_ADEF2, ALG_CG, F64, Hdcg, HdcgError

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    prec = PREC[w.prec]
    sub_prec = prec if prec in (0, 1) else 2
    coarse_prec = 0 if prec == 0 else (1 if prec == 1 else 2)
    t_setup0 = time.perf_counter()
    seeds = replica_seeds(w, rank)
    U = sy.gauge_field(w.dims, w.eps, seeds["gauge"])
    h = Hdcg(w.dims, w.Ls, antiperiodic_t=w.antiperiodic_t, stream=stream.cuda_stream)
    h.set_dwf(w.M5, w.b, w.c, w.mass)
    h.set_gauge(torch.from_numpy(U).to(dev))
    t_sub0 = time.perf_counter()
    h.build_subspace(w.block, w.nvec, sub_prec, inv_steps=args.inv_steps, inv_shift=0.0, inv_tol=args.inv_tol,
                     inv_maxiter=20000, seed=seeds["subspace"])
    t_sub = time.perf_counter() - t_sub0
    t_c0 = time.perf_counter()
    if args.coarse_prec:
        coarse_prec = PREC[args.coarse_prec]
    h.build_coarse(coarse_prec)
    t_coarse = time.perf_counter() - t_c0
    t_l0 = time.perf_counter()
    ldop = None
    if args.ldop_nvec is None:
        args.ldop_nvec = w.ldop_nvec
    if args.ldop_nvec:
        h.build_coarse_deflation(args.ldop_nvec, inv_steps=args.ldop_steps, shift=args.ldop_shift,
                                 tol=args.ldop_tol, maxiter=20000, seed=seeds["ldop"])
        lam = h.get_coarse_deflation(args.ldop_nvec)
        fin = lam[np.isfinite(lam)]
        ldop = {"nvec": args.ldop_nvec, "inv_steps": args.ldop_steps, "shift": args.ldop_shift,
                "tol": args.ldop_tol, "dropped": int(len(lam) - len(fin)),
                "ritz_min": float(fin[0]) if len(fin) else None, "ritz_max": float(fin[-1]) if len(fin) else None}
    t_ldop = time.perf_counter() - t_l0
    setup_s = time.perf_counter() - t_setup0

    outer = 0 if prec == 0 else 1
    nrhs = args.nrhs or w.nrhs
    prm = Hdcg.default_params(algorithm=ALG_ADEF2, outer_prec=outer, sloppy_prec=prec, maxiter=5000,
                              reliable_delta=args.reliable_delta, batch=1)
    prm_cg = Hdcg.default_params(algorithm=ALG_CG, outer_prec=outer, maxiter=100000,
                                 reliable_delta=args.reliable_delta)
    if nrhs == 1:
        b = torch.from_numpy(sy.gaussian_fermion(w.dims, w.Ls, seeds["source"])).to(dev)
    else:
        b = torch.from_numpy(sy.point_sources(w.dims, w.Ls, nrhs)).to(dev)
    x = torch.zeros_like(b)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    try:
        for _ in range(args.warmup):
            h.solve(b, x, w.tol, prm, nrhs=nrhs)
    except HdcgError as e:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "error": str(e), "workload": w.name, "ldop_deflation": ldop,
                              "coarse_storage": args.coarse_prec}), flush=True)
        raise
    barrier()

    clk = ClockSampler(local)
    clk.start()
    h.set_profiling(True)
    launches0 = h.launch_count()
    times, stats = [], []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.nvtx.range_push("timed")
        e0.record(stream)
        st = h.solve(b, x, w.tol, prm, nrhs=nrhs)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        torch.cuda.nvtx.range_pop()
        times.append(e0.elapsed_time(e1) / 1e3)
        stats.append(st.as_dict())
    launches = h.launch_count() - launches0
    n_hop, hop_ms, hop_bytes = h.get_hop_profile(outer)
    hop_all = {}
    for pname, pc in (("f64", 0), ("f32", 1), ("f16", 2), ("bf16", 3)):
        n_p, ms_p, by_p = h.get_hop_profile(pc)
        if n_p:
            hop_all[pname] = {"launches": n_p, "avg_launch_us": ms_p * 1e3 / n_p,
                              "GBps": by_p / (ms_p / 1e3) / 1e9 if ms_p > 0 else None}
    phases = {k: v / args.steps for k, v in h.get_phase_profile().items()}
    h.set_profiling(False)
    clocks = clk.stop()

    t_solve = max_over_ranks(statistics.mean(times), world, dev)

    # plain red-black CG on the same GPU (same precision policy)
    cg_times, cg_stats = [], None
    for _ in range(max(1, min(2, args.steps))):
        flush.zero_()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cg_stats = h.solve(b, x, w.tol, prm_cg, nrhs=nrhs).as_dict()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        cg_times.append(e0.elapsed_time(e1) / 1e3)
    t_cg = statistics.mean(cg_times)

    # end to end through the public API with pinned host buffers
    bh = b.cpu().pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    e2e = []
    for _ in range(max(1, min(3, args.steps))):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        h.solve(bh, xh, w.tol, prm, nrhs=nrhs)
        e2e.append(time.perf_counter() - t0)
    nbytes = bh.numel() * bh.element_size()  # all right-hand sides of one step

    seq = None
    if nrhs > 1:
        prm_seq = Hdcg.default_params(algorithm=ALG_ADEF2, outer_prec=outer, sloppy_prec=prec, maxiter=5000,
                                      reliable_delta=args.reliable_delta, batch=0)
        flush.zero_()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sq = h.solve(b, x, w.tol, prm_seq, nrhs=nrhs).as_dict()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        seq = {"seconds": e0.elapsed_time(e1) / 1e3, "iterations_total": sq["iterations"],
               "true_residual": sq["true_residual"]}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peak, peak_kind = peaks()
    achieved = hop_bytes / (hop_ms / 1e3) / 1e9 if hop_ms > 0 else 0.0
    # flop rate of the same launches: a quarter of one H's flops per site per pass
    n5 = (int(np.prod(w.dims)) // 2) * w.Ls
    fl_site = hop_flops_per_site(w)
    hop_tflops = (n_hop * nrhs * n5 * fl_site / 4) / (hop_ms / 1e3) / 1e12 if hop_ms > 0 else 0.0
    s0 = stats[-1]
    n_h = s0["n_mdagm_outer"] + s0["n_mdagm_sloppy"] + s0["n_mdagm_f64"]
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        per_h = oracle_h_seconds(w)
        cpu = {"value": per_h * n_h, "unit": "s", "cores": 1, "kind": "oracle",
               "sample": cpu_sample_desc(w, n_h)}
    line = {
        "metric": METRIC, "value": t_solve, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_solve * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == 0 else "f32",
        "data": "synthetic",
        "config": {"workload": w.name, "lattice": list(w.dims), "Ls": w.Ls, "M5": w.M5, "b": w.b, "c": w.c,
                   "mass": w.mass, "eps": w.eps, "block": list(w.block), "nvec": w.nvec, "tol": w.tol,
                   "storage": w.prec, "rhs_per_gpu": nrhs, "coarse_storage": args.coarse_prec or None,
                   "l2": "flushed (512 MiB write) before each step",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if peak else None,
                     "traffic": HOP_F32_TRAFFIC.get(w.name) if outer == 1 else None,
                     "kernel": "hop_kernel (4 passes per H; FP32 storage)", "launches": n_hop,
                     "avg_launch_us": hop_ms * 1e3 / max(1, n_hop), "peak_kind": f"{peak_kind} HBM copy"},
        "hop_flops": {"flop_per_site_per_H": fl_site, "achieved": hop_tflops, "unit": "TFLOP/s",
                      "kernel": "hop_kernel (FP32 storage, the roofline kernel's launches)"},
        "cpu_baseline": cpu,
        "e2e": {"value": statistics.mean(e2e), "unit": "s", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes},
        "gpu_launches": int(launches / max(1, args.steps)),
        "clocks": clocks,
        "plain_cg": {"seconds": t_cg, "iterations": cg_stats["iterations"],
                     "true_residual": cg_stats["true_residual"]},
        "speedup_vs_plain_cg": t_cg / t_solve if t_solve > 0 else None,
        "hdcg": {"iterations": s0["iterations"], "coarse_iterations": s0["coarse_iterations"],
                 "n_mdagm_outer": s0["n_mdagm_outer"], "n_mdagm_sloppy": s0["n_mdagm_sloppy"],
                 "n_mdagm_f64": s0["n_mdagm_f64"], "reliable_updates": s0["reliable_updates"],
                 "true_residual": s0["true_residual"]},
        "phases_ms_per_solve": phases,
        "hop_profile": hop_all,
        "sequential_single_rhs": seq,
        "ldop_deflation": ldop,
        "setup_seconds": {"total": setup_s, "subspace": t_sub, "coarse_operator": t_coarse,
                          "ldop_deflation": t_ldop,
                          "inverse_iteration": {"steps": args.inv_steps, "tol": args.inv_tol}},
        "reliable_delta": args.reliable_delta,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


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
    h.build_coarse(PREC[args.coarse_prec] if args.coarse_prec else sub_prec)
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
                      "coarse_storage": args.coarse_prec or w.prec,
                      "ms_per_call_device": e0.elapsed_time(e1) / args.coarse_only,
                      "ms_per_call_host": (time.perf_counter() - t0) * 1e3 / args.coarse_only}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(sy.WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--inv-steps", type=int, default=3, help="inverse-iteration steps of the subspace setup")
    ap.add_argument("--inv-tol", type=float, default=1e-4, help="CG tolerance of each inverse-iteration step")
    ap.add_argument("--reliable-delta", type=float, default=0.01, help="FP64 true-residual update factor")
    ap.add_argument("--coarse-prec", choices=["f64", "f32", "f16"], default=None,
                    help="storage of the little Dirac operator (default: the workload's)")
    ap.add_argument("--nrhs", type=int, default=0,
                    help="right-hand sides per solve (default: the workload's; reported as rhs_per_gpu)")
    ap.add_argument("--ldop-nvec", type=int, default=None,
                    help="second-level deflation vectors of the little Dirac operator (0: none; default: the "
                         "workload's)")
    ap.add_argument("--ldop-steps", type=int, default=3, help="inverse-iteration steps of that space")
    ap.add_argument("--ldop-shift", type=float, default=-1e-3,
                    help="shift of those inverse-iteration steps (negative: times the mean diagonal of A)")
    ap.add_argument("--ldop-tol", type=float, default=1e-5, help="coarse CG residual of those steps")
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
