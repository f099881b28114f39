#!/usr/bin/env python
"""Benchmark of the GB300 two-grid Helmholtz library.

Metric: fine-level two-grid cycle throughput (GDOF/s) and time to a 1e-8
relative residual, for the mixed-precision form (FP32 cycle with BF16
subdomain inverse rows, FP64 FGMRES) against the plain FP64 form.

Workload (one GPU): 2-D unit square, 40 wavelengths, Q4 elements on 100 x 100
cells (401^2 complex dofs, coarse grid 201^2), wavenumber from a seeded
smooth random velocity field (correlation length 1/8, +/-30% contrast), a
10-dof sin^2 absorbing layer plus Robin sides, a centred Gaussian source,
alpha_s = 0.5, 2 x 2-cell subdomains.  Inputs are synthetic (synth/).

A step is one two-grid cycle u <- TwoGridStep(u, f) (Algorithm 1 with the
CSDD smoother): every fine-level kernel plus the coarse solve.  Value =
dofs x replicas / step time.  With --gpus N (torchrun) each rank runs an
independent replica (the path does not shard); the time is the max over ranks.

--impl reference times the FP64 CPU oracle on the same workload instead.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
# the CPU oracle legs state their core counts: no hidden BLAS threads
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")

METRIC = "fine-level two-grid cycle GDOF/s and time-to-1e-8 residual vs plain FP64 form"
WORKLOAD = "square40_q4_n100"
HBM_FALLBACK_GBS = 6800.0
# dram__bytes_read.sum + dram__bytes_write.sum per launch of the FP32-cycle
# subdomain kernel (BF16 rows, 1 rhs) on this workload, by kernel variant, from
# an ncu capture of this script's timed region (the profile summary named), with
# the digest of the kernel's code at the time of that capture (dd_sources_digest):
# the figure is reported only while that code is unchanged, else null.
DD_TRAFFIC = {2: {"bytes": 239.06e6, "sources": "5adbefe3cfd66632",
                  "profile": "profiles/launches_square40_q4_n100.md"}}
DD_SOURCES = ("paper_2509_17494_gb300/csrc/dd.cu", "paper_2509_17494_gb300/csrc/ptx.cuh",
              "paper_2509_17494_gb300/csrc/kernels.h")


def dd_sources_digest():
    """Digest of the subdomain kernel's code: dd.cu, ptx.cuh and, of kernels.h,
    only the definition of its argument block (DDArgs), which it reads."""
    import hashlib

    h = hashlib.sha256()
    for rel in DD_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            data = fh.read()
        if rel.endswith("kernels.h"):
            txt = data.decode()
            i = txt.index("struct DDArgs {")
            data = txt[i:txt.index("};", i) + 2].encode()
        h.update(data)
    return h.hexdigest()[:16]


def dd_traffic(variant):
    rec = DD_TRAFFIC.get(variant)
    if not rec or rec["sources"] != dd_sources_digest():
        return None
    return rec["bytes"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-cycles", type=int, default=15, help="oracle cycles in the CPU-baseline sample")
    ap.add_argument("--batch-rhs", type=int, default=64, help="right-hand sides of the batched section (0: skip)")
    ap.add_argument("--batch-workload", default="square80_q4_n200",
                    help="workload of the batched section (default: 80 wavelengths, 801^2 dofs, its 64 sources)")
    ap.add_argument("--mixed-batch", action="store_true",
                    help="add 16 independent domains of 20..80 wavelengths, one cycle each, in one CUDA graph")
    ap.add_argument("--dd-variant", choices=["auto", "0", "1", "2", "3", "4", "5"], default="auto",
                    help="FP32 subdomain kernel: auto (set-up autotuner), 0 k_dd_apply, 1 k_dd_stream, 2 k_dd_stream2, "
                         "3 k_dd_stream with three CTAs per SM "
                         "(pin it when the same command runs under a profiler, whose serialised launches "
                         "change the autotuner's timings)")
    ap.add_argument("--fine-variant", choices=["auto", "0", "1"], default="auto",
                    help="FP32 and FP64 fine-apply tile variant: auto, 0 (large tiles), 1 (small tiles)")
    ap.add_argument("--cycle-variant", choices=["auto", "0", "1", "2"], default="auto",
                    help="launch structure of the cycle (th_set_kernel_variant TH_K_CYCLE)")
    ap.add_argument("--coarse-variant", choices=["auto", "0", "1", "2"], default="auto",
                    help="FP32 one-rhs coarse sweep: auto, 0 two phases, 1 one cluster barrier per step, "
                         "2 st.async row exchange")
    ap.add_argument("--learned-steps", type=int, default=400, help="training steps of the learned section (0: skip)")
    ap.add_argument("--bc-sweep", action="store_true",
                    help="iterations vs size for Robin / Dirichlet / Neumann sides (Fig. 6 (a))")
    ap.add_argument("--learned-c4-pairs", type=int, default=0,
                    help="training pairs of the corrector on the 401^2 coarse grid, 32 channels (0: skip)")
    ap.add_argument("--dim3", choices=["cube10_q2_n40", "cube2_q2_n8", "none"], default="cube10_q2_n40",
                    help="3-D workload of the three-dimensional section")
    ap.add_argument("--table1", action="store_true",
                    help="add the parameter study of the paper's Table 1 (OPT coarsening) on the GPU")
    ap.add_argument("--gal", choices=["workload", "none"], default="workload",
                    help="standard Galerkin p-coarsening ('gal') against QSFEM ('opt') on the bench workload")
    ap.add_argument("--gal-sweep", action="store_true",
                    help="add iterations vs problem size for opt and gal (the trend of the paper's Fig. 5)")
    ap.add_argument("--table2", action="store_true",
                    help="add the shift study of the paper's Table 2 (gal coarsening, p = 6) on the GPU")
    ap.add_argument("--lfa", choices=["sweep", "none"], default="sweep",
                    help="Fourier-analysis rates against dofs per wavelength on the GPU (Figs. 3 and 4)")
    ap.add_argument("--kernel-case", choices=["dd64", "coarse64", "krylov64"], default=None,
                    help="only run one small-footprint kernel workload for a profiler (64 sources on the 401^2 "
                         "workload: the smoother, the coarse solve, or 8 FGMRES steps) and print one JSON line")
    return ap.parse_args()


def kernel_case(args):
    """A profiler's workload: one operation of the batched path, 64 right-hand
    sides on the 401^2 grid, a few GB on the device (FGMRES restart 8), inside
    the NVTX range 'kernel_case' after two untimed repetitions."""
    import numpy as np
    import torch

    import paper_2509_17494_gb300 as th
    import synth

    dev = "cuda:0"
    w = synth.workload("square40_q4_n100")
    nr = 64
    S = th.TwoGridSolver(w["n"], w["p"], w["k"], w["eps"], alpha_s=w["alpha_s"], l_dd=w["l_dd"], prec="bf16",
                         restart=8, maxit=8, tol=1e-8, nrhs_max=nr, device=dev)
    F = torch.from_numpy(np.ascontiguousarray(synth.random_sources(w["n"], w["p"], 2, nr, 100))).to(dev)
    U = torch.from_numpy(np.ascontiguousarray(synth.random_complex((nr, S.N), 5))).to(dev)
    rc = torch.from_numpy(np.ascontiguousarray(synth.random_complex((nr, S.Nc), 6))).to(dev)

    def once():
        if args.kernel_case == "dd64":
            S.smooth(F, U)
        elif args.kernel_case == "coarse64":
            S.coarse_solve(rc)
        else:
            S.solve(F, check=False)

    for _ in range(2):
        once()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("kernel_case")
    once()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    S.device_status()
    print(json.dumps({"kernel_case": args.kernel_case, "workload": w["name"], "nrhs": nr, "ok": True}), flush=True)
    S.close()


# ----------------------------------------------------------------------------
# distributed helpers (replicas; the max over ranks of the step time)
# ----------------------------------------------------------------------------
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------
# algorithmic bytes of the subdomain-product kernel (per launch, one rhs)
# ----------------------------------------------------------------------------
def dd_algorithmic_bytes(n, p, l_dd, wbytes, vbytes):
    """Bytes one subdomain-product launch must move (one right-hand side):
    the inverse rows of every subdomain, U-box rows x Omega-box columns without
    padding, plus one read of the residual and one write of the results."""
    nb = -(-n // l_dd)
    base, rem = divmod(n, nb)
    sizes = [base + 1] * rem + [base] * (nb - rem)
    starts = [sum(sizes[:i]) for i in range(nb)]
    u1 = [z * p + 1 for z in sizes]                                              # U-box nodes per axis
    w1 = [(min(s + z + 1, n) - max(s - 1, 0)) * p + 1 for s, z in zip(starts, sizes)]  # Omega-box nodes
    s1 = sum(a * b for a, b in zip(u1, w1))
    w_entries = s1 * s1                     # sum over blocks (bx, by) of (ux uy) (wx wy)
    N = (n * p + 1) ** 2
    v_entries = sum(u1) ** 2
    return w_entries * wbytes + N * vbytes + v_entries * vbytes, w_entries


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback"


# ----------------------------------------------------------------------------
# native arm
# ----------------------------------------------------------------------------
def run_native(args):
    import numpy as np
    import torch

    import paper_2509_17494_gb300 as th
    import synth
    from paper_2509_17494_gb300 import _build

    rank, local, world = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or world == 1:
        _build.build()
    barrier(world)
    w = synth.workload(args.workload)
    n, p = w["n"], w["p"]
    t0 = time.time()
    S = th.TwoGridSolver(n, p, w["k"], w["eps"], alpha_s=w["alpha_s"], l_dd=w["l_dd"], prec="bf16",
                         extra_prec=("fp64",), restart=30, maxit=300, tol=1e-8, nrhs_max=1, device=dev)
    setup_s = time.time() - t0
    if args.dd_variant != "auto":
        S.set_variant("dd", "fp32", int(args.dd_variant))
    if args.fine_variant != "auto":
        S.set_variant("fine", "fp32", int(args.fine_variant))
        S.set_variant("fine", "fp64", int(args.fine_variant))
    if args.coarse_variant != "auto":
        S.set_variant("coarse", "fp32", int(args.coarse_variant))
    if args.cycle_variant != "auto":
        S.set_variant("cycle", "fp32", int(args.cycle_variant))
    N = S.N
    f = torch.from_numpy(np.ascontiguousarray(w["f"] if w["f"].ndim == 1 else w["f"][0])).to(dev)
    stream = torch.cuda.current_stream(dev)
    # FP64 and FP32 pipe rates of this GPU (FMA chains, CUDA events): the
    # denominators of the FP64 form's roofline
    pipe = {pr: th.peak_fma(pr, stream=stream.cuda_stream) / 1e12 for pr in ("fp64", "fp32")}

    def timed_cycles(prec, steps, warmup, profile=False, clocks=None, graph=True):
        S.set_precision(prec)
        u = torch.zeros_like(f)
        step = S.cycle_graph if graph else S.cycle
        for _ in range(warmup):
            step(f, u)
        torch.cuda.synchronize(dev)
        barrier(world)
        torch.cuda.synchronize(dev)
        l0 = S.launch_count()
        if profile:
            S.profile(True)
        if clocks:
            clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        tag = f"cycle_{prec}_{'graph' if graph else 'launches'}{'_prof' if profile else ''}"
        torch.cuda.nvtx.range_push(tag)   # ncu --nvtx-include "<tag>/" selects this region
        e0.record(stream)
        for _ in range(steps):
            step(f, u)
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize(dev)
        barrier(world)
        torch.cuda.synchronize(dev)
        ck = clocks.stop() if clocks else None
        prof = S.profile_read() if profile else None
        if profile:
            S.profile(False)
        ms = e0.elapsed_time(e1) / steps
        return ms, S.launch_count() - l0, prof, ck, u

    clocks = ClockSampler(local)
    ms_mixed, launches, _, ck, _ = timed_cycles("bf16", args.steps, args.warmup, clocks=clocks)
    ms_mixed = max_over_ranks(ms_mixed, world, dev)
    # the same steps launched kernel by kernel (no graph), then with per-kernel CUDA events (th_profile)
    ms_nograph, _, _, _, _ = timed_cycles("bf16", args.steps, 2, graph=False)
    # the same graph-replayed step with each launch structure of the cycle
    cyc0 = S.get_variant("cycle", "fp32")
    ms_by_cycle = {}
    for v in (0, 1, 2):
        S.set_variant("cycle", "fp32", v)
        ms_by_cycle[v] = round(max_over_ranks(timed_cycles("bf16", args.steps, 3)[0], world, dev), 4)
    S.set_variant("cycle", "fp32", cyc0)
    ms_prof, _, prof, _, _ = timed_cycles("bf16", args.steps, 1, profile=True, graph=False)
    steps64 = max(3, args.steps // 2)
    ms_fp64, _, _, _, _ = timed_cycles("fp64", steps64, max(3, args.warmup // 2))
    _, _, prof64, _, _ = timed_cycles("fp64", steps64, 1, profile=True, graph=False)
    ms_fp64 = max_over_ranks(ms_fp64, world, dev)

    # time to 1e-8 (th_solve, synchronous; host clock inside the library)
    def solve_time(prec, reps):
        S.set_precision(prec)
        out = []
        for _ in range(reps):
            torch.cuda.synchronize(dev)
            x, info = S.solve(f)
            out.append(info)
        return min(i["ms_total"] for i in out), out[-1]

    # the first solve of a context captures its per-step CUDA graphs: best of several
    tt_mixed, info_mixed = solve_time("bf16", 3)
    tt_fp64, info_fp64 = solve_time("fp64", 2)

    # end to end through the host-buffer entry point (pinned host memory)
    S.set_precision("bf16")
    fh = torch.from_numpy(np.ascontiguousarray(f.cpu().numpy())).pin_memory()
    uh = torch.zeros_like(fh).pin_memory()
    fnp, unp = fh.numpy(), uh.numpy()
    for _ in range(2):
        S.cycle_host(fnp, unp)
    barrier(world)
    te = time.perf_counter()
    e2e_steps = max(3, args.steps // 2)
    for _ in range(e2e_steps):
        S.cycle_host(fnp, unp)
    ms_e2e = (time.perf_counter() - te) * 1e3 / e2e_steps
    ms_e2e = max_over_ranks(ms_e2e, world, dev)

    S.device_status()
    gdofs = lambda ms: N * world / (ms * 1e-3) / 1e9
    # roofline of the dominant kernel class (by time) of the mixed cycle
    per_step = {k: (v[0] / args.steps, v[1] / args.steps) for k, v in prof.items()}
    dominant = max(per_step, key=lambda k: per_step[k][0])
    dd_ms, dd_cnt = prof["dd"]
    dd_avg_ms = dd_ms / max(dd_cnt, 1)
    dd_kernel = {0: "k_dd_apply", 1: "k_dd_stream (TMA bulk)", 2: "k_dd_stream2 (TMA bulk, producer warp)",
                 3: "k_dd_stream (TMA bulk, three CTAs per SM)", 4: "k_dd_stream (TMA bulk, paired FP32 FMAs)",
                 5: "k_dd_stream (TMA bulk, paired FP32 FMAs, three CTAs per SM)"}[S.get_variant("dd", "fp32")]
    alg_bytes, _ = dd_algorithmic_bytes(n, p, w["l_dd"], 4, 8)
    hbm, peak_src = peaks()
    achieved = alg_bytes / (dd_avg_ms * 1e-3) / 1e9
    roofline = {"kernel": f"{dd_kernel}, BF16 inverse rows, 1 rhs", "bound": "hbm", "achieved": round(achieved, 1),
                "peak": hbm, "peak_source": peak_src, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                "traffic": dd_traffic(S.get_variant("dd", "fp32")), "alg_bytes_per_launch": int(alg_bytes),
                "traffic_source": (DD_TRAFFIC.get(S.get_variant("dd", "fp32")) or {}).get("profile"),
                "avg_launch_ms": round(dd_avg_ms, 5),
                "dominant_by_time": dominant,
                "profiled_ms_per_step": round(ms_prof, 4),
                "share_of_step": {k: round(v[0] / ms_prof, 3) for k, v in per_step.items() if v[1] > 0},
                "variants": {"dd_fp32": S.get_variant("dd", "fp32"), "fine_fp32": S.get_variant("fine", "fp32"),
                             "dd_fp64": S.get_variant("dd", "fp64"), "fine_fp64": S.get_variant("fine", "fp64"),
                             "coarse_sweep": S.get_variant("coarse", "fp32"),
                             "outer_residual": "double-single" if S.get_variant("resid", "fp32") else "fp64"}}

    # the FP64 form's subdomain products: 8 flop per complex row entry, FP64-pipe bound
    _, w_entries = dd_algorithmic_bytes(n, p, w["l_dd"], 16, 16)
    dd64_ms, dd64_cnt = prof64["dd"]
    dd64_avg = dd64_ms / max(dd64_cnt, 1)
    dd64_tf = 8.0 * w_entries / (dd64_avg * 1e-3) / 1e12
    roofline64 = {"kernel": {0: "k_dd_apply", 1: "k_dd_stream", 2: "k_dd_stream2"}.get(S.get_variant("dd", "fp64"),
                                                                                      "k_dd_stream"),
                  "bound": "fp64", "achieved": round(dd64_tf, 3), "peak": round(pipe["fp64"], 3),
                  "peak_source": "measured here (th_peak_fma: FP64 FMA chains, CUDA events)", "unit": "TFLOP/s",
                  "frac": round(dd64_tf / pipe["fp64"], 4), "flop_per_launch": int(8 * w_entries),
                  "avg_launch_ms": round(dd64_avg, 5)}

    fine_ms = sum(v[0] for k, v in per_step.items() if k != "coarse_solve")
    line = {
        "metric": METRIC,
        "value": round(gdofs(ms_mixed), 4),
        "unit": "GDOF/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_mixed, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "dim": 2, "p": p, "cells": f"{n}x{n}", "dofs": N,
                   "coarse_dofs": S.Nc, "wavelengths": 40, "alpha_s": w["alpha_s"], "l_dd": w["l_dd"],
                   "n_s": 1, "n_dd": 1, "omega_c": 1.0, "nrhs": 1,
                   "precision": "FP32 cycle, BF16 inverse rows (FP32 accumulate), FP64 FGMRES",
                   "step": "one TwoGridStep u <- TwoGridStep(u, f) replayed from a CUDA graph: outer residual of the "
                           "FP64 iterate in double-single arithmetic (FP32 output), 2 DD smoothers, FP32 "
                           "residual, restriction, coarse block solve, prolongation, FP64 update",
                   "l2": "inputs larger than L2: the BF16 inverse rows streamed every smoother step are "
                         f"{alg_bytes / 1e6:.0f} MB > 129 MB",
                   "setup_s": round(setup_s, 2), "parallelism": f"replicas x{world}"},
        "cycle_launch": {"graph_ms_per_step": round(ms_mixed, 4), "no_graph_ms_per_step": round(ms_nograph, 4),
                         "variant": cyc0,
                         "graph_ms_by_variant": {"0 step by step": ms_by_cycle[0], "1 fused": ms_by_cycle[1],
                                                 "2 fused, programmatic dependent launch": ms_by_cycle[2]}},
        "fine_level": {"value": round(gdofs(fine_ms), 4), "unit": "GDOF/s", "ms_per_step": round(fine_ms, 4),
                       "what": "sum of the per-kernel event times of every cycle kernel except the coarse solve"},
        "time_to_tol_ms": round(tt_mixed, 3),
        "iters": info_mixed["iters"],
        "relres": info_mixed["relres_max"],
        "fp64": {"value": round(gdofs(ms_fp64), 4), "ms_per_step": round(ms_fp64, 4),
                 "time_to_tol_ms": round(tt_fp64, 3), "iters": info_fp64["iters"],
                 "relres": info_fp64["relres_max"],
                 "share_of_step": {k: round(v[0] / steps64 / ms_fp64, 3) for k, v in prof64.items() if v[1] > 0},
                 "dd_roofline": roofline64},
        "pipe_peaks_tflops": {k: round(v, 3) for k, v in pipe.items()},
        "speedup_vs_fp64": {"cycle": round(ms_fp64 / ms_mixed, 2), "time_to_tol": round(tt_fp64 / tt_mixed, 2)},
        "roofline": roofline,
        "e2e": {"value": round(gdofs(ms_e2e), 4), "unit": "GDOF/s", "ms_per_step": round(ms_e2e, 4),
                "h2d_bytes_per_step": 2 * N * 16, "d2h_bytes_per_step": N * 16},
        "gpu_launches": int(launches),
        "clocks": ck,
    }
    S.close()
    del S
    if args.batch_rhs > 0:
        line["batched"] = batched_section(args, synth.workload(args.batch_workload), dev, world)
    if args.mixed_batch:
        line["mixed_batch"] = mixed_batch_section(dev, world)
    if args.learned_steps > 0:
        line["learned"] = learned_section(args, dev)
    if args.learned_c4_pairs > 0:
        line["learned_c4"] = learned_c4_section(args, dev)
    if args.dim3 != "none":
        line["dim3"] = dim3_section(args, dev, world)
    if args.table1:
        line["table1"] = table1_section(dev)
    if args.gal != "none":
        line["galerkin"] = galerkin_section(args, w, dev)
    if args.gal_sweep:
        line["gal_sweep"] = gal_sweep_section(dev)
    if args.bc_sweep:
        line["bc_sweep"] = bc_sweep_section(dev)
    if args.table2:
        line["table2"] = table2_section(dev)
    if args.lfa != "none":
        line["lfa"] = lfa_section(rank == 0 and world == 1 and not args.no_cpu_baseline)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_cycles)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


# ----------------------------------------------------------------------------
# many sources at once, and the learned coarse corrector
# ----------------------------------------------------------------------------
def batched_section(args, w, dev, world):
    """nrhs seeded point sources on one workload (by default 80 wavelengths on
    801^2 dofs with its 64 sources) in one graph-replayed cycle: the subdomain
    products run on the tensor cores (k_dd_umma), the coarse solve on tiles of
    right-hand sides."""
    import numpy as np
    import torch

    import paper_2509_17494_gb300 as th
    import synth

    nr = args.batch_rhs
    t0 = time.time()
    S = th.TwoGridSolver(w["n"], w["p"], w["k"], w["eps"], alpha_s=w["alpha_s"], l_dd=w["l_dd"], prec="bf16",
                         restart=30, maxit=300, tol=1e-8, nrhs_max=nr, device=dev)
    setup_s = time.time() - t0
    src = w["f"] if (w["f"].ndim == 2 and w["f"].shape[0] == nr) else synth.random_sources(w["n"], w["p"], 2, nr, 100)
    F = torch.from_numpy(np.ascontiguousarray(src)).to(dev)
    U = torch.zeros_like(F)
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        S.cycle_graph(F, U)
    torch.cuda.synchronize(dev)
    steps = max(3, args.steps // 2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("batched_cycle")
    e0.record(stream)
    for _ in range(steps):
        S.cycle_graph(F, U)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    ms = max_over_ranks(ms, world, dev)
    S.profile(True)
    for _ in range(3):
        S.cycle(F, U)
    torch.cuda.synchronize(dev)
    prof = S.profile_read()
    S.profile(False)
    dd_ms, dd_cnt = prof["dd"]
    dd_avg = dd_ms / max(dd_cnt, 1)
    alg_bytes, _ = dd_algorithmic_bytes(w["n"], w["p"], w["l_dd"], 4, 8)
    NR, NC = 81, 289
    nsub = (w["n"] // w["l_dd"]) ** 2
    flops = 8.0 * NR * NC * nsub * nr
    S.solve(F)  # captures the per-step CUDA graphs
    _, info = S.solve(F)
    hbm, src = peaks()
    out = {"workload": w["name"], "dofs": S.N, "setup_s": round(setup_s, 1),
           "nrhs": nr, "sources": "seeded Gaussian point sources (synth.random_sources, seed 100)",
           "value": round(S.N * nr * world / (ms * 1e-3) / 1e9, 4), "unit": "GDOF/s", "ms_per_cycle": round(ms, 4),
           "time_to_tol_ms": round(info["ms_total"], 2), "iters": info["iters"], "relres_max": info["relres_max"],
           "dd_tensor_core": {"kernel": "k_dd_umma (tcgen05, BF16 x BF16 -> FP32 in tensor memory)",
                              "avg_launch_ms": round(dd_avg, 5),
                              "achieved_tflops": round(flops / (dd_avg * 1e-3) / 1e12, 1),
                              "achieved_gbs": round(alg_bytes / (dd_avg * 1e-3) / 1e9, 1),
                              "hbm_peak_gbs": hbm, "peak_source": src},
           "per_kernel_ms_per_cycle": {k: round(v[0] / 3, 4) for k, v in prof.items() if v[1] > 0}}
    S.close()
    return out


def mixed_batch_section(dev, world):
    """16 independent domains of 20, 24, ..., 80 wavelengths (Q4, 2.5 W cells per
    side, each its own random field and centred source, 10-dof layer), one
    mixed-precision TwoGridStep each, all captured into one CUDA graph and
    replayed: the cycle throughput of the whole batch; then each domain's solve
    to 1e-8."""
    import numpy as np
    import torch

    import paper_2509_17494_gb300 as th
    import synth

    Ws = list(range(20, 81, 4))
    t0 = time.time()
    solvers, Fs, Us = [], [], []
    for i, W in enumerate(Ws):
        n = int(round(2.5 * W))
        k = synth.random_wavenumber(n, 2, float(W), seed=10 + i)
        eps = synth.absorbing_layer(n, 2, 4, k, 10.0)
        S = th.TwoGridSolver(n, 4, k, eps, alpha_s=0.5, l_dd=2, prec="bf16", extra_prec=("fp64",), restart=30,
                             maxit=300, tol=1e-8, device=dev)
        S.set_graphs(False)  # the batch is captured as a whole below
        solvers.append(S)
        Fs.append(torch.from_numpy(synth.gaussian_source(n, 4, 2)).to(dev))
        Us.append(torch.zeros_like(Fs[-1]))
    setup_s = time.time() - t0
    dofs = sum(S.N for S in solvers)
    cs = torch.cuda.Stream(dev)
    sides = [torch.cuda.Stream(dev) for _ in solvers]
    cs.wait_stream(torch.cuda.current_stream(dev))
    for S, F, U, st in zip(solvers, Fs, Us, sides):  # first launches outside the capture
        st.wait_stream(cs)
        with torch.cuda.stream(st):
            S.cycle(F, U)
    torch.cuda.synchronize(dev)
    # one graph: every domain's step on a stream of its own, forked from and
    # joined into the capture stream, so the domains' kernels run concurrently
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=cs):
        for S, F, U, st in zip(solvers, Fs, Us, sides):
            st.wait_stream(cs)
            with torch.cuda.stream(st):
                S.cycle(F, U)
        for st in sides:
            cs.wait_stream(st)
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize(dev)
    steps = 10
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(dev)
    e0.record(stream)
    for _ in range(steps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, world, dev)
    iters, tts = [], []
    for S, F in zip(solvers, Fs):
        S.set_graphs(True)
        _, info = S.solve(F, check=False)
        iters.append(info["iters"] if info["converged"] else -1)
        tts.append(info["ms_total"])
        S.device_status()
    del graph
    for S in solvers:
        S.close()
    return {"domains": len(Ws), "wavelengths": Ws, "dofs_total": dofs, "setup_s": round(setup_s, 1),
            "graph": "one CUDA graph holding one TwoGridStep of every domain (mixed precision), each domain's "
                     "launch sequence on a stream of its own (forked from and joined into the capture stream)",
            "value": round(dofs * world / (ms * 1e-3) / 1e9, 4), "unit": "GDOF/s", "ms_per_batch_cycle": round(ms, 3),
            "iters": iters, "time_to_tol_ms_sum": round(sum(tts), 1)}


def dim3_section(args, dev, world):
    """The unit cube with Q2 elements and the fitted 27-point coarse operator:
    all sources of the workload in one graph-replayed cycle, FP32 cycle with
    BF16 subdomain rows (tensor cores, tiles of 16 sources) and with FP32 rows
    (CUDA cores) against the plain FP64 form, and the time to 1e-8."""
    import numpy as np
    import torch

    import paper_2509_17494_gb300 as th
    import synth

    w = synth.workload(args.dim3)
    F = np.ascontiguousarray(w["f"].reshape(-1, (w["n"] * w["p"] + 1) ** 3))
    nr = F.shape[0]
    t0 = time.time()
    S = th.TwoGridSolver(w["n"], w["p"], w["k"], w["eps"], alpha_s=w["alpha_s"], l_dd=w["l_dd"], prec="bf16",
                         extra_prec=("fp32", "fp64"), restart=30, maxit=300, nrhs_max=nr, device=dev, dim=3)
    setup_s = time.time() - t0
    Fd = torch.from_numpy(F).to(dev)
    stream = torch.cuda.current_stream(dev)
    out = {"workload": args.dim3, "dofs": S.N, "coarse_dofs": S.Nc, "nrhs": nr, "setup_s": round(setup_s, 1),
           "stencil": "fitted 27-point (project construction; the paper only cites a 3-D scheme)"}
    for prec in ("bf16", "fp32", "fp64"):
        S.set_precision(prec)
        U = torch.zeros_like(Fd)
        for _ in range(3):
            S.cycle_graph(Fd, U)
        torch.cuda.synchronize(dev)
        steps = 5
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push(f"dim3_cycle_{prec}")
        e0.record(stream)
        for _ in range(steps):
            S.cycle_graph(Fd, U)
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize(dev)
        ms = max_over_ranks(e0.elapsed_time(e1) / steps, world, dev)
        S.profile(True)
        S.cycle(Fd, U)
        torch.cuda.synchronize(dev)
        prof = S.profile_read()
        S.profile(False)
        _, info = S.solve(Fd, check=False)
        out[prec] = {"value": round(S.N * nr * world / (ms * 1e-3) / 1e9, 4), "unit": "GDOF/s",
                     "ms_per_cycle": round(ms, 3), "time_to_tol_ms": round(info["ms_total"], 1),
                     "iters": info["iters"], "converged": info["converged"], "relres_max": info["relres_max"],
                     "per_kernel_ms_per_cycle": {k: round(v[0], 3) for k, v in prof.items() if v[1] > 0}}
    out["speedup_vs_fp64"] = {pr: {"cycle": round(out["fp64"]["ms_per_cycle"] / out[pr]["ms_per_cycle"], 2),
                                   "time_to_tol": round(out["fp64"]["time_to_tol_ms"] / out[pr]["time_to_tol_ms"], 2)}
                              for pr in ("bf16", "fp32")}
    S.close()
    return out


# The paper's Table 1 (OPT coarsening): (a) alpha_s x n_dd x subdomain size at
# p = 4 (10 ppw) and p = 6 (8 ppw); (b) n_s x omega_c x ppw.  Its domain, Krylov
# method and tolerance are not stated; here: unit square, constant k, Robin
# sides, centred source, FGMRES(60) to 1e-6, p = 4 on 25^2 and p = 6 on 20^2 cells.
TABLE1A_PAPER = {(4, 4, 1): [7, 7, 7, 7, 7], (4, 4, 2): [6, 6, 6, 6, 6], (4, 6, 1): [7, 6, 6, 6, 7],
                 (4, 6, 2): [6, 5, 5, 6, 6], (6, 4, 1): [9, 8, 8, 8, 8], (6, 4, 2): [7, 7, 7, 7, 8],
                 (6, 6, 1): [9, 8, 8, 8, 8], (6, 6, 2): [7, 7, 7, 7, 8]}
TABLE1B_PAPER = {(4, 1, 1.0): [9, 7, 5], (4, 1, 0.8): [8, 6, 7], (4, 1, 0.6): [11, 11, 12],
                 (4, 2, 1.0): [8, 6, 5], (4, 2, 0.8): [7, 6, 7], (4, 2, 0.6): [11, 11, 12],
                 (6, 1, 1.0): [19, 8, 7, 5], (6, 1, 0.8): [16, 6, 5, 7], (6, 1, 0.6): [15, 8, 10, 11],
                 (6, 2, 1.0): [16, 8, 7, 5], (6, 2, 0.8): [12, 5, 5, 7], (6, 2, 0.6): [11, 8, 10, 11]}


def table1_section(dev):
    import numpy as np
    import torch

    import paper_2509_17494_gb300 as th
    import synth

    cells = {4: 25, 6: 20}

    def iters(p, ppw, **kw):
        n = cells[p]
        W = n * p / ppw
        k = synth.constant_wavenumber(n, 2, W)
        S = th.TwoGridSolver(n, p, k, None, restart=60, maxit=200, tol=1e-6, device=dev, **kw)
        f = torch.from_numpy(synth.gaussian_source(n, p, 2)).to(dev)
        _, info = S.solve(f, check=False)
        S.close()
        return info["iters"] if info["converged"] else -1

    out = {"setup": "unit square, constant k, Robin sides, centred source, FGMRES(60) to 1e-6; "
                    "p = 4 on 25^2 cells, p = 6 on 20^2 cells", "a": {}, "b": {}}
    alphas = [0.1, 0.15, 0.2, 0.3, 0.4]
    for (p, l_dd, n_dd), paper in TABLE1A_PAPER.items():
        ppw = 10 if p == 4 else 8
        got = [iters(p, ppw, alpha_s=a, l_dd=l_dd, n_dd=n_dd) for a in alphas]
        out["a"][f"p{p}_ldd{l_dd}_ndd{n_dd}"] = {"alpha_s": alphas, "gpu": got, "paper": paper}
    for (p, n_s, om), paper in TABLE1B_PAPER.items():
        ppws = [8, 10, 14] if p == 4 else [6, 8, 10, 14]
        got = [iters(p, q, alpha_s=0.2, l_dd=4, n_s=n_s, omega_c=om) for q in ppws]
        out["b"][f"p{p}_ns{n_s}_omega{om}"] = {"ppw": ppws, "gpu": got, "paper": paper}
    return out


def galerkin_section(args, w, dev):
    """The paper's comparison method on the bench workload: standard Galerkin
    p-type coarsening (coarse Q_{p/2} on the same mesh, its block-sweep solve),
    with the shifts the paper uses for its size study (alpha_s = alpha_c = 0.02)
    and without coarse correction, against the QSFEM coarse level ('opt'), all
    in the mixed form (FP32 cycle, BF16 rows, FP64 FGMRES)."""
    import numpy as np
    import torch

    import paper_2509_17494_gb300 as th

    f = torch.from_numpy(np.ascontiguousarray(w["f"] if w["f"].ndim == 1 else w["f"][0])).to(dev)
    out = {"setup": "bench workload, mixed precision, FGMRES(30) to 1e-8, at most 300 iterations"}

    def run(label, coarse, alpha_s, alpha_c=0.0, none=False):
        t0 = time.time()
        S = th.TwoGridSolver(w["n"], w["p"], w["k"], w["eps"], alpha_s=alpha_s, l_dd=w["l_dd"], prec="bf16",
                             extra_prec=("fp64",), restart=30, maxit=300, tol=1e-8, device=dev, coarse=coarse,
                             alpha_c=alpha_c)
        setup = time.time() - t0
        if none:
            S.set_coarse("none")
        u = torch.zeros_like(f)
        for _ in range(3):
            S.cycle_graph(f, u)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            S.cycle_graph(f, u)
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / 10
        best = None
        for _ in range(2):
            _, info = S.solve(f, check=False)
            best = info if best is None or info["ms_total"] < best["ms_total"] else best
        S.device_status()
        S.close()
        out[label] = {"alpha_s": alpha_s, "alpha_c": alpha_c if coarse == "gal" else None,
                      "iters": best["iters"], "converged": best["converged"], "relres": best["relres_max"],
                      "time_to_tol_ms": round(best["ms_total"], 2), "cycle_ms": round(ms, 4),
                      "setup_s": round(setup, 2)}

    run("opt", "qsfem", w["alpha_s"])
    run("gal", "gal", 0.02, 0.02)
    run("gal_noCGC", "gal", 0.02, 0.02, none=True)
    return out


def gal_sweep_section(dev):
    """Iterations vs problem size at 8 points per wavelength (constant k, Robin
    sides, centred source, FGMRES(60) to 1e-6, Q4, 4 x 4-cell subdomains): QSFEM
    ('opt', alpha_s = 0.2) against Galerkin ('gal', alpha_s = alpha_c = 0.02)
    and Galerkin without coarse correction."""
    import torch

    import paper_2509_17494_gb300 as th
    import synth

    p, ppw, l_dd = 4, 8, 4
    out = {"setup": "unit square, constant k, Robin sides, centred source, Q4, 8 ppw, l_dd = 4, "
                    "FGMRES(60) to 1e-6", "wavelengths": [], "opt": [], "gal": [], "gal_noCGC": []}
    for W in (5, 10, 20, 40):
        n = int(round(W * ppw / p))
        k = synth.constant_wavenumber(n, 2, W)
        f = torch.from_numpy(synth.gaussian_source(n, p, 2)).to(dev)
        out["wavelengths"].append(W)
        for label, kw, none in (("opt", dict(alpha_s=0.2), False),
                                ("gal", dict(alpha_s=0.02, coarse="gal", alpha_c=0.02), False),
                                ("gal_noCGC", dict(alpha_s=0.02, coarse="gal", alpha_c=0.02), True)):
            S = th.TwoGridSolver(n, p, k, None, l_dd=l_dd, restart=60, maxit=400, tol=1e-6, device=dev, **kw)
            if none:
                S.set_coarse("none")
            _, info = S.solve(f, check=False)
            S.close()
            out[label].append(info["iters"] if info["converged"] else -1)
    return out


def bc_sweep_section(dev):
    """Fig. 6 (a): iterations of the QSFEM ('opt') method against problem size for
    different boundary conditions (constant k, 8 points per wavelength, Q4,
    4 x 4-cell subdomains, alpha_s = 0.2, centred source, FGMRES(60) to 1e-6):
    Robin on every side; Dirichlet on two non-opposite sides (x low, y low) and
    Robin on the others; Neumann there instead.  A thin damping layer (10 dofs)
    keeps the Dirichlet / Neumann problems away from resonance."""
    import torch

    import paper_2509_17494_gb300 as th
    import synth

    p, ppw, l_dd = 4, 8, 4
    variants = {"robin": "robin",
                "dirichlet_2_sides": {"xlo": "dirichlet", "ylo": "dirichlet", "xhi": "robin", "yhi": "robin"},
                "neumann_2_sides": {"xlo": "neumann", "ylo": "neumann", "xhi": "robin", "yhi": "robin"}}
    out = {"setup": "unit square, constant k, Q4, 8 ppw, l_dd = 4, alpha_s = 0.2, 10-dof damping layer, "
                    "centred source, FGMRES(60) to 1e-6", "wavelengths": [], **{v: [] for v in variants}}
    for W in (5, 10, 20, 40):
        n = int(round(W * ppw / p))
        k = synth.constant_wavenumber(n, 2, W)
        eps = synth.absorbing_layer(n, 2, p, k, 10.0)
        f = torch.from_numpy(synth.gaussian_source(n, p, 2)).to(dev)
        out["wavelengths"].append(W)
        for label, bc in variants.items():
            S = th.TwoGridSolver(n, p, k, eps, bc=bc, alpha_s=0.2, l_dd=l_dd, restart=60, maxit=400, tol=1e-6,
                                 device=dev)
            _, info = S.solve(f, check=False)
            S.close()
            out[label].append(info["iters"] if info["converged"] else -1)
    return out


# Table 2 of the paper: FGMRES iterations with 'gal' coarsening, p = 6, rows
# alpha_c = 0, 0.01, 0.02, 0.05, 0.1, 0.2, 0.5 and no coarse correction, columns
# alpha_s = 0.01, 0.02, 0.05, 0.1 (-1 stands for "> 200").
TABLE2_PAPER = {
    6: [[-1, -1, 110, -1], [-1, -1, 61, 102], [-1, 177, 46, 73], [-1, 30, 31, 47], [35, 21, 25, 35],
        [21, 19, 21, 29], [21, 20, 22, 25], [23, 22, 24, 29]],
    8: [[15, 15, 14, 15], [14, 14, 14, 14], [14, 13, 13, 14], [15, 15, 15, 16], [18, 18, 18, 19],
        [22, 21, 21, 23], [25, 24, 25, 28], [29, 27, 28, 32]],
}


def table2_section(dev):
    """The shift study of the paper's Table 2 with our kernels: 'gal' coarsening,
    p = 6, 6 and 8 points per wavelength, alpha_s x alpha_c.  The paper does not
    state the domain size; here 20 x 20 cells (121^2 dofs: 20 / 15 wavelengths),
    constant k, Robin sides, centred source, 4 x 4-cell subdomains (the paper's
    ~40-dof subdomains exceed the subdomain kernels' 1024-row limit at p = 6),
    FGMRES(60) to 1e-6, at most 200 iterations (-1 = not converged)."""
    import torch

    import paper_2509_17494_gb300 as th
    import synth

    p, n, l_dd = 6, 20, 4
    a_s = [0.01, 0.02, 0.05, 0.1]
    a_c = [0.0, 0.01, 0.02, 0.05, 0.1, 0.2, 0.5, None]   # None: no coarse-grid correction
    out = {"setup": "20^2 cells, p = 6, constant k, Robin sides, centred source, l_dd = 4, FGMRES(60) to 1e-6",
           "alpha_s": a_s, "alpha_c": ["noCGC" if c is None else c for c in a_c]}
    f = torch.from_numpy(synth.gaussian_source(n, p, 2)).to(dev)
    for ppw in (6, 8):
        k = synth.constant_wavenumber(n, 2, n * p / ppw)
        rows = []
        for c in a_c:
            row = []
            for s in a_s:
                S = th.TwoGridSolver(n, p, k, None, alpha_s=s, l_dd=l_dd, restart=60, maxit=200, tol=1e-6, device=dev,
                                     coarse="gal", alpha_c=0.0 if c is None else c)
                if c is None:
                    S.set_coarse("none")
                _, info = S.solve(f, check=False)
                S.close()
                row.append(info["iters"] if info["converged"] else -1)
            rows.append(row)
        out[f"ppw{ppw}"] = {"gpu": rows, "paper": TABLE2_PAPER[ppw]}
    return out


def lfa_section(with_oracle):
    """Asymptotic two-grid rates sup_theta rho(M(theta)) from the GPU Fourier
    analysis (Section 6) against dofs per wavelength, as in Figs. 3 and 4: QSFEM
    ('opt') and Galerkin ('gal') coarse levels for p = 2, 4, 6 (exact shifted
    smoother, alpha_s = 0.2, eps = 0.01 k^2 / pi, 48 x 48 theta grid), and for
    opt the smoothing-step / relaxation variants of Fig. 4.  With the oracle the
    same analysis of one parameter point on the host (numpy eigvals) gives the
    CPU rate of theta points per second."""
    import math

    import numpy as np

    import paper_2509_17494_gb300 as th

    npts, D, a_s = 48, 0.01, 0.2
    ppws = [4, 5, 6, 7, 8, 10, 12, 16, 20]
    out = {"setup": "periodic plane, constant k, eps = 0.01 k^2 / pi, alpha_s = 0.2, exact shifted smoother, "
                    f"{npts} x {npts} theta grid", "ppw": ppws, "opt": {}, "gal": {}, "opt_variants": {}}
    n_theta = 0
    t0 = time.perf_counter()
    for p in (2, 4, 6):
        params = [[2 * math.pi * p / q, D / math.pi, a_s, 1.0] for q in ppws]
        out["opt"][f"p{p}"] = [round(float(v), 4) for v in th.lfa_rho(p, params, npts=npts)]
        out["gal"][f"p{p}"] = [round(float(v), 4) for v in th.lfa_rho(p, params, npts=npts, coarse="gal")]
        n_theta += 2 * len(params) * npts * npts
    for p in (4, 6):
        for n_s, om in ((1, 0.8), (2, 1.0), (2, 0.8)):
            params = [[2 * math.pi * p / q, D / math.pi, a_s, om] for q in ppws]
            out["opt_variants"][f"p{p}_ns{n_s}_omega{om}"] = [round(float(v), 4)
                                                              for v in th.lfa_rho(p, params, n_s=n_s, npts=npts)]
            n_theta += len(params) * npts * npts
    gpu_s = time.perf_counter() - t0
    out["gpu"] = {"theta_points": n_theta, "wall_s": round(gpu_s, 3),
                  "theta_per_s": round(n_theta / gpu_s, 1)}
    # coarse-level dispersion error D_P / k (Section 3.2) at the coarse spacing
    # h_c = 2 h / p, i.e. half the fine dofs per wavelength: eta_c = 4 pi / ppw
    ppw_d = [7, 8, 10, 12, 16, 20]
    etas = [4 * math.pi / q for q in ppw_d]
    t2 = time.perf_counter()
    disp = {kind: [float("%.3e" % v) for v in th.dispersion(kind, etas, nt=256)] for kind in ("qsfem", "q1", "fd5")}
    out["dispersion"] = {"what": "D_P / k of the coarse stencil at eta_c = 4 pi / (fine dofs per wavelength), "
                                 "max over 256 directions (th_dispersion, FP64 on the GPU)",
                         "ppw": ppw_d, **disp, "gpu_wall_s": round(time.perf_counter() - t2, 3)}
    if with_oracle:
        from oracle import lfa as olfa

        t1 = time.perf_counter()
        ops = olfa.BlochOperators(4, 2 * math.pi * 4 / 8, D / math.pi, a_s)
        grid = olfa.theta_grid(16)
        ops.rho(grid)
        cpu_s = time.perf_counter() - t1
        out["oracle"] = {"sample": "p = 4, 8 dofs per wavelength, 16 x 16 theta grid (numpy eigvals, one process)",
                         "theta_per_s": round(len(grid) / cpu_s, 1)}
    return out


def learned_section(args, dev):
    """The learned coarse corrector on the 25 x 25 Q4 workload: trained on the GPU
    (own kernels) for a few seconds, then FGMRES iterations with the direct
    coarse solve, with no coarse correction, and with the corrector (alone and
    with the fallback to the direct solve at 1.5x the plain count)."""
    import numpy as np
    import torch

    import paper_2509_17494_gb300 as th
    import synth

    w = synth.workload("square10_q4_n25")
    S = th.TwoGridSolver(w["n"], w["p"], w["k"], w["eps"], alpha_s=0.5, l_dd=2, prec="bf16", extra_prec=("fp64",),
                         nrhs_max=8, restart=40, maxit=400, device=dev)
    levels, base = 4, 16
    S.unet_init(synth.he_normal(th.unet_param_shapes(levels, base), 77), levels=levels, base=base, batch_max=8)
    m = S.n * S.p // 2 + 1

    def pairs(count, seed):
        half = count // 2
        f = torch.from_numpy(synth.random_complex((half, S.N), seed)).to(dev)
        S.set_precision("fp64")
        u = torch.zeros_like(f)
        S.smooth(f, u)
        rc1 = S.restrict(S.residual(f, u))
        rc2 = torch.from_numpy(synth.smooth_coarse_noise(m, count - half, seed + 1)).to(dev)
        rc = torch.cat([rc1, rc2]).contiguous()
        uc = S.coarse_solve(rc)
        S.set_precision("bf16")
        return rc, uc

    t0 = time.time()
    losses = []
    for it in range(args.learned_steps):
        if it % 5 == 0:
            rc, uc = pairs(8, 1000 + it)
        losses.append(S.unet_train_step(rc, uc, lr=2e-3 if it < 0.7 * args.learned_steps else 5e-4))
    torch.cuda.synchronize(dev)
    train_s = time.time() - t0
    rc, uc = pairs(8, 99999)
    uh = S.unet_correct(rc)
    held = float((torch.linalg.vector_norm(uh - uc, dim=1) / torch.linalg.vector_norm(uc, dim=1)).mean())
    f = torch.from_numpy(np.ascontiguousarray(w["f"])).to(dev)
    res = {}
    S.set_coarse("direct")
    res["direct"] = S.solve(f)[1]
    S.set_coarse("none")
    res["none"] = S.solve(f, check=False)[1]
    S.set_coarse("learned", 0)
    res["learned"] = S.solve(f, check=False)[1]
    S.set_coarse("learned", res["direct"]["iters"])
    res["learned_with_fallback"] = S.solve(f, check=False)[1]
    S.set_coarse("direct")
    r1 = rc[:1].contiguous()
    for _ in range(3):
        S.unet_correct(r1)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(20):
        S.unet_correct(r1)
    e1.record()
    torch.cuda.synchronize(dev)
    out = {"workload": "square10_q4_n25", "network": f"U-Net {levels} levels, base {base} channels, BF16",
           "params": th.unet_param_count(levels, base), "train_steps": args.learned_steps,
           "train_s": round(train_s, 2), "loss_first10": round(float(np.mean(losses[:10])), 4),
           "loss_last10": round(float(np.mean(losses[-10:])), 4), "heldout_relerr": round(held, 4),
           "correct_ms_1rhs": round(e0.elapsed_time(e1) / 20, 4),
           "iters": {k: v["iters"] for k, v in res.items()},
           "converged": {k: v["converged"] for k, v in res.items()},
           "fallbacks": res["learned_with_fallback"]["fallbacks"]}
    S.close()
    return out


def learned_c4_section(args, dev):
    """The learned corrector at the size of its specification: the 401^2 coarse
    grid of the 80-wavelength Q4 problem (801^2 fine dofs, random k-field), a
    U-Net of 4 levels and 32 base channels, trained on the GPU on pairs (r_c,
    A_q^{-1} r_c) from the FP64 direct coarse solve (half restricted residuals of
    random fine right-hand sides after one smoothing step, half smooth random
    coarse fields), 8 pairs per Adam step, each pair used once; then FGMRES
    iterations and time to 1e-8 with the direct solve, with no correction, with
    the corrector alone and with the fallback at 1.5x the plain count."""
    import numpy as np
    import torch

    import paper_2509_17494_gb300 as th
    import synth

    w = synth.workload("square80_q4_n200")
    t0 = time.time()
    S = th.TwoGridSolver(w["n"], w["p"], w["k"], w["eps"], alpha_s=0.5, l_dd=2, prec="bf16", extra_prec=("fp64",),
                         nrhs_max=64, restart=60, maxit=400, device=dev)
    setup_s = time.time() - t0
    levels, base, B = 4, 32, 8
    S.unet_init(synth.he_normal(th.unet_param_shapes(levels, base), 77), levels=levels, base=base, batch_max=16)
    m = S.n * S.p // 2 + 1
    npairs = args.learned_c4_pairs
    gen = 64   # pairs per generation batch (one coarse solve of 64 right-hand sides)

    def pairs(count, seed):
        half = count // 2
        f = torch.from_numpy(synth.random_complex((half, S.N), seed)).to(dev)
        S.set_precision("fp64")
        u = torch.zeros_like(f)
        S.smooth(f, u)
        rc1 = S.restrict(S.residual(f, u))
        del f, u
        rc2 = torch.from_numpy(synth.smooth_coarse_noise(m, count - half, seed + 1)).to(dev)
        rc = torch.cat([rc1, rc2]).contiguous()
        uc = S.coarse_solve(rc)
        S.set_precision("bf16")
        return rc, uc

    t1 = time.time()
    losses, gen_s, seen = [], 0.0, 0
    steps = npairs // B
    for it in range(steps):
        if it % (gen // B) == 0:
            tg = time.time()
            rc, uc = pairs(gen, 5000 + it)
            torch.cuda.synchronize(dev)
            gen_s += time.time() - tg
        k = (it % (gen // B)) * B
        lr = 2e-3 if it < 0.7 * steps else 5e-4
        losses.append(S.unet_train_step(rc[k:k + B].contiguous(), uc[k:k + B].contiguous(), lr=lr))
        seen += B
    torch.cuda.synchronize(dev)
    train_s = time.time() - t1
    rc, uc = pairs(16, 424242)
    uh = S.unet_correct(rc)
    held = float((torch.linalg.vector_norm(uh - uc, dim=1) / torch.linalg.vector_norm(uc, dim=1)).mean())
    f = torch.from_numpy(np.ascontiguousarray(w["f"][0])).to(dev)
    res = {}
    S.set_coarse("direct")
    res["direct"] = S.solve(f)[1]
    S.set_coarse("none")
    res["none"] = S.solve(f, check=False)[1]
    S.set_coarse("learned", 0)
    res["learned"] = S.solve(f, check=False)[1]
    S.set_coarse("learned", res["direct"]["iters"])
    res["learned_with_fallback"] = S.solve(f, check=False)[1]
    S.set_coarse("direct")
    r1 = rc[:1].contiguous()

    def time_it(fn, reps=10):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    correct_ms = time_it(lambda: S.unet_correct(r1))
    direct_ms = time_it(lambda: S.coarse_solve(r1))
    out = {"workload": "square80_q4_n200 (coarse grid 401^2)",
           "network": f"U-Net {levels} levels, base {base} channels, BF16 weights, FP32 accumulation",
           "params": th.unet_param_count(levels, base), "setup_s": round(setup_s, 1),
           "pairs": seen, "batch": B, "adam_steps": steps, "pair_generation_s": round(gen_s, 1),
           "train_s_total": round(train_s, 1), "loss_first20": round(float(np.mean(losses[:20])), 4),
           "loss_last20": round(float(np.mean(losses[-20:])), 4), "heldout_relerr": round(held, 4),
           "correct_ms_1rhs": round(correct_ms, 3), "direct_coarse_solve_ms_1rhs": round(direct_ms, 3),
           "iters": {k: v["iters"] for k, v in res.items()},
           "time_to_tol_ms": {k: round(v["ms_total"], 2) for k, v in res.items()},
           "converged": {k: v["converged"] for k, v in res.items()},
           "fallbacks": res["learned_with_fallback"]["fallbacks"]}
    S.close()
    return out


# ----------------------------------------------------------------------------
# the FP64 CPU oracle as the baseline / reference arm
# ----------------------------------------------------------------------------
def oracle_setup(name):
    import synth
    from oracle import twogrid

    w = synth.workload(name)
    P = twogrid.Problem(w["n"], w["p"], w["k"], w["eps"], alpha_s=w["alpha_s"])
    TG = twogrid.TwoGrid(P, l_dd=w["l_dd"])
    f = w["f"] if w["f"].ndim == 1 else w["f"][0]
    return P, TG, f


def _oracle_cycles_worker(name, cycles, bar, q):
    """One process of the all-core oracle sample: its own set-up, then `cycles`
    oracle cycles started together with every other process (single-threaded)."""
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    import numpy as np

    try:
        P, TG, f = oracle_setup(name)
        u = TG.step(np.zeros_like(f), f)
        bar.wait(timeout=900)
        t = time.perf_counter()
        for _ in range(cycles):
            u = TG.step(u, f)
        q.put(time.perf_counter() - t)
    except Exception as e:  # reported by the parent as a missing sample
        q.put(repr(e))


def cpu_baseline(name, cycles):
    """The FP64 oracle on the host: `cycles` cycles on one core, then the same
    number in every one of the host's cores at once (one process per core, each
    an independent replica of the problem with its own set-up; the processes are
    started with spawn, so none inherits this process's CUDA state)."""
    import multiprocessing as mp

    import numpy as np

    P, TG, f = oracle_setup(name)
    u = np.zeros_like(f)
    u = TG.step(u, f)  # warm
    t = time.perf_counter()
    for _ in range(cycles):
        u = TG.step(u, f)
    dt = (time.perf_counter() - t) / cycles
    out = {"value": round(P.N / dt / 1e9, 6), "unit": "GDOF/s", "cores": 1, "kind": "oracle",
           "sample": f"{cycles} TwoGridStep cycles of the FP64 NumPy/SciPy oracle on the full {name} "
                     f"workload (set-up excluded; SuperLU local solves, CSR applies and the banded coarse "
                     f"solve, one thread), {dt * 1e3:.0f} ms per cycle"}
    ncores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    if ncores < 2:
        return out
    ctx = mp.get_context("spawn")
    bar = ctx.Barrier(ncores)
    q = ctx.Queue()
    procs = [ctx.Process(target=_oracle_cycles_worker, args=(name, cycles, bar, q), daemon=True)
             for _ in range(ncores - 1)]
    for pr in procs:
        pr.start()
    times = []
    try:
        bar.wait(timeout=900)
        t = time.perf_counter()
        for _ in range(cycles):
            u = TG.step(u, f)
        times.append(time.perf_counter() - t)
        for _ in procs:
            times.append(q.get(timeout=900))
    except Exception as e:
        times.append(repr(e))
    for pr in procs:
        pr.join(timeout=60)
    ok = [x for x in times if isinstance(x, float)]
    if len(ok) == ncores:
        wall = max(ok)
        out["all_cores"] = {"value": round(ncores * cycles * P.N / wall / 1e9, 6), "unit": "GDOF/s",
                            "cores": ncores, "kind": "oracle",
                            "sample": f"{ncores} single-threaded processes (one per host core), each an "
                                      f"independent replica of the {name} oracle running {cycles} cycles at "
                                      f"once; slowest process {wall * 1e3 / cycles:.0f} ms per cycle"}
    else:
        out["all_cores"] = {"unavailable": f"{len(ok)} of {ncores} processes reported: "
                                           f"{[x for x in times if not isinstance(x, float)][:1]}"}
    return out


def run_reference(args):
    rank, _, world = dist_env()
    if world > 1 and rank != 0:
        return
    import numpy as np

    P, TG, f = oracle_setup(args.workload)
    u = np.zeros_like(f)
    for _ in range(args.warmup):
        u = TG.step(u, f)
    t = time.perf_counter()
    for _ in range(args.steps):
        u = TG.step(u, f)
    ms = (time.perf_counter() - t) * 1e3 / args.steps
    val = P.N / (ms * 1e-3) / 1e9
    line = {"metric": METRIC, "value": round(val, 6), "unit": "GDOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "step": "one TwoGridStep of the FP64 CPU oracle"},
            "cpu_baseline": {"value": round(val, 6), "unit": "GDOF/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} oracle cycles on the full workload (set-up excluded)"},
            "e2e": {"value": round(val, 6), "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.warmup < 3:
        args.warmup = 3
    if args.kernel_case:
        from paper_2509_17494_gb300 import _build

        _build.build()
        kernel_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
