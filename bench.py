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

METRIC = "fine-level two-grid cycle GDOF/s and time-to-1e-8 residual vs plain FP64 form"
WORKLOAD = "square40_q4_n100"
HBM_FALLBACK_GBS = 6800.0
# dram__bytes_read.sum + dram__bytes_write.sum of one k_dd_apply (BF16 rows,
# 1 rhs) launch on this workload, from the ncu capture summarised in
# profiles/k_dd_apply_bf16_square40_q4_n100.md; None once the kernel changes.
DD_TRAFFIC_BYTES = {0: 241.1e6, 1: None}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-cycles", type=int, default=15, help="oracle cycles in the CPU-baseline sample")
    return ap.parse_args()


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
    N = S.N
    f = torch.from_numpy(np.ascontiguousarray(w["f"] if w["f"].ndim == 1 else w["f"][0])).to(dev)
    stream = torch.cuda.current_stream(dev)

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
        e0.record(stream)
        for _ in range(steps):
            step(f, u)
        e1.record(stream)
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

    tt_mixed, info_mixed = solve_time("bf16", 3)
    tt_fp64, info_fp64 = solve_time("fp64", 1)

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
    dd_kernel = "k_dd_stream (TMA bulk)" if S.get_variant("dd", "fp32") else "k_dd_apply"
    alg_bytes, _ = dd_algorithmic_bytes(n, p, w["l_dd"], 4, 8)
    hbm, peak_src = peaks()
    achieved = alg_bytes / (dd_avg_ms * 1e-3) / 1e9
    roofline = {"kernel": f"{dd_kernel}, BF16 inverse rows, 1 rhs", "bound": "hbm", "achieved": round(achieved, 1),
                "peak": hbm, "peak_source": peak_src, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                "traffic": DD_TRAFFIC_BYTES.get(S.get_variant("dd", "fp32")), "alg_bytes_per_launch": int(alg_bytes),
                "avg_launch_ms": round(dd_avg_ms, 5),
                "dominant_by_time": dominant,
                "profiled_ms_per_step": round(ms_prof, 4),
                "share_of_step": {k: round(v[0] / ms_prof, 3) for k, v in per_step.items() if v[1] > 0},
                "variants": {"dd_fp32": S.get_variant("dd", "fp32"), "fine_fp32": S.get_variant("fine", "fp32"),
                             "dd_fp64": S.get_variant("dd", "fp64"), "fine_fp64": S.get_variant("fine", "fp64")}}

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
                   "step": "one TwoGridStep u <- TwoGridStep(u, f) replayed from a CUDA graph: FP64 residual, "
                           "2 DD smoothers, FP32 residual, restriction, coarse block solve, prolongation",
                   "l2": "inputs larger than L2: the BF16 inverse rows streamed every smoother step are "
                         f"{alg_bytes / 1e6:.0f} MB > 129 MB",
                   "setup_s": round(setup_s, 2), "parallelism": f"replicas x{world}"},
        "cycle_launch": {"graph_ms_per_step": round(ms_mixed, 4), "no_graph_ms_per_step": round(ms_nograph, 4)},
        "fine_level": {"value": round(gdofs(fine_ms), 4), "unit": "GDOF/s", "ms_per_step": round(fine_ms, 4),
                       "what": "sum of the per-kernel event times of every cycle kernel except the coarse solve"},
        "time_to_tol_ms": round(tt_mixed, 3),
        "iters": info_mixed["iters"],
        "relres": info_mixed["relres_max"],
        "fp64": {"value": round(gdofs(ms_fp64), 4), "ms_per_step": round(ms_fp64, 4),
                 "time_to_tol_ms": round(tt_fp64, 3), "iters": info_fp64["iters"],
                 "relres": info_fp64["relres_max"],
                 "share_of_step": {k: round(v[0] / steps64 / ms_fp64, 3) for k, v in prof64.items() if v[1] > 0}},
        "speedup_vs_fp64": {"cycle": round(ms_fp64 / ms_mixed, 2), "time_to_tol": round(tt_fp64 / tt_mixed, 2)},
        "roofline": roofline,
        "e2e": {"value": round(gdofs(ms_e2e), 4), "unit": "GDOF/s", "ms_per_step": round(ms_e2e, 4),
                "h2d_bytes_per_step": 2 * N * 16, "d2h_bytes_per_step": N * 16},
        "gpu_launches": int(launches),
        "clocks": ck,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_cycles)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


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


def cpu_baseline(name, cycles):
    import numpy as np

    P, TG, f = oracle_setup(name)
    u = np.zeros_like(f)
    u = TG.step(u, f)  # warm
    t = time.perf_counter()
    for _ in range(cycles):
        u = TG.step(u, f)
    dt = (time.perf_counter() - t) / cycles
    return {"value": round(P.N / dt / 1e9, 6), "unit": "GDOF/s", "cores": 1, "kind": "oracle",
            "sample": f"{cycles} TwoGridStep cycles of the FP64 NumPy/SciPy oracle on the full {name} "
                      f"workload (set-up excluded; SuperLU local solves, CSR applies and the banded coarse "
                      f"solve are single-threaded), {dt * 1e3:.0f} ms per cycle"}


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
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
