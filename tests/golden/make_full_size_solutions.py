"""Writes tests/golden/full_size_solutions.json: sampled entries of the oracle's
solutions on the two largest workloads, for the full-size GPU parity tests.

Uses only the FP64 CPU oracle (oracle/) and the seeded inputs (synth/):
  * the 80-wavelength 801^2 Q4 grid (random k-field, 10-dof layer, Robin
    sides), the first three of its 64 seeded point sources;
  * the 10-wavelength 81^3 Q2 cube (random k-field, 10-dof layer, Robin
    sides), the first of its 8 seeded point sources.
Each solution is the oracle's right-preconditioned FGMRES (two-grid step of
Algorithm 1 with the CSDD smoother of Algorithm 2 and the QSFEM coarse level)
run to a relative residual of 1e-10, i.e. two orders below the 1e-8 the
library's solves stop at, so the stored values are the discrete solution
A^{-1} f up to (condition number) x 1e-10.  The 3-D coarse level is factored
by SuperLU instead of the banded LU (same solution, far less memory).

Stored per solution: 1000 seeded sample indices and the solution there, its
2-norm and max-norm, the oracle's iterations and final true residual.

Run once on a CPU (about 15-30 minutes, a few GB of memory):
    python tests/golden/make_full_size_solutions.py
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import krylov, twogrid  # noqa: E402

OUT = os.path.join(HERE, "full_size_solutions.json")
SAMPLES = 1000
TOL = 1e-10


def solve_case(name, sources, coarse_solver):
    w = synth.workload(name)
    t0 = time.time()
    P = twogrid.Problem(w["n"], w["p"], w["k"], w["eps"], dim=w["dim"], alpha_s=w["alpha_s"])
    TG = twogrid.TwoGrid(P, l_dd=w["l_dd"], coarse_solver=coarse_solver)
    print(f"{name}: set-up {time.time() - t0:.1f} s, N = {P.N}", flush=True)
    F = w["f"].reshape(-1, P.N)
    out = []
    for s in sources:
        t1 = time.time()
        x, it, rr, _ = krylov.fgmres(lambda v: P.A @ v, TG.precondition, F[s], tol=TOL, restart=60, maxit=400)
        idx = np.sort(synth.rng(7000 + s).choice(P.N, SAMPLES, replace=False))
        out.append({"workload": name, "source": int(s), "N": int(P.N), "tol": TOL, "iters": int(it),
                    "relres": float(rr), "norm2": float(np.linalg.norm(x)), "norm_inf": float(np.abs(x).max()),
                    "index": idx.tolist(), "re": x[idx].real.tolist(), "im": x[idx].imag.tolist()})
        print(f"  source {s}: {it} iterations, relres {rr:.2e}, {time.time() - t1:.1f} s", flush=True)
    return out


def main():
    cases = []
    cases += solve_case("square80_q4_n200", [0, 1, 2], "banded")
    cases += solve_case("cube10_q2_n40", [0], "splu")
    doc = {"generator": "tests/golden/make_full_size_solutions.py (FP64 CPU oracle only)",
           "method": "oracle FGMRES(60) with the oracle two-grid preconditioner to relres 1e-10",
           "cases": cases}
    with open(OUT, "w") as fh:
        json.dump(doc, fh, indent=0)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
