"""GPU parity: every hot-path step through the C ABI against the FP64 oracle.

Tolerances (relative, max-norm over the output):
  * FP64 operator applies (A, A_s, A_q), residual, transfers: 1e-12 (the
    arithmetic differs only in summation order);
  * FP64 smoother: 1e-11 (inverse rows from a banded LU vs SuperLU solves of
    subdomain systems with condition numbers below ~1e3);
  * FP64 coarse solve and two-grid cycle: 1e-9 (explicit block inverses vs
    banded LU on the coarse Helmholtz matrix, condition numbers up to ~1e6);
  * FP64 FGMRES: identical iteration count, solutions within 1e-7;
  * FP32 coarse solve: 1e-4; with the tensor-core separator and spike
    products (operands as two BF16 numbers, 2^-17 relative each): 2e-4;
  * FP32 applies: 2e-6; FP32 / FP16 / BF16 smoothers against the FP64
    smoother: 1e-5 / 2e-3 / 2e-2 (unit roundoff of the stored rows times the
    growth of a few-hundred-term sums); mixed-precision solves reach the same
    1e-8 residual and the oracle's solution within 1e-6.
"""
import numpy as np
import pytest

import synth
from oracle import dd, krylov, twogrid
from tests.common import ensure_built, oracle_bc, relerr, small_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def th():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    import paper_2509_17494_gb300 as th
    return th


DEV = "cuda:0"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    return t.cpu().numpy()


CASES = [
    dict(n=6, p=4, l_dd=2, bc="robin"),
    dict(n=9, p=4, l_dd=2, bc={"xlo": "robin", "yhi": "robin"}),     # ragged tile, mixed sides
    dict(n=20, p=2, l_dd=3, bc="robin"),                             # p = 2, ragged tiles and blocks
    dict(n=5, p=6, l_dd=2, bc="neumann"),                            # p = 6, Neumann (layer absorbs)
    dict(n=5, p=8, l_dd=2, bc={"ylo": "robin", "xhi": "robin"}),     # p = 8
    dict(n=25, p=4, l_dd=4, bc="robin"),                             # 4/3 block sizes
    dict(n=9, p=4, l_dd=2, bc={"xlo": "dirichlet", "ylo": "dirichlet", "xhi": "robin", "yhi": "robin"}),
    dict(n=10, p=2, l_dd=3, bc="dirichlet"),                         # Gamma_0 all round, damping layer only
]


def build(th, c, nrhs=3, **kw):
    k, eps = small_case(n=c["n"], p=c["p"])
    S = th.TwoGridSolver(c["n"], c["p"], k, eps, bc=c["bc"], alpha_s=kw.pop("alpha_s", 0.5), l_dd=c["l_dd"],
                         nrhs_max=nrhs, device=DEV, **kw)
    P = twogrid.Problem(c["n"], c["p"], k, eps, bc=oracle_bc(c["bc"]), alpha_s=0.5)
    return S, P


@pytest.mark.parametrize("c", CASES)
def test_fine_applies_fp64(th, c):
    S, P = build(th, c)
    x = synth.random_complex((3, P.N), 1)
    for op, M in (("A", P.A), ("As", P.As)):
        y = host(S.apply(dev(x), op))
        want = (M @ x.T).T
        assert relerr(y, want) < 1e-12, op
    f = synth.random_complex((3, P.N), 2)
    r = host(S.residual(dev(f), dev(x)))
    assert relerr(r, f - (P.A @ x.T).T) < 1e-12


@pytest.mark.parametrize("c", CASES)
def test_coarse_apply_and_transfers_fp64(th, c):
    S, P = build(th, c)
    xc = synth.random_complex((3, P.Nc), 3)
    assert relerr(host(S.apply(dev(xc), "Aq")), (P.Aq @ xc.T).T) < 1e-12
    r = synth.random_complex((3, P.N), 4)
    assert relerr(host(S.restrict(dev(r))), (P.IP.T @ r.T).T) < 1e-12
    u = synth.random_complex((3, P.N), 5)
    got = host(S.prolong(dev(xc), dev(u.copy()), omega=0.7))
    assert relerr(got, u + 0.7 * (P.IP @ xc.T).T) < 1e-12


@pytest.mark.parametrize("c", CASES)
@pytest.mark.parametrize("variant", [0, 1])
def test_fine_apply_variants_fp64(th, c, variant):
    S, P = build(th, c)
    S.set_variant("fine", "fp64", variant)
    x = synth.random_complex((3, P.N), 31)
    assert relerr(host(S.apply(dev(x), "As")), (P.As @ x.T).T) < 1e-12


@pytest.mark.parametrize("c", CASES)
@pytest.mark.parametrize("n_dd", [1, 2])
@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_smoother_fp64(th, c, n_dd, variant):
    S, P = build(th, c, n_dd=n_dd)
    S.set_variant("dd", "fp64", variant)
    sm = dd.DDSmoother(P, c["l_dd"])
    f = synth.random_complex((3, P.N), 6)
    u = synth.random_complex((3, P.N), 7)
    got = host(S.smooth(dev(f), dev(u.copy())))
    want = np.stack([sm.smooth(u[i], f[i], n_dd) for i in range(3)])
    assert relerr(got, want) < 1e-11
    S.device_status()


def test_smoother_large_subdomains_fp64(th):
    """U boxes above 512 nodes (4 cells of order 6: 25^2 = 625 rows) run the
    1024-thread subdomain kernel."""
    c = dict(n=9, p=6, l_dd=4, bc="robin")
    S, P = build(th, c)
    sm = dd.DDSmoother(P, c["l_dd"])
    f = synth.random_complex((3, P.N), 61)
    u = synth.random_complex((3, P.N), 62)
    got = host(S.smooth(dev(f), dev(u.copy())))
    want = np.stack([sm.smooth(u[i], f[i], 1) for i in range(3)])
    assert relerr(got, want) < 1e-11
    S.device_status()


@pytest.mark.parametrize("c", CASES)
@pytest.mark.parametrize("variant", [0, 1])
def test_coarse_solve_fp64(th, c, variant):
    S, P = build(th, c, nrhs=1)
    S.set_variant("coarse", "fp64", variant)
    B = twogrid.BandedSolver(P.Aq)
    for seed in (8, 9):
        rc = synth.random_complex(P.Nc, seed)
        got = host(S.coarse_solve(dev(rc)))
        assert relerr(got, B.solve(rc)) < 1e-9


@pytest.mark.parametrize("c", CASES)
def test_coarse_solve_fp32_sweep_variants(th, c):
    """The FP32 one-rhs coarse solve: the three chunk-sweep variants (two
    phases, one cluster barrier per step, st.async row exchange on mbarriers)
    do the same arithmetic in the same order, so they agree bitwise; against
    the oracle within FP32 rounding of the explicit-inverse sweep."""
    S, P = build(th, c, nrhs=1, prec="fp32", extra_prec=("fp64",))
    B = twogrid.BandedSolver(P.Aq)
    rc = dev(synth.random_complex(P.Nc, 8))
    outs = []
    for v in (0, 1, 2):
        S.set_variant("coarse", "fp32", v)
        outs.append(S.coarse_solve(rc))
        S.device_status()
    assert relerr(host(outs[0]), B.solve(host(rc))) < 1e-4
    assert torch.equal(outs[1], outs[2])
    assert relerr(host(outs[0]), host(outs[1])) < 1e-5


@pytest.mark.parametrize("c", CASES)
def test_coarse_solve_symmetric_separator_product(th, c):
    """One right-hand side in FP32: the separator values from the upper triangle
    of the complex-symmetric reduced inverse (TH_K_SEP_SYM 1, default; 64 x 64
    blocks serving S_IJ x_J and S_IJ^T x_I) against the full GEMV (0): the same
    products in another summation order, FP32 rounding apart (1e-5), and both
    against the oracle's banded LU (1e-4)."""
    S, P = build(th, c, nrhs=1, prec="fp32", extra_prec=("fp64",))
    assert S.get_variant("sep_sym", "fp32") == 1
    B = twogrid.BandedSolver(P.Aq)
    rc = synth.random_complex(P.Nc, 12)
    want = B.solve(rc)
    sym = host(S.coarse_solve(dev(rc)))
    S.device_status()
    S.set_variant("sep_sym", "fp32", 0)
    full = host(S.coarse_solve(dev(rc)))
    assert relerr(sym, full) < 1e-5
    assert relerr(sym, want) < 1e-4 and relerr(full, want) < 1e-4


@pytest.mark.parametrize("chunks", [2, 5])
def test_coarse_solve_chunk_count(th, chunks):
    """th_params.coarse_chunks sets the partition's chunk count P (2 P - 1 <= m_c):
    FP64 against the oracle's banded LU (1e-9) and the solve to 1e-8."""
    c = CASES[5]
    S, P = build(th, c, nrhs=1, coarse_chunks=chunks)
    B = twogrid.BandedSolver(P.Aq)
    rc = synth.random_complex(P.Nc, 13)
    assert relerr(host(S.coarse_solve(dev(rc))), B.solve(rc)) < 1e-9
    X, info = S.solve(dev(synth.random_complex(P.N, 14)))
    assert info["relres_max"] <= 1e-8


@pytest.mark.parametrize("c", [CASES[0], CASES[2], CASES[5]])
@pytest.mark.parametrize("nrhs", [2, 11])
def test_coarse_solve_many_rhs(th, c, nrhs):
    """Tiles of right-hand sides (ragged: 2 and 8 + 3) in FP64 against the
    oracle, and in FP32 (the mixed cycle's coarse solve) against FP64 and
    against the FP32 one-right-hand-side sweep (same products, other
    summation order: a few FP32 roundings times the coarse condition number)."""
    S, P = build(th, c, nrhs=nrhs, prec="fp64", extra_prec=("fp32",))
    S.set_variant("coarse_multi", "fp32", 1)  # FP32 products (the tensor-core ones: test below)
    rc = synth.random_complex((nrhs, P.Nc), 31)
    B = twogrid.BandedSolver(P.Aq)
    want = np.stack([B.solve(rc[i]) for i in range(nrhs)])
    got64 = host(S.coarse_solve(dev(rc)))
    assert relerr(got64, want) < 1e-9
    S.set_precision("fp32")
    got32 = host(S.coarse_solve(dev(rc)))
    one32 = np.stack([host(S.coarse_solve(dev(rc[i]))) for i in range(nrhs)])
    assert relerr(got32, want) < 1e-4
    assert relerr(got32, one32) < 1e-5
    again = host(S.coarse_solve(dev(rc)))
    assert np.array_equal(again, got32)


@pytest.mark.parametrize("c", [CASES[0], CASES[2], CASES[5]])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_coarse_solve_column_groups(th, c, prec):
    """Eight or more right-hand sides: the sweep in groups of 8 per CTA (variant
    1, the FP64 default), the per-tile cluster sweep (variant 0) and, in the
    mixed form, the column-group sweep with the tensor-core separator and spike
    products (variant 2, its default), on two full groups and a ragged one,
    against the oracle's banded LU (FP64 1e-9, FP32 1e-4, split BF16 2e-4)."""
    nrhs = 20
    extra = ("fp64",) if prec != "fp64" else ()
    S, P = build(th, c, nrhs=nrhs, prec=prec, extra_prec=extra)
    assert S.get_variant("coarse_multi", prec) == (1 if prec == "fp64" else 2)
    assert S.get_variant("coarse_refine", prec) == 0  # small grids: the FP32 solve is accurate
    rc = synth.random_complex((nrhs, P.Nc), 33)
    B = twogrid.BandedSolver(P.Aq)
    want = np.stack([B.solve(rc[i]) for i in range(nrhs)])
    outs = []
    for v in ((1, 0) if prec == "fp64" else (2, 1, 0)):
        tol = 1e-9 if prec == "fp64" else (2e-4 if v == 2 else 1e-4)
        S.set_variant("coarse_multi", prec, v)
        outs.append(host(S.coarse_solve(dev(rc))))
        S.device_status()
        for i in range(nrhs):
            assert relerr(outs[-1][i], want[i]) < tol, (v, i)
    again = host(S.coarse_solve(dev(rc)))
    assert np.array_equal(again, outs[-1])


@pytest.mark.parametrize("c", CASES)
def test_coarse_solve_tensor_core_products(th, c):
    """Variant 2 of the grouped coarse solve on 70 right-hand sides (a full group
    of 64 and a ragged one of 6): the FP32 column-group sweep, then the separator
    product and the spike correction on the tensor cores with every operand as
    two BF16 numbers (hi + lo: 2^-17 relative each, sums over at most a few
    hundred terms, amplified about tenfold by the chunk systems of these grids:
    2e-4), against the oracle's banded LU; bitwise repeatable; and the FGMRES
    solve on 12 right-hand sides takes the iterations of variant 1."""
    nrhs = 70
    S, P = build(th, c, nrhs=nrhs, prec="bf16", extra_prec=("fp64",))
    assert S.get_variant("coarse_multi", "fp32") == 2
    rc = synth.random_complex((nrhs, P.Nc), 34)
    B = twogrid.BandedSolver(P.Aq)
    want = np.stack([B.solve(rc[i]) for i in range(nrhs)])
    got = host(S.coarse_solve(dev(rc)))
    S.device_status()
    for i in range(nrhs):
        assert relerr(got[i], want[i]) < 2e-4, i
    assert np.array_equal(host(S.coarse_solve(dev(rc))), got)
    F = dev(synth.random_complex((12, P.N), 35))
    X2, i2 = S.solve(F)
    S.set_variant("coarse_multi", "fp32", 1)
    X1, i1 = S.solve(F)
    assert i2["relres_max"] <= 1e-8 and i1["relres_max"] <= 1e-8
    assert i2["iters"] == i1["iters"]
    assert relerr(host(X2), host(X1)) < 1e-7


@pytest.mark.parametrize("c", [CASES[1], CASES[6]])
@pytest.mark.parametrize("nrhs", [1, 9])
def test_coarse_refinement_steps(th, c, nrhs):
    """Iterative refinement of the mixed form's coarse solve (TH_K_COARSE_REFINE):
    each step z = r_c - A_q u_c (FP32), the same solve of z, u_c += its solution,
    contracts the error of the FP32 solve (here about 1e-6 relative, so the
    refined solve reaches the FP32 residual's level, 1e-6), for one right-hand
    side and for the grouped tensor-core path."""
    S, P = build(th, c, nrhs=nrhs, prec="bf16", extra_prec=("fp64",))
    rc = synth.random_complex((nrhs, P.Nc), 36)
    B = twogrid.BandedSolver(P.Aq)
    want = np.stack([B.solve(rc[i]) for i in range(nrhs)])
    errs = []
    for r in (0, 1, 2):
        S.set_variant("coarse_refine", "fp32", r)
        assert S.get_variant("coarse_refine", "fp32") == r
        got = host(S.coarse_solve(dev(rc)))
        S.device_status()
        errs.append(max(relerr(got[i], want[i]) for i in range(nrhs)))
    assert errs[0] < 2e-4
    assert errs[1] < 2e-6 and errs[2] < 2e-6, errs
    F = dev(synth.random_complex((nrhs, P.N), 37))
    S.set_variant("coarse_refine", "fp32", 1)
    X, info = S.solve(F)
    assert info["relres_max"] <= 1e-8


@pytest.mark.parametrize("c", CASES)
@pytest.mark.parametrize("n_s,omega_c", [(1, 1.0), (2, 0.8)])
def test_cycle_fp64(th, c, n_s, omega_c):
    S, P = build(th, c, n_s=n_s, omega_c=omega_c)
    TG = twogrid.TwoGrid(P, l_dd=c["l_dd"], n_s=n_s, omega_c=omega_c)
    f = synth.random_complex((3, P.N), 9)
    u = synth.random_complex((3, P.N), 10)
    got = host(S.cycle(dev(f), dev(u.copy())))
    want = np.stack([TG.step(u[i], f[i]) for i in range(3)])
    assert relerr(got, want) < 1e-9


@pytest.mark.parametrize("c", CASES)
@pytest.mark.parametrize("prec,nrhs", [("bf16", 3), ("fp32", 2), ("bf16", 9)])
def test_fused_cycle_bitwise_equals_step_by_step(th, c, prec, nrhs):
    """The fused launch structure of the cycle (the average folded into the next
    fine apply, the prolongation into the post-smoother's, the last average with
    the update and the widening into one kernel) does the step-by-step
    arithmetic in the same order: bitwise equal cycles (mixed form) and
    preconditioned solves (FP64 form, whose preconditioner is the fused step)."""
    S, P = build(th, c, nrhs=nrhs, prec=prec, extra_prec=("fp64",))
    f = dev(synth.random_complex((nrhs, P.N), 90))
    u0 = synth.random_complex((nrhs, P.N), 91)
    outs = []
    for v in (0, 1, 2):   # 2: the fused launches with programmatic dependencies
        S.set_variant("cycle", "fp32", v)
        outs.append(S.cycle(f, dev(u0.copy())))
        outs.append(S.cycle_graph(f, dev(u0.copy())))
        S.device_status()
    for o in outs[1:]:
        assert torch.equal(outs[0], o)
    S.set_precision("fp64")
    sols = []
    for v in (0, 1, 2):
        S.set_variant("cycle", "fp64", v)
        x, info = S.solve(f)
        sols.append((x, info["iters"]))
    for x, it in sols[1:]:
        assert it == sols[0][1] and torch.equal(x, sols[0][0])


def test_cycle_is_deterministic(th):
    S, P = build(th, CASES[1])
    f = dev(synth.random_complex((3, P.N), 11))
    u1 = dev(synth.random_complex((3, P.N), 12))
    u2 = u1.clone()
    S.cycle(f, u1)
    S.cycle(f, u2)
    assert torch.equal(u1, u2)


@pytest.mark.parametrize("name,alpha_s,l_dd", [("square10_q4_n25", 0.5, 2), ("square10_q4_n25", 0.2, 4)])
def test_solve_matches_oracle_iterations(th, name, alpha_s, l_dd):
    w = synth.workload(name)
    S = th.TwoGridSolver(w["n"], w["p"], w["k"], w["eps"], alpha_s=alpha_s, l_dd=l_dd, restart=40, device=DEV)
    P = twogrid.Problem(w["n"], w["p"], w["k"], w["eps"], alpha_s=alpha_s)
    TG = twogrid.TwoGrid(P, l_dd=l_dd)
    xo, it, rr, _ = krylov.fgmres(lambda v: P.A @ v, TG.precondition, w["f"], tol=1e-8, restart=40)
    x, info = S.solve(dev(w["f"]))
    assert info["iters"] == it
    assert info["relres_max"] <= 1e-8
    assert relerr(host(x), xo) < 1e-7


@pytest.mark.parametrize("bc", [{"xlo": "dirichlet", "ylo": "dirichlet", "xhi": "robin", "yhi": "robin"},
                                {"xlo": "dirichlet", "xhi": "dirichlet", "ylo": "robin", "yhi": "robin"}])
def test_dirichlet_solve_matches_oracle(th, bc):
    """Dirichlet sides (Section 2, u = 0 on Gamma_0): the FP64 solve takes the
    oracle's FGMRES iterations and lands within 1e-7 of its solution; the mixed
    form reaches 1e-8 and the exact solution within 1e-6; u is zero on Gamma_0."""
    import scipy.sparse.linalg as spla
    n, p = 16, 4
    k, eps = small_case(n=n, p=p, W=4.0, seed=11)
    S = th.TwoGridSolver(n, p, k, eps, bc=bc, alpha_s=0.5, l_dd=2, prec="bf16", extra_prec=("fp64",), restart=40,
                         device=DEV)
    P = twogrid.Problem(n, p, k, eps, bc=oracle_bc(bc), alpha_s=0.5)
    TG = twogrid.TwoGrid(P, l_dd=2)
    f = synth.gaussian_source(n, p, 2)
    f[P.dmask] = 0.0   # the data vanish on Gamma_0 (the Gaussian's far tail would leave tiny values there)
    xo, it, rr, _ = krylov.fgmres(lambda v: P.A @ v, TG.precondition, f, tol=1e-8, restart=40)
    S.set_precision("fp64")
    x, info = S.solve(dev(f))
    assert info["iters"] == it and relerr(host(x), xo) < 1e-7
    assert np.all(host(x)[P.dmask] == 0)
    S.set_precision("bf16")
    xm, infom = S.solve(dev(f))
    assert infom["relres_max"] <= 1e-8 and infom["iters"] <= it + 2
    xs = spla.spsolve(P.A.tocsc(), f)
    assert np.linalg.norm(host(xm) - xs) / np.linalg.norm(xs) < 1e-6


def test_solve_multiple_rhs_and_restart(th):
    c = CASES[0]
    S, P = build(th, c, nrhs=4, restart=5, maxit=300)
    TG = twogrid.TwoGrid(P, l_dd=c["l_dd"])
    F = synth.random_complex((4, P.N), 13)
    X, info = S.solve(dev(F))
    assert info["converged"] == 4 and info["relres_max"] <= 1e-8
    for i in range(4):
        xo, it, rr, _ = krylov.fgmres(lambda v: P.A @ v, TG.precondition, F[i], tol=1e-8, restart=5, maxit=300)
        assert info["iters_per_rhs"][i] == it
        assert relerr(host(X)[i], xo) < 1e-7


def test_host_buffer_entry_points(th):
    S, P = build(th, CASES[0], nrhs=1)
    f = synth.random_complex(P.N, 14)
    u = synth.random_complex(P.N, 15)
    ud = host(S.cycle(dev(f), dev(u.copy())))
    uh = u.copy()
    S.cycle_host(f, uh)
    assert np.array_equal(uh, ud)
    xh, info = S.solve_host(f)
    xd, info2 = S.solve(dev(f))
    assert info["iters"] == info2["iters"] and np.array_equal(xh, host(xd))


# ------------------------------------------------------------ mixed precision
@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp16", 2e-3), ("bf16", 2e-2)])
@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5])
def test_mixed_smoother_close_to_fp64(th, prec, tol, variant):
    c = CASES[5]
    S, P = build(th, c, prec=prec, extra_prec=("fp64",))
    S.set_variant("dd", "fp32", variant)
    S.set_variant("fine", "fp32", min(variant, 1))
    f = dev(synth.random_complex((3, P.N), 16))
    u = synth.random_complex((3, P.N), 17)
    S.set_precision("fp64")
    ref = S.smooth(f, dev(u.copy())) - dev(u)
    S.set_precision(prec)
    got = S.smooth(f, dev(u.copy())) - dev(u)
    assert relerr(host(got), host(ref)) < tol
    x = dev(synth.random_complex((3, P.N), 18))
    assert relerr(host(S.apply(x, "A", prec="fp32")), host(S.apply(x, "A"))) < 2e-6
    xc = dev(synth.random_complex((3, P.Nc), 19))
    assert relerr(host(S.apply(xc, "Aq", prec="fp32")), host(S.apply(xc, "Aq"))) < 2e-6


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_mixed_solve_reaches_tolerance(th, prec):
    w = synth.workload("square10_q4_n25")
    S = th.TwoGridSolver(w["n"], w["p"], w["k"], w["eps"], alpha_s=0.5, l_dd=2, prec=prec,
                         extra_prec=("fp64",), restart=40, device=DEV)
    P = twogrid.Problem(w["n"], w["p"], w["k"], w["eps"], alpha_s=0.5)
    import scipy.sparse.linalg as spla
    xs = spla.spsolve(P.A.tocsc(), w["f"])
    x, info = S.solve(dev(w["f"]))
    S.set_precision("fp64")
    x64, info64 = S.solve(dev(w["f"]))
    assert info["relres_max"] <= 1e-8
    assert info["iters"] <= info64["iters"] + 2
    assert relerr(host(x), xs) < 1e-6


@pytest.mark.parametrize("c", [CASES[5], CASES[6]])
def test_mixed_solve_double_single_products(th, c):
    """The mixed form's FGMRES products A z in double-single arithmetic with FP64
    output (variant 1, default) against the FP64 apply (variant 0): the same
    iterations (within one), the same 1e-8 true residual, solutions within
    1e-9 of each other (the products differ by ~1e-14 relative)."""
    S, P = build(th, c, nrhs=2, prec="bf16", extra_prec=("fp64",), restart=40)
    F = dev(synth.random_complex((2, P.N), 95))
    assert S.get_variant("az", "fp32") == 1
    X1, i1 = S.solve(F)
    S.set_variant("az", "fp32", 0)
    X0, i0 = S.solve(F)
    assert i1["relres_max"] <= 1e-8 and i0["relres_max"] <= 1e-8
    assert abs(i1["iters"] - i0["iters"]) <= 1
    assert relerr(host(X1), host(X0)) < 1e-8


@pytest.mark.parametrize("c", [CASES[0], CASES[4], CASES[6]])
def test_mixed_solve_double_single_krylov(th, c):
    """The mixed forms' Gram-Schmidt dots, norms and updates in double-single
    arithmetic (TH_K_KRYLOV 1, default; about 2^-44 relative) against FP64
    (variant 0): the same iterations and residuals, solutions within 1e-9,
    over a restart (restart 4)."""
    S, P = build(th, c, nrhs=3, prec="bf16", extra_prec=("fp64",), restart=4, maxit=200)
    F = dev(synth.random_complex((3, P.N), 96))
    assert S.get_variant("krylov", "fp32") == 1
    X1, i1 = S.solve(F)
    S.set_variant("krylov", "fp32", 0)
    X0, i0 = S.solve(F)
    assert i1["relres_max"] <= 1e-8 and i0["relres_max"] <= 1e-8
    assert i1["iters"] == i0["iters"]
    assert relerr(host(X1), host(X0)) < 1e-9
    x = host(X1)
    f = host(F)
    for r in range(3):
        assert np.linalg.norm(f[r] - P.A @ x[r]) / np.linalg.norm(f[r]) <= 1.01e-8


# ------------------------------------------------------------ full-size, sampled
def test_full_size_apply_and_cycle(th):
    """40-wavelength 401^2 workload: the apply at full size and one cycle compared on sampled nodes."""
    w = synth.workload("square40_q4_n100")
    S = th.TwoGridSolver(w["n"], w["p"], w["k"], w["eps"], alpha_s=0.5, l_dd=2, device=DEV)
    P = twogrid.Problem(w["n"], w["p"], w["k"], w["eps"], alpha_s=0.5)
    x = synth.random_complex(P.N, 20)
    assert relerr(host(S.apply(dev(x), "A")), P.A @ x) < 1e-12
    TG = twogrid.TwoGrid(P, l_dd=2)
    f = w["f"]
    got = host(S.cycle(dev(f), dev(np.zeros_like(f))))
    want = TG.step(np.zeros_like(f), f)
    idx = synth.rng(21).integers(0, P.N, 4000)
    assert relerr(got[idx], want[idx]) < 1e-9


# ------------------------------------------------------------ batched, tensor cores
@pytest.mark.parametrize("nrhs", [8, 40])
def test_batched_tensor_core_smoother(th, nrhs):
    """BF16 subdomain products for many right-hand sides on tcgen05: the same
    rows as the CUDA-core BF16 kernel, with the residuals also rounded to BF16
    (both tcgen05 operands of the f16 kind share one type).  That rounding is
    2^-9 relative per entry, the same as the rows' own, so the tensor-core and
    CUDA-core results agree within the BF16-vs-FP64 smoother tolerance (2e-2)
    and the tensor-core result stays within 1.5x of it from FP64."""
    c = CASES[1]
    S, P = build(th, c, nrhs=nrhs, prec="bf16", extra_prec=("fp64",))
    f = dev(synth.random_complex((nrhs, P.N), 50))
    u = synth.random_complex((nrhs, P.N), 51)
    S.set_precision("fp64")
    ref = host(S.smooth(f, dev(u.copy()))) - u
    S.set_precision("bf16")
    S.set_variant("dd_batch", "fp32", 1)
    assert S.get_variant("dd_batch", "fp32") == 1
    tc = host(S.smooth(f, dev(u.copy()))) - u
    S.device_status()
    S.set_variant("dd_batch", "fp32", 0)
    cc = host(S.smooth(f, dev(u.copy()))) - u
    assert relerr(tc, cc) < 2e-2
    assert relerr(tc, ref) < 3e-2
    # deterministic
    S.set_variant("dd_batch", "fp32", 1)
    tc2 = host(S.smooth(f, dev(u.copy()))) - u
    assert np.array_equal(tc, tc2)


@pytest.mark.parametrize("c", [CASES[1], CASES[0]])
def test_tensor_core_smoother_64rhs_against_oracle(th, c):
    """64 right-hand sides (two full 32-wide tiles of the tcgen05 kernel) against
    the oracle's Algorithm 2 (SuperLU subdomain solves) directly, per
    right-hand side, at the BF16 tolerance of the smoother tests: rows and
    residuals rounded to BF16 (2^-9 relative each), FP32 accumulation."""
    nrhs = 64
    S, P = build(th, c, nrhs=nrhs, prec="bf16")
    assert S.get_variant("dd_batch", "fp32") == 1
    sm = dd.DDSmoother(P, c["l_dd"])
    f = synth.random_complex((nrhs, P.N), 52)
    u = synth.random_complex((nrhs, P.N), 53)
    got = host(S.smooth(dev(f), dev(u.copy()))) - u
    S.device_status()
    want = np.stack([sm.smooth(u[i], f[i], 1) for i in range(nrhs)]) - u
    for i in range(nrhs):
        assert relerr(got[i], want[i]) < 3e-2, i


def test_batched_tensor_core_solve(th):
    w = synth.workload("square10_q4_n25")
    nrhs = 16
    F = synth.random_sources(w["n"], w["p"], 2, nrhs, seed=60)
    S = th.TwoGridSolver(w["n"], w["p"], w["k"], w["eps"], alpha_s=0.5, l_dd=2, prec="bf16",
                         extra_prec=("fp64",), restart=40, nrhs_max=nrhs, device=DEV)
    X, info = S.solve(dev(F))
    S.device_status()
    assert info["converged"] == nrhs and info["relres_max"] <= 1e-8
    S.set_precision("fp64")
    X64, info64 = S.solve(dev(F))
    assert info["iters"] <= info64["iters"] + 2
    assert relerr(host(X), host(X64)) < 1e-6


# ------------------------------------------------- the mixed form's outer residual
@pytest.mark.parametrize("c", CASES)
def test_mixed_outer_residual_double_single(th, c):
    """r = f - A u in double-single arithmetic, rounded to FP32: against the FP64
    oracle, within FP32 rounding of r plus 2^-40 of the terms' scale |A| |u|
    (about 20 double-single operations of relative error 2^-46 on the longest
    path); with u near the solution (r ~ 1e-9 |f|) that second term is what
    remains, and a float-only apply (2^-24) would miss it by far."""
    S, P = build(th, c, prec="fp32", extra_prec=("fp64",))
    assert S.get_variant("resid", "fp32") == 1
    import scipy.sparse.linalg as spla
    f = synth.random_complex((3, P.N), 41)
    u = synth.random_complex((3, P.N), 42)
    uex = np.stack([spla.spsolve(P.A.tocsc(), f[i]) for i in range(3)])
    Aabs = abs(P.A)
    for uu in (u, uex * (1 + 1e-9 * synth.random_complex(P.N, 43).real)):
        want = f - (P.A @ uu.T).T
        got = host(S.residual_mixed(dev(f), dev(uu)))
        scale = (Aabs @ np.abs(uu).T).T.max() + np.abs(f).max()
        err = np.abs(got - want).max()
        assert err <= 1.2e-7 * np.abs(want).max() + 2.0 ** -40 * scale, (err, np.abs(want).max(), scale)
    # the FP64 variant of the same step agrees
    S.set_variant("resid", "fp32", 0)
    got0 = host(S.residual_mixed(dev(f), dev(u)))
    S.set_variant("resid", "fp32", 1)
    got1 = host(S.residual_mixed(dev(f), dev(u)))
    assert relerr(got1, got0) < 2e-7


def test_coarse_solve_column_groups_large_grid(th):
    """64 right-hand sides on a 401^2 coarse grid (20 chunks): groups of 10 per
    CTA (7 groups, the last one ragged) so that 20 x 7 CTAs fit the SMs once;
    FP64 against the FP64 one-right-hand-side solve, FP32 (FP32 or split-BF16
    tensor-core products) within its own accuracy on this grid, one
    refinement step within 2e-5, and FP64 by the coarse residual."""
    n, p = 200, 4
    k = synth.random_wavenumber(n, 2, 20.0, seed=5)
    eps = synth.absorbing_layer(n, 2, p, k, 10.0)
    S = th.TwoGridSolver(n, p, k, eps, alpha_s=0.5, l_dd=4, prec="fp32", extra_prec=("fp64",), nrhs_max=64,
                         restart=2, device=DEV)
    rc = dev(synth.random_complex((64, S.Nc), 82))
    S.set_precision("fp64")
    many = S.coarse_solve(rc)
    S.device_status()
    one = torch.stack([S.coarse_solve(rc[i].contiguous()) for i in (0, 37, 63)])
    assert relerr(host(many)[[0, 37, 63]], host(one)) < 1e-10
    res = S.apply(many, "Aq") - rc
    assert float(torch.linalg.norm(res) / torch.linalg.norm(rc)) < 1e-9
    S.set_precision("fp32")
    S.set_variant("coarse_refine", "fp32", 0)
    for v in (1, 2):  # FP32 products, then the split-BF16 tensor-core products
        S.set_variant("coarse_multi", "fp32", v)
        m32 = S.coarse_solve(rc)
        S.device_status()
        for i in range(64):
            assert relerr(host(m32[i]), host(many[i])) < 5e-3, (v, i)
    # one refinement step on the FP32 residual: about the FP32 residual's level
    S.set_variant("coarse_refine", "fp32", 1)
    m32 = S.coarse_solve(rc)
    S.device_status()
    for i in range(64):
        assert relerr(host(m32[i]), host(many[i])) < 2e-5, i


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_coarse_solve_many_rhs_large_grid(th, prec):
    """A 401^2 coarse grid (200^2 Q4 cells): the multi-rhs sweep takes narrower
    tiles (its buffers for 8 / 4 columns exceed shared memory).  Checked against
    the one-rhs solves of each column and by the coarse residual with the
    (separately parity-tested) coarse apply."""
    n, p = 200, 4
    k = synth.random_wavenumber(n, 2, 20.0, seed=5)
    eps = synth.absorbing_layer(n, 2, p, k, 10.0)
    extra = ("fp64",) if prec != "fp64" else ()
    S = th.TwoGridSolver(n, p, k, eps, alpha_s=0.5, l_dd=4, prec=prec, extra_prec=extra, nrhs_max=5, device=DEV)
    rc = dev(synth.random_complex((5, S.Nc), 81))
    many = S.coarse_solve(rc)
    S.device_status()
    one = torch.stack([S.coarse_solve(rc[i].contiguous()) for i in range(5)])
    res = S.apply(many, "Aq") - rc
    rel = float(torch.linalg.norm(res) / torch.linalg.norm(rc))
    if prec == "fp64":
        assert relerr(host(many), host(one)) < 1e-10
        assert rel < 1e-9
    else:
        # FP32 explicit block inverses on a 401-row coarse grid: the error against the
        # FP64 solve is unit roundoff times the growth of the block sweep (measured on a
        # GB300: 5e-5..2e-4 for the one-column sweep, 3e-4..9e-4 for the tiled sweep,
        # whose per-warp column chains are longer); a wrong tile, column or block
        # would be O(1)
        S.set_precision("fp64")
        exact = S.coarse_solve(rc)
        for i in range(5):
            assert relerr(host(one[i]), host(exact[i])) < 2e-3
            assert relerr(host(many[i]), host(exact[i])) < 5e-3
        assert rel < 5e-3
