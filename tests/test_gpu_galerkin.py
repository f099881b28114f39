"""GPU parity of standard Galerkin p-type coarsening ('gal', Section 4)
against the FP64 oracle, through the C ABI.

The coarse operator is I_P^T A_{alpha_c} I_P (the Q_{p/2} operator on the same
mesh), applied from its stencil and solved by the block sweep with the
set-up's explicit inverses.  Tolerances as for the QSFEM coarse level: FP64
apply 1e-12, coarse solve and two-grid cycle 1e-9, FGMRES the same iteration
count; FP32 apply 2e-6 and the mixed-precision solve reaches the same 1e-8."""
import numpy as np
import pytest

import synth
from oracle import krylov, twogrid
from tests.common import ensure_built, oracle_bc, relerr, small_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def th():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    import paper_2509_17494_gb300 as th
    return th


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    return t.cpu().numpy()


CASES = [
    dict(n=6, p=4, l_dd=2, bc="robin", alpha_c=0.02),
    dict(n=9, p=4, l_dd=3, bc={"xlo": "robin", "yhi": "robin"}, alpha_c=0.0),   # ragged blocks, mixed sides
    dict(n=12, p=2, l_dd=3, bc="robin", alpha_c=0.1),                           # p = 2: Q1 coarse space
    dict(n=5, p=6, l_dd=2, bc="neumann", alpha_c=0.05),                         # p = 6: Q3 coarse space
    dict(n=3, p=8, l_dd=2, bc={"ylo": "robin", "xhi": "robin"}, alpha_c=0.2),   # p = 8: Q4 coarse space
]


def build(th, c, nrhs=3, **kw):
    k, eps = small_case(n=c["n"], p=c["p"])
    S = th.TwoGridSolver(c["n"], c["p"], k, eps, bc=c["bc"], alpha_s=0.2, l_dd=c["l_dd"], nrhs_max=nrhs,
                         device=DEV, coarse="gal", alpha_c=c["alpha_c"], **kw)
    P = twogrid.Problem(c["n"], c["p"], k, eps, bc=oracle_bc(c["bc"]), alpha_s=0.2, coarse_kind="gal",
                        alpha_c=c["alpha_c"])
    return S, P


@pytest.mark.parametrize("c", CASES)
def test_gal_coarse_apply_and_solve_fp64(th, c):
    S, P = build(th, c)
    xc = synth.random_complex((3, P.Nc), 3)
    assert relerr(host(S.apply(dev(xc), "Aq")), (P.Aq @ xc.T).T) < 1e-12
    B = twogrid.BandedSolver(P.Aq)
    want = np.stack([B.solve(xc[i]) for i in range(3)])
    assert relerr(host(S.coarse_solve(dev(xc))), want) < 1e-9


@pytest.mark.parametrize("c", CASES)
def test_gal_cycle_fp64(th, c):
    S, P = build(th, c)
    TG = twogrid.TwoGrid(P, l_dd=c["l_dd"])
    f = synth.random_complex((3, P.N), 9)
    u = synth.random_complex((3, P.N), 10)
    got = host(S.cycle(dev(f), dev(u.copy())))
    want = np.stack([TG.step(u[i], f[i]) for i in range(3)])
    assert relerr(got, want) < 1e-9
    a, b = dev(u.copy()), dev(u.copy())
    S.cycle(dev(f), a)
    S.cycle_graph(dev(f), b)
    assert torch.equal(a, b)


def test_gal_solve_matches_oracle_iterations(th):
    w = synth.workload("square10_q4_n25")
    S = th.TwoGridSolver(w["n"], w["p"], w["k"], w["eps"], alpha_s=0.2, l_dd=2, restart=60, maxit=300, device=DEV,
                         coarse="gal", alpha_c=0.02)
    P = twogrid.Problem(w["n"], w["p"], w["k"], w["eps"], alpha_s=0.2, coarse_kind="gal", alpha_c=0.02)
    TG = twogrid.TwoGrid(P, l_dd=2)
    xo, it, rr, _ = krylov.fgmres(lambda v: P.A @ v, TG.precondition, w["f"], tol=1e-8, restart=60, maxit=300)
    x, info = S.solve(dev(w["f"]))
    assert info["iters"] == it, (info["iters"], it)
    assert info["relres_max"] <= 1e-8
    assert relerr(host(x), xo) < 1e-7


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_gal_mixed(th, prec):
    c = CASES[0]
    S, P = build(th, c, nrhs=2, prec=prec, extra_prec=("fp64",), restart=60, maxit=300)
    xc = dev(synth.random_complex((2, P.Nc), 19))
    assert relerr(host(S.apply(xc, "Aq", prec="fp32")), host(S.apply(xc, "Aq"))) < 2e-6
    F = synth.random_complex((2, P.N), 20)
    U, info = S.solve(dev(F))
    S.set_precision("fp64")
    U64, info64 = S.solve(dev(F))
    assert info["converged"] == 2 and info["relres_max"] <= 1e-8
    assert info["iters"] <= info64["iters"] + 2
    assert relerr(host(U), host(U64)) < 1e-6


def test_gal_unsupported_combinations(th):
    k, eps = small_case(n=4, p=4)
    with pytest.raises(th.ThError) as e:
        th.TwoGridSolver(4, 2, np.full((4, 4, 4), 5.0), None, dim=3, coarse="gal", device=DEV)
    assert e.value.code == 8   # TH_ERR_UNSUPPORTED
    S = th.TwoGridSolver(4, 4, k, eps, coarse="gal", device=DEV)
    with pytest.raises(th.ThError) as e:
        S.unet_init(np.zeros(th.unet_param_count(4, 16), np.float32), levels=4, base=16)
    assert e.value.code == 8


def test_no_coarse_correction_is_two_smoothings(th):
    """th_set_coarse(TH_COARSE_NONE) without a learned corrector: u_c = 0, so the
    cycle is the pre- and post-smoother alone (the paper's 'noCGC' rows)."""
    c = CASES[1]
    S, P = build(th, c)
    TG = twogrid.TwoGrid(P, l_dd=c["l_dd"])
    S.set_coarse("none")
    f = synth.random_complex((3, P.N), 31)
    u = synth.random_complex((3, P.N), 32)
    got = host(S.cycle(dev(f), dev(u.copy())))
    want = np.stack([TG.smooth(TG.smooth(u[i], f[i]), f[i]) for i in range(3)])
    assert relerr(got, want) < 1e-9
    S.set_coarse("direct")
    got = host(S.cycle(dev(f), dev(u.copy())))
    want = np.stack([TG.step(u[i], f[i]) for i in range(3)])
    assert relerr(got, want) < 1e-9
