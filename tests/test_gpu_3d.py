"""GPU parity in three dimensions (unit cube, Q2, fitted 27-point coarse
operator) against the FP64 oracle, through the C ABI.

Tolerances as in the 2-D parity tests: FP64 applies and transfers 1e-12,
smoother 1e-11, coarse solve and cycle 1e-9, FGMRES with the same iteration
count; the mixed form reaches the same 1e-8 residual."""
import numpy as np
import pytest

import synth
from oracle import dd, krylov, twogrid
from tests.common import ensure_built, relerr

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


CASES3 = [
    dict(n=4, l_dd=2, bc="robin", W=1.5, seed=5),
    dict(n=5, l_dd=2, bc={"xlo": "robin", "zhi": "robin", "yhi": "robin"}, W=1.2, seed=6),   # ragged blocks, mixed sides
    dict(n=6, l_dd=3, bc="robin", W=2.0, seed=7),
]
_ORACLE_BC = {"xlo": (2, 0), "xhi": (2, 1), "ylo": (1, 0), "yhi": (1, 1), "zlo": (0, 0), "zhi": (0, 1)}


def _case(c):
    n, p = c["n"], 2
    k = 2 * np.pi * c["W"] / synth.random_velocity(n, 3, c["seed"])
    eps = synth.absorbing_layer(n, 3, p, k, width_dofs=2)
    return n, p, k, eps


def _oracle_bc(bc):
    if isinstance(bc, str):
        return bc
    return {_ORACLE_BC[s]: v for s, v in bc.items()}


def build(th, c, nrhs=3, **kw):
    n, p, k, eps = _case(c)
    S = th.TwoGridSolver(n, p, k, eps, bc=c["bc"], alpha_s=kw.pop("alpha_s", 0.5), l_dd=c["l_dd"], nrhs_max=nrhs,
                         device=DEV, dim=3, **kw)
    P = twogrid.Problem(n, p, k, eps, bc=_oracle_bc(c["bc"]), dim=3, alpha_s=0.5)
    return S, P


@pytest.mark.parametrize("c", CASES3)
def test_fine_applies_3d(th, c):
    S, P = build(th, c)
    x = synth.random_complex((3, P.N), 1)
    for op, M in (("A", P.A), ("As", P.As)):
        assert relerr(host(S.apply(dev(x), op)), (M @ x.T).T) < 1e-12, op
    f = synth.random_complex((3, P.N), 2)
    assert relerr(host(S.residual(dev(f), dev(x))), f - (P.A @ x.T).T) < 1e-12


@pytest.mark.parametrize("c", CASES3)
def test_coarse_apply_transfers_and_solve_3d(th, c):
    S, P = build(th, c)
    xc = synth.random_complex((3, P.Nc), 3)
    assert relerr(host(S.apply(dev(xc), "Aq")), (P.Aq @ xc.T).T) < 1e-12
    r = synth.random_complex((3, P.N), 4)
    assert relerr(host(S.restrict(dev(r))), (P.IP.T @ r.T).T) < 1e-12
    u = synth.random_complex((3, P.N), 5)
    got = host(S.prolong(dev(xc), dev(u.copy()), omega=0.7))
    assert relerr(got, u + 0.7 * (P.IP @ xc.T).T) < 1e-12
    B = twogrid.BandedSolver(P.Aq)
    want = np.stack([B.solve(xc[i]) for i in range(3)])
    assert relerr(host(S.coarse_solve(dev(xc))), want) < 1e-9


@pytest.mark.parametrize("c", CASES3)
@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_smoother_3d(th, c, variant):
    S, P = build(th, c)
    S.set_variant("dd", "fp64", variant)
    sm = dd.DDSmoother(P, c["l_dd"])
    f = synth.random_complex((3, P.N), 6)
    u = synth.random_complex((3, P.N), 7)
    got = host(S.smooth(dev(f), dev(u.copy())))
    want = np.stack([sm.smooth(u[i], f[i], 1) for i in range(3)])
    assert relerr(got, want) < 1e-11
    S.device_status()


@pytest.mark.parametrize("c", CASES3[:2])
def test_cycle_3d(th, c):
    S, P = build(th, c)
    TG = twogrid.TwoGrid(P, l_dd=c["l_dd"])
    f = synth.random_complex((3, P.N), 9)
    u = synth.random_complex((3, P.N), 10)
    got = host(S.cycle(dev(f), dev(u.copy())))
    want = np.stack([TG.step(u[i], f[i]) for i in range(3)])
    assert relerr(got, want) < 1e-9
    # graph replay is bitwise the same
    a = dev(u.copy())
    b = dev(u.copy())
    S.cycle(dev(f), a)
    S.cycle_graph(dev(f), b)
    assert torch.equal(a, b)


def test_solve_3d_matches_oracle_iterations(th):
    w = synth.workload("cube2_q2_n8")
    S = th.TwoGridSolver(w["n"], w["p"], w["k"], w["eps"], alpha_s=0.5, l_dd=2, restart=40, device=DEV, dim=3)
    P = twogrid.Problem(w["n"], w["p"], w["k"], w["eps"], dim=3, alpha_s=0.5)
    TG = twogrid.TwoGrid(P, l_dd=2)
    xo, it, rr, _ = krylov.fgmres(lambda v: P.A @ v, TG.precondition, w["f"], tol=1e-8, restart=40)
    u, info = S.solve(dev(w["f"]))
    assert info["converged"] == 1 and info["relres_max"] <= 1e-8
    assert info["iters"] == it, (info["iters"], it)
    assert relerr(host(u), xo) < 1e-7


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_mixed_solve_3d(th, prec):
    w = synth.workload("cube2_q2_n8")
    S = th.TwoGridSolver(w["n"], w["p"], w["k"], w["eps"], alpha_s=0.5, l_dd=2, restart=40, prec=prec,
                         extra_prec=("fp64",), nrhs_max=2, device=DEV, dim=3)
    F = np.stack([w["f"], synth.random_complex(S.N, 40)])
    U, info = S.solve(dev(F))
    S.set_precision("fp64")
    U64, info64 = S.solve(dev(F))
    assert info["converged"] == 2 and info["relres_max"] <= 1e-8
    assert info["iters"] <= info64["iters"] + 2
    assert relerr(host(U), host(U64)) < 1e-6


@pytest.mark.parametrize("nrhs", [8, 13])
def test_tensor_core_smoother_3d(th, nrhs):
    """3-D subdomains (125 U-box rows x 729 columns) on the tensor cores: tiles
    of 16 right-hand sides (the doubled operand buffer of 32 exceeds shared
    memory), against the CUDA-core BF16 kernel and the FP64 smoother."""
    c = CASES3[0]  # 2-cell blocks: 5^3 = 125 U-box rows, 9^3 = 729 columns
    S, P = build(th, c, nrhs=nrhs, prec="bf16", extra_prec=("fp64",))
    f = synth.random_complex((nrhs, P.N), 70)
    u = synth.random_complex((nrhs, P.N), 71)
    S.set_precision("fp64")
    ref = host(S.smooth(dev(f), dev(u.copy()))) - u
    S.set_precision("bf16")
    S.set_variant("dd_batch", "fp32", 1)
    assert S.get_variant("dd_batch", "fp32") == 1
    tc = host(S.smooth(dev(f), dev(u.copy()))) - u
    S.device_status()
    S.set_variant("dd_batch", "fp32", 0)
    cc = host(S.smooth(dev(f), dev(u.copy()))) - u
    assert relerr(tc, cc) < 2e-2
    assert relerr(tc, ref) < 3e-2


def test_tensor_core_smoother_3d_64rhs_against_oracle(th):
    """64 right-hand sides (four tiles of 16) of the 3-D tensor-core products
    against the oracle's Algorithm 2 directly, per right-hand side."""
    c = CASES3[1]  # ragged blocks, mixed sides
    nrhs = 64
    S, P = build(th, c, nrhs=nrhs, prec="bf16")
    assert S.get_variant("dd_batch", "fp32") == 1
    sm = dd.DDSmoother(P, c["l_dd"])
    f = synth.random_complex((nrhs, P.N), 74)
    u = synth.random_complex((nrhs, P.N), 75)
    got = host(S.smooth(dev(f), dev(u.copy()))) - u
    S.device_status()
    want = np.stack([sm.smooth(u[i], f[i], 1) for i in range(nrhs)]) - u
    for i in range(nrhs):
        assert relerr(got[i], want[i]) < 3e-2, i


@pytest.mark.parametrize("variant", [0, 1, 3, 4, 5])
def test_mixed_smoother_3d_stream_variants(th, variant):
    """FP32 arithmetic on BF16 rows with 3-D gathers (z offsets in the column
    table): the streamed kernels, with and without paired FP32 FMAs, on a tile of
    four right-hand sides plus a ragged one, against the FP64 smoother."""
    c = CASES3[0]
    S, P = build(th, c, nrhs=5, prec="bf16", extra_prec=("fp64",))
    f = synth.random_complex((5, P.N), 72)
    u = synth.random_complex((5, P.N), 73)
    S.set_precision("fp64")
    ref = host(S.smooth(dev(f), dev(u.copy()))) - u
    S.set_precision("bf16")
    S.set_variant("dd_batch", "fp32", 0)
    S.set_variant("dd", "fp32", variant)
    got = host(S.smooth(dev(f), dev(u.copy()))) - u
    S.device_status()
    assert relerr(got, ref) < 2e-2


@pytest.mark.parametrize("c", CASES3[:2])
def test_mixed_outer_residual_double_single_3d(th, c):
    """The 3-D outer residual in double-single arithmetic, FP32 output: against
    the FP64 oracle within FP32 rounding plus 2^-40 of the terms' scale, also
    with u within 1e-9 of the solution (where f - A u cancels)."""
    import scipy.sparse.linalg as spla
    S, P = build(th, c, prec="fp32", extra_prec=("fp64",))
    assert S.get_variant("resid", "fp32") == 1
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
