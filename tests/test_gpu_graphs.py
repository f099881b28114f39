"""CUDA-graph replay of the two-grid cycle and of the FGMRES preconditioner.

A replayed graph launches the same kernels in the same order on the same
buffers as th_cycle, and every kernel is deterministic, so the results must be
bitwise identical to the kernel-by-kernel path (and hence share its parity with
the oracle, which the other GPU tests establish)."""
import numpy as np
import pytest

import synth
from tests.common import ensure_built

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


def _solver(th, prec, nrhs_max=3, **kw):
    w = synth.workload("square10_q4_n25")
    S = th.TwoGridSolver(w["n"], w["p"], w["k"], w["eps"], alpha_s=0.5, l_dd=2, prec=prec,
                         extra_prec=("fp32",) if prec == "bf16" else (), nrhs_max=nrhs_max, device=DEV, **kw)
    return S, w


def _rhs(w, nrhs, seed):
    rng = np.random.default_rng(seed)
    F = np.stack([w["f"] * (1 + 0.3 * rng.standard_normal()) + 1e-3 * synth.random_complex(w["f"].size, seed + r)
                  for r in range(nrhs)])
    return torch.from_numpy(F if nrhs > 1 else F[0]).to(DEV)


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_cycle_graph_bitwise_equals_cycle(th, prec, nrhs):
    S, w = _solver(th, prec)
    f = _rhs(w, nrhs, 11)
    u1 = torch.zeros_like(f)
    u2 = torch.zeros_like(f)
    l0 = S.launch_count()
    for _ in range(3):
        S.cycle(f, u1)
    l1 = S.launch_count()
    for _ in range(3):
        S.cycle_graph(f, u2)   # first call captures, all three replay
    l2 = S.launch_count()
    torch.cuda.synchronize()
    S.device_status()
    assert torch.equal(u1, u2)
    assert l2 - l1 == l1 - l0 > 0
    assert torch.linalg.vector_norm(u1) > 0


def test_graph_cache_follows_settings(th):
    S, w = _solver(th, "bf16")
    f = _rhs(w, 1, 5)
    u = torch.zeros_like(f)
    S.cycle_graph(f, u)
    # switching precision or kernel variant must not replay the stale graph
    S.set_precision("fp32")
    a = torch.zeros_like(f)
    b = torch.zeros_like(f)
    S.cycle(f, a)
    S.cycle_graph(f, b)
    assert torch.equal(a, b)
    S.set_variant("dd", "fp32", 1 - S.get_variant("dd", "fp32"))
    a.zero_()
    b.zero_()
    S.cycle(f, a)
    S.cycle_graph(f, b)
    assert torch.equal(a, b)
    # graphs off: plain launches, same result
    S.set_graphs(False)
    c = torch.zeros_like(f)
    S.cycle_graph(f, c)
    assert torch.equal(a, c)
    torch.cuda.synchronize()
    S.device_status()


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_solve_with_and_without_graphs_identical(th, prec):
    S, w = _solver(th, prec, nrhs_max=2, restart=8)   # restart 8: the graph cache is reused across cycles
    f = _rhs(w, 2, 21)
    S.set_graphs(False)
    u0, info0 = S.solve(f)
    S.set_graphs(True)
    u1, info1 = S.solve(f)
    u2, info2 = S.solve(f)   # second solve replays the cached graphs
    assert info0["iters"] == info1["iters"] == info2["iters"]
    assert info0["converged"] == 2
    assert torch.equal(u0, u1) and torch.equal(u1, u2)


def test_profiling_bypasses_graphs(th):
    S, w = _solver(th, "bf16")
    f = _rhs(w, 1, 3)
    u = torch.zeros_like(f)
    S.cycle_graph(f, u)
    S.profile(True)
    S.cycle_graph(f, u)
    torch.cuda.synchronize()
    p = S.profile_read()
    S.profile(False)
    assert p["dd"][1] >= 2 and p["coarse_solve"][1] >= 1


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_uneven_domains_concurrent_in_one_graph(th, prec):
    """A mixed batch of independent domains of uneven size (6, 9 and 13 cells per
    side, each its own random field, layer and source): one TwoGridStep of every
    domain captured into one CUDA graph, each domain's launches on a stream of
    its own (forked from and joined into the capture stream) so that they run
    concurrently.  Every domain's result equals its own step launched alone,
    bitwise, and (FP64) the oracle's TwoGridStep within 1e-9."""
    from oracle import twogrid
    from tests.common import small_case
    doms = []
    for i, n in enumerate((6, 9, 13)):
        k, eps = small_case(n=n, p=4, W=n / 4.0, seed=20 + i)
        extra = ("fp64",) if prec != "fp64" else ()
        S = th.TwoGridSolver(n, 4, k, eps, alpha_s=0.5, l_dd=2, prec=prec, extra_prec=extra, device=DEV)
        S.set_graphs(False)
        f = synth.random_complex(S.N, 40 + i)
        u = synth.random_complex(S.N, 50 + i)
        doms.append((S, k, eps, f, u, n))
    alone = []
    for S, k, eps, f, u, n in doms:
        alone.append(S.cycle(torch.from_numpy(f).to(DEV), torch.from_numpy(u.copy()).to(DEV)))
    torch.cuda.synchronize()
    main = torch.cuda.Stream()
    sides = [torch.cuda.Stream() for _ in doms]
    F = [torch.from_numpy(f).to(DEV) for (_, _, _, f, _, _) in doms]
    U = [torch.from_numpy(u.copy()).to(DEV) for (_, _, _, _, u, _) in doms]
    U0 = [x.clone() for x in U]
    main.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=main):
        for (S, *_), f, x, st in zip(doms, F, U, sides):
            st.wait_stream(main)
            with torch.cuda.stream(st):
                S.cycle(f, x)
        for st in sides:
            main.wait_stream(st)
    for x, x0 in zip(U, U0):   # the capture ran nothing: start from the initial iterates
        x.copy_(x0)
    graph.replay()
    torch.cuda.synchronize()
    for (S, k, eps, f, u, n), x, a in zip(doms, U, alone):
        S.device_status()
        assert torch.equal(x, a)
        if prec == "fp64":
            P = twogrid.Problem(n, 4, k, eps, alpha_s=0.5)
            want = twogrid.TwoGrid(P, l_dd=2).step(u.copy(), f)
            got = x.cpu().numpy()
            assert np.abs(got - want).max() / np.abs(want).max() < 1e-9
    for d in doms:
        d[0].close()
