"""Failure detection through the C ABI, without faulting or stalling the GPU.

* A right-hand side with a NaN: th_solve returns TH_ERR_NONFINITE (the
  residual norm is not finite) and the context stays usable.
* maxit below the iterations the tolerance needs: TH_ERR_NOCONV, the last
  iterate returned, and the same context converges afterwards.
* Bounded device waits: with th_set_wait_limit(ctx, 0) every kernel that waits
  on an mbarrier (streamed and tensor-core subdomain products, the coarse
  chunk sweep's row exchange, the corrector's convolutions) records a timeout
  and returns before its first barrier, bulk copy, st.async or MMA;
  th_device_status reports TH_ERR_TIMEOUT (and clears it).  With the default
  limit restored the next call on the same context matches the oracle again.
"""
import numpy as np
import pytest

import synth
from oracle import dd, krylov, twogrid
from tests.common import ensure_built, relerr, small_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"
TH_ERR_NOCONV, TH_ERR_NONFINITE, TH_ERR_TIMEOUT = 4, 6, 7


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


def _case(th, n=9, nrhs=1, **kw):
    k, eps = small_case(n=n, p=4)
    S = th.TwoGridSolver(n, 4, k, eps, alpha_s=0.5, l_dd=2, nrhs_max=nrhs, restart=30, device=DEV, **kw)
    P = twogrid.Problem(n, 4, k, eps, alpha_s=0.5)
    return S, P


def _expect_timeout(th, S):
    with pytest.raises(th.ThError) as e:
        S.device_status()
    assert e.value.code == TH_ERR_TIMEOUT
    S.device_status()  # cleared


def test_nan_in_source_is_reported_and_context_recovers(th):
    S, P = _case(th)
    f = synth.random_complex(P.N, 3)
    bad = f.copy()
    bad[P.N // 2] = np.nan
    _, info = S.solve(dev(bad), check=False)
    assert info["status"] == TH_ERR_NONFINITE
    x, info = S.solve(dev(f))
    TG = twogrid.TwoGrid(P, l_dd=2)
    xo, it, _, _ = krylov.fgmres(lambda v: P.A @ v, TG.precondition, f, tol=1e-8, restart=30)
    assert info["iters"] == it and relerr(host(x), xo) < 1e-7


def test_maxit_below_need_is_reported(th):
    S, P = _case(th, maxit=3)
    f = synth.random_complex(P.N, 4)
    x, info = S.solve(dev(f), check=False)
    assert info["status"] == TH_ERR_NOCONV and info["converged"] == 0
    rr = np.linalg.norm(f - P.A @ host(x)) / np.linalg.norm(f)
    assert 1e-8 < rr < 1.0    # the last iterate: progress, not convergence
    S2, _ = _case(th, maxit=200)
    _, info2 = S2.solve(dev(f))
    assert info2["converged"] == 1 and info2["iters"] > 3


def test_zero_wait_limit_streamed_subdomain_products(th):
    """One right-hand side on BF16 rows: the TMA-ring kernels (variants 1 and 2)."""
    S, P = _case(th, prec="bf16", extra_prec=("fp64",))
    sm = dd.DDSmoother(P, 2)
    f = synth.random_complex(P.N, 5)
    u = synth.random_complex(P.N, 6)
    want = sm.smooth(u, f, 1) - u
    for variant in (1, 2):
        S.set_variant("dd", "fp32", variant)
        S.set_wait_limit(0)
        S.smooth(dev(f), dev(u.copy()))
        _expect_timeout(th, S)
        S.set_wait_limit(-1)
        got = host(S.smooth(dev(f), dev(u.copy()))) - u
        S.device_status()
        assert relerr(got, want) < 2e-2


def test_zero_wait_limit_tensor_core_products(th):
    nrhs = 8
    S, P = _case(th, nrhs=nrhs, prec="bf16")
    assert S.get_variant("dd_batch", "fp32") == 1
    sm = dd.DDSmoother(P, 2)
    f = synth.random_complex((nrhs, P.N), 7)
    u = synth.random_complex((nrhs, P.N), 8)
    S.set_wait_limit(0)
    S.smooth(dev(f), dev(u.copy()))
    _expect_timeout(th, S)
    S.set_wait_limit(-1)
    got = host(S.smooth(dev(f), dev(u.copy()))) - u
    S.device_status()
    want = np.stack([sm.smooth(u[i], f[i], 1) for i in range(nrhs)]) - u
    assert relerr(got, want) < 3e-2


def test_zero_wait_limit_coarse_row_exchange(th):
    """The coarse chunk sweep whose rows travel by st.async onto mbarriers (variant 2)."""
    S, P = _case(th, n=25, prec="fp32", extra_prec=("fp64",))
    S.set_variant("coarse", "fp32", 2)
    B = twogrid.BandedSolver(P.Aq)
    rc = synth.random_complex(P.Nc, 9)
    S.set_wait_limit(0)
    S.coarse_solve(dev(rc))
    _expect_timeout(th, S)
    S.set_wait_limit(-1)
    got = host(S.coarse_solve(dev(rc)))
    S.device_status()
    assert relerr(got, B.solve(rc)) < 1e-4


def test_zero_wait_limit_tensor_core_coarse_products(th):
    """The tensor-core separator and spike products of the grouped coarse solve
    (8 right-hand sides, split-BF16 operands)."""
    nrhs = 8
    S, P = _case(th, n=25, nrhs=nrhs, prec="bf16", extra_prec=("fp64",))
    assert S.get_variant("coarse_multi", "fp32") == 2
    B = twogrid.BandedSolver(P.Aq)
    rc = synth.random_complex((nrhs, P.Nc), 10)
    S.set_wait_limit(0)
    S.coarse_solve(dev(rc))
    _expect_timeout(th, S)
    S.set_wait_limit(-1)
    got = host(S.coarse_solve(dev(rc)))
    S.device_status()
    for i in range(nrhs):
        assert relerr(got[i], B.solve(rc[i])) < 2e-4, i


def test_zero_wait_limit_corrector_convolutions(th):
    w = synth.workload("square10_q4_n25")
    S = th.TwoGridSolver(w["n"], w["p"], w["k"], w["eps"], alpha_s=0.5, l_dd=2, prec="bf16",
                         extra_prec=("fp64",), nrhs_max=2, device=DEV)
    shapes = th.unet_param_shapes(4, 16)
    S.unet_init(synth.he_normal(shapes, 77), levels=4, base=16, batch_max=2)
    x = torch.from_numpy(synth.rng(3).standard_normal((1, S.unet_mp, S.unet_mp, 3)).astype(np.float32)).to(DEV)
    ref = S.unet_forward(x).clone()
    S.device_status()
    S.set_wait_limit(0)
    S.unet_forward(x)
    _expect_timeout(th, S)
    S.set_wait_limit(-1)
    again = S.unet_forward(x)
    S.device_status()
    assert torch.equal(again, ref)
