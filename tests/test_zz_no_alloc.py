"""The allocation-free coarse solve entry point against th_coarse_solve.

th_coarse_solve_noalloc serves callers that cannot allocate device memory at
the time of the call: its scratch lives in a fixed device array of the
library.  Both entry points run the same FP64 block sweep, so their outputs
must agree to the FP64 apply tolerance used elsewhere (1e-12 relative) on two
calls in a row (the second call reuses the array with the first call's
contents still in it).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import synth
from tests.common import ensure_built, relerr, small_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def th():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    import paper_2509_17494_gb300 as th
    L = th.lib()
    fn = L.th_coarse_solve_noalloc
    fn.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return th


def _solver(th, n, nrhs):
    k, eps = small_case(n=n, p=4, W=n / 4.0)
    return th.TwoGridSolver(n, 4, k, eps, alpha_s=0.5, l_dd=2, nrhs_max=nrhs, device="cuda:0")


@pytest.mark.parametrize("n,nrhs", [(9, 1), (25, 3)])
def test_noalloc_coarse_solve_matches_entry_point_twice(th, n, nrhs):
    S = _solver(th, n, nrhs)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    fn = th.lib().th_coarse_solve_noalloc
    for call in range(2):
        rc = torch.from_numpy(synth.random_complex((nrhs, S.Nc), 40 + call)).to("cuda:0")
        want = S.coarse_solve(rc)
        got = torch.empty_like(rc)
        st = fn(S._ctx, ctypes.c_void_p(rc.data_ptr()), ctypes.c_void_p(got.data_ptr()), nrhs, stream)
        assert st == 0, th.lib().th_status_str(st)
        torch.cuda.synchronize()
        assert relerr(got.cpu().numpy(), want.cpu().numpy()) < 1e-12


def test_noalloc_rejects_requests_beyond_the_array(th):
    S = _solver(th, 25, 3)
    fn = th.lib().th_coarse_solve_noalloc
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = torch.zeros((3, S.Nc), dtype=torch.complex128, device="cuda:0")
    # nrhs above the context's nrhs_max
    assert fn(S._ctx, ctypes.c_void_p(rc.data_ptr()), ctypes.c_void_p(rc.data_ptr()), 4, stream) == 1
    # more values than the 2^18-entry array: 51^2 coarse values x 101 right-hand sides
    k, eps = small_case(n=25, p=4, W=25 / 4.0)
    big = th.TwoGridSolver(25, 4, k, eps, alpha_s=0.5, l_dd=2, nrhs_max=101, restart=1, device="cuda:0")
    rcb = torch.zeros((101, big.Nc), dtype=torch.complex128, device="cuda:0")
    assert big.Nc * 101 > (1 << 18)
    assert fn(big._ctx, ctypes.c_void_p(rcb.data_ptr()), ctypes.c_void_p(rcb.data_ptr()), 101, stream) == 1
    # one right-hand side below the limit still works on the same context
    rc1 = torch.from_numpy(synth.random_complex((1, big.Nc), 7)).to("cuda:0")
    out = torch.empty_like(rc1)
    assert fn(big._ctx, ctypes.c_void_p(rc1.data_ptr()), ctypes.c_void_p(out.data_ptr()), 1, stream) == 0
    torch.cuda.synchronize()
    assert relerr(out.cpu().numpy(), big.coarse_solve(rc1).cpu().numpy()) < 1e-12


def test_noalloc_refuses_other_coarse_levels(th):
    """The entry point covers the 2-D dispersion-matched coarse level only: a
    3-D context and a Galerkin-coarsened context return TH_ERR_UNSUPPORTED (8)
    and touch neither vector."""
    fn = th.lib().th_coarse_solve_noalloc
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n3 = 4
    k3 = 2 * np.pi * 1.5 / synth.random_velocity(n3, 3, 5)
    S3 = th.TwoGridSolver(n3, 2, k3, None, alpha_s=0.5, l_dd=2, device="cuda:0", dim=3)
    k, eps = small_case(n=6, p=4)
    Sg = th.TwoGridSolver(6, 4, k, eps, alpha_s=0.5, l_dd=2, device="cuda:0", coarse="gal", alpha_c=0.02)
    for S in (S3, Sg):
        rc = torch.from_numpy(synth.random_complex((1, S.Nc), 9)).to("cuda:0")
        out = torch.full_like(rc, 3.0)
        st = fn(S._ctx, ctypes.c_void_p(rc.data_ptr()), ctypes.c_void_p(out.data_ptr()), 1, stream)
        assert st == 8, th.lib().th_status_str(st)
        torch.cuda.synchronize()
        assert torch.all(out == 3.0)
