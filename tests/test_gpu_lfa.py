"""GPU Fourier analysis (Section 6) against the oracle's Bloch-symbol LFA.

Per theta the library's rho(M(theta)) (Gelfand's formula, 40 normalised
squarings) is compared with the largest eigenvalue modulus the oracle takes
from numpy.linalg.eigvals of its own symbol; both build the symbols from
blocks of a periodic assembly, independently.  Tolerance 1e-7 relative (the
Gelfand limit error is ~1e-10, FP64 elimination of symbols with condition
numbers up to ~1e4)."""
import math

import numpy as np
import pytest

from oracle import lfa
from tests.common import ensure_built

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def th():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    import paper_2509_17494_gb300 as th
    return th


@pytest.mark.parametrize("p,ppw,n_s,omega_c,coarse,alpha_c", [(2, 8, 1, 1.0, "qsfem", 0.0), (4, 6, 1, 1.0, "qsfem", 0.0),
                                                               (4, 10, 2, 0.8, "qsfem", 0.0), (6, 7, 1, 1.0, "qsfem", 0.0),
                                                               (4, 8, 1, 1.0, "gal", 0.0), (6, 10, 2, 1.0, "gal", 0.05),
                                                               (2, 12, 1, 1.0, "gal", 0.0)])
def test_lfa_per_theta_matches_oracle(th, p, ppw, n_s, omega_c, coarse, alpha_c):
    D, alpha_s, npts = 0.01, 0.2, 10
    kh = 2 * math.pi * p / ppw
    rmax, rth = th.lfa_rho(p, [[kh, D / math.pi, alpha_s, omega_c]], n_s=n_s, npts=npts, per_theta=True,
                           coarse=coarse, alpha_c=alpha_c)
    ops = lfa.BlochOperators(p, kh, D / math.pi, alpha_s, coarse, alpha_c)
    grid = lfa.theta_grid(npts)
    want = np.array([np.max(np.abs(np.linalg.eigvals(ops.M_hat(t, n_s, omega_c)))) for t in grid]).reshape(npts, npts)
    got = rth[0]
    assert np.all(np.abs(got - want) <= 1e-7 * np.maximum(want, 1.0)), np.abs(got - want).max()
    assert abs(rmax[0] - want.max()) <= 1e-7 * max(want.max(), 1.0)


def test_lfa_batch_and_thresholds(th):
    """A batch of parameter points equals the points one by one, and the
    rates reproduce the thresholds of Section 6 (p = 4: below 1/2 at 10 dofs per
    wavelength, above 1 at 6; p = 6: below 1 at 7, above 1 at 6)."""
    D, a_s = 0.01, 0.2
    pts4 = [[2 * math.pi * 4 / ppw, D / math.pi, a_s, 1.0] for ppw in (6, 10)]
    both = th.lfa_rho(4, pts4, npts=24)
    one = [th.lfa_rho(4, [q], npts=24)[0] for q in pts4]
    assert np.array_equal(both, np.array(one))
    assert both[1] < 0.5 and both[0] > 1.0
    pts6 = [[2 * math.pi * 6 / ppw, D / math.pi, a_s, 1.0] for ppw in (6, 7)]
    r6 = th.lfa_rho(6, pts6, npts=20)
    assert r6[1] < 1.0 and r6[0] > 1.0


def test_lfa_argument_errors(th):
    with pytest.raises(th.ThError) as e:
        th.lfa_rho(8, [[1.0, 0.0, 0.2, 1.0]], npts=4)
    assert e.value.code == 8
    with pytest.raises(th.ThError):
        th.lfa_rho(4, [[-1.0, 0.0, 0.2, 1.0]], npts=4)


@pytest.mark.parametrize("kind", ["qsfem", "q1", "fd5"])
def test_dispersion_error_matches_oracle(th, kind):
    """D_P / k (Section 3.2) per direction on the GPU against the oracle's trace of
    the zero set (scan + Brent on each ray, dense scan + bounded minimisation over
    rays): within 1e-10 of k.  The QSFEM stencils come from the library's
    cancellation-free weights and the oracle's 50-digit ones."""
    from oracle import dispersion
    etas = [0.4, 1.0, 2 * math.pi / 5, 1.6]
    nt = 12
    dmax, dth = th.dispersion(kind, etas, nt=nt, per_theta=True)
    for i, eta in enumerate(etas):
        want_max, want = dispersion.dispersion_error(kind, eta, nt=nt)
        assert np.abs(dth[i] - want).max() < 1e-10, (eta, np.abs(dth[i] - want).max())
        assert abs(dmax[i] - want_max) < 1e-10
    if kind == "qsfem":
        # the exact zeros: with nt = 32 the directions are the multiples of pi/16, the odd ones
        # (pi/16, 3 pi/16 and their images under the stencil's symmetries) are zeros of sigma_P on |xi| = k
        _, d32 = th.dispersion(kind, [1.0], nt=32, per_theta=True)
        t = -math.pi + 2 * math.pi * np.arange(32) / 32
        on = np.isclose(np.mod(t * 16 / math.pi, 2), 1.0)
        assert np.all(d32[0][on] < 1e-11)
