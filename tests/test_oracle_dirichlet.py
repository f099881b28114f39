"""Pins of the oracle's Dirichlet sides (Section 2: u = 0 on Gamma_0, the
solution space H^1_0(Omega; Gamma_0)), kept on the full node grid by identity
rows and columns.

* Manufactured solution u = sin(pi x) sin(pi y) (zero on every side),
  -Laplace u - k^2 u = (2 pi^2 - k^2) u: the L2 error decays like h^(p+1).
* The identity-row form equals the eliminated system on the other nodes, and
  the Dirichlet unknowns equal their right-hand side.
* Mixed sides (Dirichlet on two non-opposite sides, Robin on the others, a
  damping layer): the smoother's fixed point is the A_s solution, the exact
  solution is a fixed point of the two-grid step, the coarse correction's
  prolongation vanishes on Gamma_0, and FGMRES converges.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import dd, fem, krylov, twogrid
from tests.common import small_case


@pytest.mark.parametrize("p", [2, 4])
def test_dirichlet_manufactured_convergence(p):
    kk = 2.0

    def u(x, y):
        return np.sin(math.pi * x) * np.sin(math.pi * y) + 0j

    errs, ns = [], [2, 4, 8]
    for n in ns:
        kc = np.full((n, n), kk)
        A = fem.assemble((n, n), p, 1.0 / n, kc ** 2 + 0j, kc, [])
        M = fem.assemble((n, n), p, 1.0 / n, np.full((n, n), -1.0 + 0j), 0 * kc, []) - \
            fem.assemble((n, n), p, 1.0 / n, np.zeros((n, n)) + 0j, 0 * kc, [])
        mask = fem.boundary_mask(n * p + 1, 2, fem.all_sides(2))
        AD = fem.impose_dirichlet(A, mask)
        b = M @ ((2 * math.pi ** 2 - kk ** 2) * fem.interpolate_nodal(n, p, u))
        b[mask] = 0.0
        uh = spla.spsolve(AD.tocsc(), b)
        assert np.all(uh[mask] == 0)
        errs.append(fem.l2_error_2d(n, p, uh, u))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(ns) - 1)]
    assert rates[-1] > p + 1 - 0.35, (errs, rates)


def test_identity_rows_equal_eliminated_system():
    n, p = 5, 4
    k, eps = small_case(n=n, p=p)
    bc = {(1, 0): "dirichlet", (0, 0): "dirichlet", (1, 1): "robin", (0, 1): "robin"}
    P = twogrid.Problem(n, p, k, eps, bc=bc, alpha_s=0.5)
    Pfull = twogrid.Problem(n, p, k, eps, bc={(1, 1): "robin", (0, 1): "robin"}, alpha_s=0.5)
    I = ~P.dmask
    f = synth.random_complex(P.N, 3)
    u = spla.spsolve(P.A.tocsc(), f)
    ui = spla.spsolve(Pfull.A[I][:, I].tocsc(), f[I])
    assert np.abs(u[I] - ui).max() < 1e-11 * np.abs(ui).max()
    assert np.array_equal(u[P.dmask], f[P.dmask])
    # the Dirichlet nodes are the x-low and y-low node lines
    m = n * p + 1
    grid = P.dmask.reshape(m, m)
    assert grid[0, :].all() and grid[:, 0].all() and not grid[1:, 1:].any()


def test_dirichlet_two_grid_fixed_points_and_solve():
    n, p = 8, 4
    k, eps = small_case(n=n, p=p, W=2.0)
    bc = {(1, 0): "dirichlet", (0, 0): "dirichlet", (1, 1): "robin", (0, 1): "robin"}
    P = twogrid.Problem(n, p, k, eps, bc=bc, alpha_s=0.5)
    f = synth.random_complex(P.N, 5)
    f[P.dmask] = 0.0
    sm = dd.DDSmoother(P, 2)
    us = spla.spsolve(P.As.tocsc(), f)
    assert np.abs(sm.dd_step(us, f) - us).max() < 1e-10 * np.abs(us).max()
    TG = twogrid.TwoGrid(P, l_dd=2)
    ue = spla.spsolve(P.A.tocsc(), f)
    assert np.abs(TG.step(ue, f) - ue).max() < 1e-9 * np.abs(ue).max()
    # the prolonged coarse correction vanishes on Gamma_0
    uc = synth.random_complex(P.Nc, 6)
    assert np.all(TG.prolong(uc)[P.dmask] == 0)
    x, it, rr, _ = krylov.fgmres(lambda v: P.A @ v, TG.precondition, f, tol=1e-8, restart=40)
    assert rr <= 1e-8 and it < 40
    assert np.abs(x[P.dmask]).max() == 0.0
