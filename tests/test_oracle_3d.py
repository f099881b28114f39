"""Pins of the oracle in three dimensions: Q2 finite elements, the fitted
27-point coarse operator, the smoother and the two-grid cycle.

The 27-point scheme is the project's construction (the paper only cites one),
so its pins are facts any such scheme must meet plus the property the fit is
for: small ξ consistency with |ξ|² − η², an assembly that reproduces the
symbol on plane waves, the ε and Robin terms as Q1 masses, complex symmetry,
and a phase error far below the Q1 finite element's in random directions
(none of them among the fitted ones)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.optimize import brentq

from oracle import dd, fem, qsfem, twogrid
import synth


def _q1fe_symbol(eta, xi):
    k = lambda x: 2 - 2 * np.cos(x)
    m = lambda x: (2 + np.cos(x)) / 3
    a, b, c = xi
    return k(a) * m(b) * m(c) + m(a) * k(b) * m(c) + m(a) * m(b) * k(c) - eta ** 2 * m(a) * m(b) * m(c)


def test_fit27_dispersion_far_below_q1_fe():
    dirs = synth.rng(11).standard_normal((150, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    for eta, bound in ((1.0, 1e-5), (1.57, 1e-4)):
        fit, fe = [], []
        for d in dirs:
            fit.append(abs(brentq(lambda t: qsfem.symbol27(eta, t * d), 0.5 * eta, 1.5 * eta) - eta) / eta)
            fe.append(abs(brentq(lambda t: _q1fe_symbol(eta, t * d), 0.5 * eta, 1.5 * eta) - eta) / eta)
        assert max(fit) < bound, max(fit)
        assert max(fe) > 100 * max(fit)


def test_fit27_small_wavevector_consistency():
    """N sigma_P(xi) = |xi|^2 - eta^2 + O(|xi|^4 + eta^4): a consistent -Lap - k^2."""
    r = synth.rng(12)
    for eta in (0.02, 0.05):
        for _ in range(5):
            d = r.standard_normal(3)
            xi = 0.7 * eta * d / np.linalg.norm(d)
            got = qsfem.symbol27(eta, xi)
            want = xi @ xi - eta ** 2
            assert abs(got - want) < 5 * eta ** 4, (eta, got, want)


def test_fit27_normalisation_and_zeros():
    for eta in (0.2, 1.0, 2.0):
        assert abs(qsfem.symbol27(eta, [0, 0, 0]) + eta ** 2) < 1e-13 * max(1, eta ** 2)
        for d in qsfem.DIRS3:
            assert abs(qsfem.symbol27(eta, eta * d)) < 1e-13
        # the directions lie in the symmetry-reduced triangle 0 <= x <= y <= z
    assert np.all(np.diff(qsfem.DIRS3, axis=1) > 0) and np.all(qsfem.DIRS3 > 0)


def test_assembled_27_point_operator_acts_as_its_symbol_on_plane_waves():
    """Periodic coarse grid, constant k: A_q e^{i xi . j} = h_c N sigma_P(xi) e^{i xi . j}."""
    n, p = 4, 2
    nc = n * p // 2
    hc = 1.0 / nc
    kk = 5.0
    kc = np.full((n, n, n), kk)
    A = qsfem.assemble_coarse(n, p, kc, 0 * kc, (), True)
    m = nc
    z, y, x = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    for l in ((1, 0, 0), (1, 2, 3), (0, 3, 1)):
        xi = 2 * np.pi * np.array(l) / m
        wave = np.exp(1j * (xi[0] * z + xi[1] * y + xi[2] * x)).reshape(-1)
        lam = hc * qsfem.symbol27(kk * hc, xi)
        assert np.allclose(A @ wave, lam * wave, atol=1e-12 * max(1.0, abs(lam)))


def test_coarse3_damping_and_robin_terms_are_q1_masses():
    n, p = 3, 2
    nc = n * p // 2
    hc = 1.0 / nc
    kc = synth.rng(13).uniform(3.0, 6.0, (n, n, n))
    A0 = qsfem.assemble_coarse(n, p, kc, 0 * kc)
    A1 = qsfem.assemble_coarse(n, p, kc, 0 * kc + 1.0)
    M1 = sp.diags([1 / 6, 2 / 3, 1 / 6], [-1, 0, 1], shape=(nc + 1, nc + 1)).toarray() * hc
    M1[0, 0] = M1[-1, -1] = hc / 3
    M3 = np.kron(np.kron(M1, M1), M1)
    assert np.allclose((A1 - A0).toarray(), -1j * M3, atol=1e-15)
    # Robin on z-low: the added face term integrates to -i k over the unit face
    kconst = np.full((n, n, n), 4.0)
    B0 = qsfem.assemble_coarse(n, p, kconst, 0 * kconst, ())
    B1 = qsfem.assemble_coarse(n, p, kconst, 0 * kconst, [(0, 0)])
    D = (B1 - B0).toarray()
    assert abs(D.sum() + 4.0j) < 1e-13
    face = np.zeros((nc + 1) ** 3, bool)
    face[: (nc + 1) ** 2] = True
    assert np.all(D[~face, :] == 0) and np.all(D[:, ~face] == 0)
    assert abs(B1 - B1.T).max() < 1e-15 and abs(A1 - A1.T).max() < 1e-15


def test_q2_3d_manufactured_convergence():
    """u = cos(pi x) cos(pi y) cos(pi z) (natural boundary), f = (3 pi^2 - k^2) u:
    the Q2 error, measured against the interpolant in the mass norm, decays at least like h^3."""
    p, kk = 2, 2.0
    errs, ns = [], [2, 4, 8]
    for n in ns:
        kc = np.full((n, n, n), kk)
        A = fem.assemble((n, n, n), p, 1.0 / n, kc ** 2 + 0j, kc, [])
        M = fem.assemble((n, n, n), p, 1.0 / n, np.full((n, n, n), -1.0 + 0j), 0 * kc, []) - \
            fem.assemble((n, n, n), p, 1.0 / n, np.zeros((n, n, n), complex), 0 * kc, [])
        ufun = lambda z, y, x: np.cos(np.pi * x) * np.cos(np.pi * y) * np.cos(np.pi * z)
        ui = fem.interpolate_nodal(n, p, ufun, dim=3)
        b = M @ ((3 * np.pi ** 2 - kk ** 2) * ui)
        uh = spla.spsolve(A.tocsc(), b)
        errs.append(math.sqrt(abs(np.vdot(uh - ui, M @ (uh - ui)))))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(ns) - 1)]
    assert rates[-1] > p + 1 - 0.35, (errs, rates)


def _small3(n=4, p=2, seed=5):
    k = 2 * np.pi * 1.5 / synth.random_velocity(n, 3, seed)
    eps = synth.absorbing_layer(n, 3, p, k, width_dofs=2)
    return twogrid.Problem(n, p, k, eps, dim=3, alpha_s=0.5)


def test_ddstep_fixed_point_3d():
    P = _small3()
    S = dd.DDSmoother(P, l_dd=2)
    u = synth.random_complex(P.N, 14)
    f = P.As @ u
    assert np.allclose(S.dd_step(u, f), u, atol=1e-10 * np.abs(u).max())
    v = synth.random_complex(P.N, 15)
    assert not np.allclose(S.dd_step(v, f), v, atol=1e-3)


def test_two_grid_3d_fixed_point_and_banded_coarse():
    P = _small3()
    T = twogrid.TwoGrid(P, l_dd=2)
    f = synth.random_complex(P.N, 16)
    u = spla.spsolve(P.A.tocsc(), f)
    assert np.allclose(T.step(u, f), u, atol=1e-9 * np.abs(u).max())
    rc = synth.random_complex(P.Nc, 17)
    B = twogrid.BandedSolver(P.Aq)
    assert np.allclose(B.solve(rc), spla.spsolve(P.Aq.tocsc(), rc), atol=1e-10 * np.abs(B.solve(rc)).max())
    # complex symmetry of the 3-D operators
    for M in (P.A, P.As, P.Aq):
        assert abs(M - M.T).max() <= 1e-13 * abs(M).max()


def test_two_grid_3d_preconditions_fgmres():
    from oracle import krylov
    P = _small3(n=4, p=2)
    T = twogrid.TwoGrid(P, l_dd=2)
    f = synth.random_complex(P.N, 18)
    x, its, rel, _ = krylov.fgmres(lambda v: P.A @ v, T.precondition, f, tol=1e-8, restart=40, maxit=80)
    assert rel <= 1e-8 and its < 25, (its, rel)
