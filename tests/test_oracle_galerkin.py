"""Pins of the oracle's Galerkin p-type coarsening ('gal', Section 4).

The coarse operator is I_P^T A_{alpha_c} I_P.  Because Q_{p/2} on the same
mesh is a subspace of Q_p, the same matrix must come out of assembling the
order-p/2 finite-element operator directly, in the equispaced nodal basis of
the coarse grid.  For p = 2 and p = 4 the order-p/2 GLL points are the
equispaced points, so the oracle's own order-p/2 assembly is that basis; for
p = 6 the GLL(3) assembly is mapped to the equispaced basis by a change of
basis built here from a Vandermonde solve (no shared interpolation code)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import fem, galerkin, krylov, twogrid


def _problem(n, p, seed=3, bc="robin", alpha_c=0.0, W=2.0):
    k = 2 * np.pi * W / synth.random_velocity(n, 2, seed)
    eps = synth.absorbing_layer(n, 2, p, k, width_dofs=2)
    return twogrid.Problem(n, p, k, eps, bc=bc, alpha_s=0.2, coarse_kind="gal", alpha_c=alpha_c)


def _direct_order_half(P, alpha_c, T1=None):
    q = P.p // 2
    A = fem.assemble((P.n, P.n), q, P.h, fem.shifted_coefficient(P.k, P.eps, alpha_c), P.k, P.robin_sides)
    if T1 is None:
        return A
    T = sp.kron(sp.csr_matrix(T1), sp.csr_matrix(T1), format="csr")
    return (T.T @ A @ T).tocsr()


@pytest.mark.parametrize("p", [2, 4])
@pytest.mark.parametrize("alpha_c", [0.0, 0.1])
def test_gal_equals_direct_assembly_where_gll_is_equispaced(p, alpha_c):
    P = _problem(5, p, alpha_c=alpha_c, bc={(0, 0): "robin", (1, 1): "robin"})
    D = _direct_order_half(P, alpha_c)
    assert P.Aq.shape == D.shape
    assert abs(P.Aq - D).max() <= 1e-12 * abs(D).max()


def _equispaced_to_gll3(n):
    """1-D map from the equispaced Q3 nodal values to the GLL(3) nodal values."""
    xe = np.linspace(0.0, 1.0, 4)
    c = np.sqrt(5.0) / 5.0                      # interior GLL(3) points on [-1, 1] are +-1/sqrt(5)
    xg = np.array([0.0, 0.5 - 0.5 * c, 0.5 + 0.5 * c, 1.0])
    Ve = np.vander(xe, 4, increasing=True)
    Vg = np.vander(xg, 4, increasing=True)
    Tc = Vg @ np.linalg.inv(Ve)
    m = 3 * n + 1
    T = np.zeros((m, m))
    for e in range(n):
        T[3 * e:3 * e + 4, 3 * e:3 * e + 4] = Tc   # shared end points: rows identical (identity there)
    return T


def test_gal_p6_equals_changed_basis_q3_assembly():
    P = _problem(4, 6, alpha_c=0.05)
    D = _direct_order_half(P, 0.05, _equispaced_to_gll3(P.n))
    assert abs(P.Aq - D).max() <= 1e-11 * abs(D).max()


def test_gal_symmetric_and_shift_sign():
    P0 = _problem(4, 4, alpha_c=0.0)
    P1 = _problem(4, 4, alpha_c=0.3)
    for M in (P0.Aq, P1.Aq):
        assert abs(M - M.T).max() <= 1e-13 * abs(M).max()
    # the shift adds -i alpha_c k^2 times a mass matrix: negative semidefinite imaginary part
    d = (P1.Aq - P0.Aq).toarray()
    assert np.allclose(d.real, 0, atol=1e-13 * abs(d).max())
    ev = np.linalg.eigvalsh(d.imag)
    assert ev.max() < 1e-12 * abs(ev).max()


def test_gal_two_grid_fixed_point_and_fgmres():
    P = _problem(8, 4, alpha_c=0.02)
    T = twogrid.TwoGrid(P, l_dd=2)
    f = synth.random_complex(P.N, 21)
    u = spla.spsolve(P.A.tocsc(), f)
    assert np.allclose(T.step(u, f), u, atol=1e-9 * np.abs(u).max())
    x, its, rel, _ = krylov.fgmres(lambda v: P.A @ v, T.precondition, f, tol=1e-8, restart=60, maxit=120)
    assert rel <= 1e-8, (its, rel)
