"""Oracle: standard Galerkin p-type coarsening ('gal'), plain FP64, CPU.

TEST INFRASTRUCTURE ONLY (see oracle/fem.py).

Section 4 ("Standard Galerkin p-type coarsening"), the paper's comparison
method: the coarse space V_c is Q_{p/2} on the same mesh, so V_c is a subspace
of the fine space V and the prolongation is the embedding.  In nodal
coordinates the embedding is the interpolation I_P of Section 4.2 (the Q_{p/2}
coarse functions are represented by their values on the equispaced points of
each cell, the coarse-grid vertices).  The coarse matrix is the fine bilinear
form restricted to V_c, with the optional small complex shift of the
coarse-level operator that the paper's Table 2 varies (alpha_c):

    A_c = I_P^T A_{alpha_c} I_P,
    A_{alpha_c}: volume coefficient k^2 (1 + i alpha_c) + i eps, Robin term -i k (unshifted).

The Robin term stays unshifted, the same reading as for the smoother's A_s.
"""
from __future__ import annotations

import scipy.sparse as sp

from . import fem


def galerkin_coarse(prob, alpha_c: float = 0.0) -> sp.csr_matrix:
    """A_c = I_P^T A_{alpha_c} I_P on the coarse node grid of `prob` (lexicographic)."""
    ncells = (prob.n,) * prob.dim
    A_shift = fem.assemble(ncells, prob.p, prob.h, fem.shifted_coefficient(prob.k, prob.eps, alpha_c),
                           prob.k, prob.robin_sides, prob.periodic)
    Ac = (prob.IP.T @ A_shift @ prob.IP).tocsr()
    Ac.sum_duplicates()
    return Ac
