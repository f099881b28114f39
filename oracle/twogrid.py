"""Oracle: the two-grid cycle (plain FP64, CPU).

TEST INFRASTRUCTURE ONLY (see oracle/fem.py).

Algorithm 1 (TwoGridStep): n_s smoother steps; r_c = I_P^* (f - A u);
solve A_c u_c = r_c; u += omega_c I_P u_c; n_s smoother steps.  Used as a
preconditioner with u = 0 on input (Section 4).  The restriction I_P^* is the
transpose of the real prolongation (residuals are dual vectors).  The coarse
operator is A_q of Section 3.3 ('opt'), or the Galerkin operator of standard
p-type coarsening ('gal', oracle/galerkin.py), and is solved directly (banded
LU, LAPACK zgbtrf/zgbtrs, lexicographic ordering).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg.lapack as lapack
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import dd, fem, galerkin, qsfem


class Problem:
    """Discretised Helmholtz problem: A, A_s, A_q, I_P on the unit square."""

    def __init__(self, n: int, p: int, k_cell, eps_cell=None, bc="robin", dim: int = 2,
                 alpha_s: float = 0.5, periodic: bool = False, coarse: bool = True,
                 coarse_kind: str = "qsfem", alpha_c: float = 0.0):
        self.dim, self.n, self.p = dim, n, p
        self.h = 1.0 / n
        self.k = np.asarray(k_cell, dtype=float).reshape((n,) * dim)
        self.eps = (np.zeros_like(self.k) if eps_cell is None
                    else np.asarray(eps_cell, dtype=float).reshape((n,) * dim))
        self.periodic = periodic
        self.alpha_s = alpha_s
        self.robin_sides = [] if periodic else fem.robin_set(dim, bc)
        # Dirichlet sides (Gamma_0): the unknowns there are kept on the node grid,
        # decoupled by identity rows and columns (fem.impose_dirichlet)
        self.dirichlet_sides = [] if periodic else fem.dirichlet_set(dim, bc)
        nc = (n,) * dim
        self.dmask = fem.boundary_mask(n * p + 1, dim, self.dirichlet_sides) if not periodic else None
        self.A = fem.assemble(nc, p, self.h, fem.helmholtz_coefficient(self.k, self.eps),
                              self.k, self.robin_sides, periodic)
        self.As = fem.assemble(nc, p, self.h, fem.shifted_coefficient(self.k, self.eps, alpha_s),
                               self.k, self.robin_sides, periodic)
        if self.dirichlet_sides:
            self.A = fem.impose_dirichlet(self.A, self.dmask)
            self.As = fem.impose_dirichlet(self.As, self.dmask)
        self.N = self.A.shape[0]
        if coarse:
            self.IP = fem.prolongation(n, p, dim, periodic)
            self.coarse_kind = coarse_kind
            if coarse_kind == "qsfem":
                self.Aq = qsfem.assemble_coarse(n, p, self.k, self.eps, self.robin_sides, periodic)
            elif coarse_kind == "gal":
                if self.dirichlet_sides:
                    raise ValueError("Galerkin coarsening with Dirichlet sides is not built")
                self.Aq = galerkin.galerkin_coarse(self, alpha_c)
            else:
                raise ValueError(coarse_kind)
            if self.dirichlet_sides:
                # the coarse space vanishes on Gamma_0 as well: I_P maps only the
                # coarse nodes off it, and A_q is decoupled there
                cmask = fem.boundary_mask(n * p // 2 + 1, dim, self.dirichlet_sides)
                self.IP = (self.IP @ sp.diags((~cmask).astype(float))).tocsr()
                self.Aq = fem.impose_dirichlet(self.Aq, cmask)
            self.Nc = self.Aq.shape[0]


class BandedSolver:
    """Direct solve of A_q with LAPACK's banded LU (factor once, solve per call)."""

    def __init__(self, A: sp.spmatrix):
        A = A.tocoo()
        n = A.shape[0]
        bw = int(np.max(np.abs(A.row - A.col)))
        self.kl = self.ku = bw
        ab = np.zeros((2 * bw + bw + 1, n), dtype=np.complex128)
        ab[bw + bw + A.row - A.col, A.col] = A.data     # LAPACK band layout with kl extra rows
        lu, piv, info = lapack.zgbtrf(ab, bw, bw)
        if info != 0:
            raise np.linalg.LinAlgError(f"zgbtrf info={info}")
        self.lu, self.piv = lu, piv

    def solve(self, b):
        x, info = lapack.zgbtrs(self.lu, self.kl, self.ku, b, self.piv)
        if info != 0:
            raise np.linalg.LinAlgError(f"zgbtrs info={info}")
        return x


class SparseLUSolver:
    def __init__(self, A):
        self.lu = spla.splu(A.tocsc())

    def solve(self, b):
        return self.lu.solve(b)


class TwoGrid:
    """Algorithm 1 with the CSDD smoother and the QSFEM coarse level."""

    def __init__(self, prob: Problem, l_dd: int = 2, n_dd: int = 1, n_s: int = 1,
                 omega_c: float = 1.0, coarse_solver: str = "banded"):
        self.prob = prob
        self.n_dd, self.n_s, self.omega_c = n_dd, n_s, omega_c
        self.smoother = dd.DDSmoother(prob, l_dd)
        if coarse_solver == "banded" and not prob.periodic:
            self.coarse = BandedSolver(prob.Aq)
        else:
            self.coarse = SparseLUSolver(prob.Aq)

    def smooth(self, u, f):
        return self.smoother.smooth(u, f, self.n_dd)

    def restrict(self, r):
        return self.prob.IP.T @ r

    def prolong(self, uc):
        return self.prob.IP @ uc

    def step(self, u, f):
        """TwoGridStep(u, f) -> updated u."""
        P = self.prob
        for _ in range(self.n_s):
            u = self.smooth(u, f)
        rc = self.restrict(f - P.A @ u)
        uc = self.coarse.solve(rc)
        u = u + self.omega_c * self.prolong(uc)
        for _ in range(self.n_s):
            u = self.smooth(u, f)
        return u

    def precondition(self, f):
        """Left/right preconditioner: TwoGridStep with u = 0 on input."""
        return self.step(np.zeros_like(f), f)
