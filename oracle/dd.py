"""Oracle: complex-shifted domain-decomposition smoother (plain FP64, CPU).

TEST INFRASTRUCTURE ONLY (see oracle/fem.py).

Section 4.1 and Algorithm 2 (CSDDSmoother / DDStep), Eq. RAS_like_update;
partition as in Section 4.5:
  * U^(i): blocks of l_dd cells per direction forming a partition of the
    cells; when n is not a multiple of l_dd the ceil(n/l_dd) blocks are made
    as equal as possible, larger ones first (the paper: some are one smaller);
  * Omega^(i) = U^(i) plus one layer of neighbouring cells (edge or vertex
    neighbours), clipped at the domain boundary;
  * A_s^(i): the shifted bilinear form on Omega^(i), with an absorbing
    condition -i k (unshifted k) on the internal boundary of Omega^(i) and the
    original condition on parts of the original boundary;
  * DDStep: w_i = (A_s^(i))^{-1} [ -(R_i A_s - A_s^(i) R_i) u + R_i f ],
    then u_j = (1/L_j) sum_{i : j in Dofs(U^(i))} (R_i^T w_i)_j;
  * CSDDSmoother: r = f - A u;  v = 0;  n_dd times DDStep(v, r; A_s);  u += v.

The local solves use a sparse LU (SuperLU) of each A_s^(i).
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem


def partition_1d(n: int, l_dd: int):
    """[(start, size)] of the ceil(n/l_dd) blocks, sizes as equal as possible, larger first."""
    nb = -(-n // l_dd)
    base, rem = divmod(n, nb)
    sizes = [base + 1] * rem + [base] * (nb - rem)
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(int)
    return list(zip(starts.tolist(), sizes))


class Subdomain:
    """One overlapping subdomain: index sets, local shifted matrix and its LU."""

    def __init__(self, ublock, oblock, omega_dofs, u_dofs, u_local, As_local):
        self.ublock = ublock          # per axis (cell start, cell stop) of U^(i)
        self.oblock = oblock          # per axis (cell start, cell stop) of Omega^(i)
        self.omega_dofs = omega_dofs  # R_i as global indices (box lexicographic)
        self.u_dofs = u_dofs          # Dofs(U^(i)), global
        self.u_local = u_local        # positions of Dofs(U^(i)) inside omega_dofs
        self.As = As_local            # A_s^(i), sparse
        self.lu = spla.splu(As_local.tocsc())

    def solve(self, b):
        return self.lu.solve(b)


def _box_dofs(lo_hi, p, m):
    """Global indices of the closed dof box of a cell box, lexicographic."""
    dim = len(lo_hi)
    ranges = [np.arange(lo * p, hi * p + 1) for (lo, hi) in lo_hi]
    grids = np.meshgrid(*ranges, indexing="ij")
    strides = [m ** (dim - 1 - ax) for ax in range(dim)]
    g = sum(gr * s for gr, s in zip(grids, strides))
    return g.reshape(-1)


class DDSmoother:
    """Data of Algorithm 2 for one problem (non-periodic, or periodic with one subdomain)."""

    def __init__(self, prob, l_dd: int):
        self.prob = prob
        dim, n, p = prob.dim, prob.n, prob.p
        self.l_dd = l_dd
        if prob.periodic:
            # only the single-subdomain case (Omega^(1) = whole torus, A_s^(1) = A_s)
            assert l_dd >= n
            N = prob.N
            sd = Subdomain(None, None, np.arange(N), np.arange(N), np.arange(N), prob.As)
            self.subs = [sd]
            self.L = np.ones(N)
            return
        m = n * p + 1
        parts = partition_1d(n, l_dd)
        robin = set(prob.robin_sides)
        cs = fem.shifted_coefficient(prob.k, prob.eps, prob.alpha_s)
        self.subs = []
        L = np.zeros(prob.N)
        for blk in itertools.product(parts, repeat=dim):
            ub = [(s, s + z) for (s, z) in blk]
            ob = [(max(s - 1, 0), min(s + z + 1, n)) for (s, z) in blk]
            sl = tuple(slice(lo, hi) for (lo, hi) in ob)
            sides = []
            for ax in range(dim):
                for end in (0, 1):
                    on_boundary = (ob[ax][0] == 0) if end == 0 else (ob[ax][1] == n)
                    if (not on_boundary) or ((ax, end) in robin):   # Dirichlet and Neumann sides: natural here
                        sides.append((ax, end))
            ncl = [hi - lo for (lo, hi) in ob]
            Asl = fem.assemble(ncl, p, prob.h, cs[sl], prob.k[sl], sides)
            odofs = _box_dofs(ob, p, m)
            if getattr(prob, "dirichlet_sides", None):
                # inherited Dirichlet condition on the parts of Gamma_0 in the subdomain's boundary
                Asl = fem.impose_dirichlet(Asl, prob.dmask[odofs])
            udofs = _box_dofs(ub, p, m)
            pos = {g: i for i, g in enumerate(odofs.tolist())}
            uloc = np.array([pos[g] for g in udofs.tolist()])
            self.subs.append(Subdomain(ub, ob, odofs, udofs, uloc, Asl))
            L[udofs] += 1.0
        self.L = L

    def dd_step(self, u, f):
        """DDStep(u, f; A_s) of Algorithm 2 -> new u (Eq. RAS_like_update)."""
        As_u = self.prob.As @ u
        acc = np.zeros_like(u)
        for sd in self.subs:
            ui = u[sd.omega_dofs]
            rhs = -(As_u[sd.omega_dofs] - sd.As @ ui) + f[sd.omega_dofs]
            w = sd.solve(rhs)
            acc[sd.u_dofs] += w[sd.u_local]
        return acc / self.L

    def smooth(self, u, f, n_dd: int = 1):
        """CSDDSmoother(u, f): returns the updated u."""
        r = f - self.prob.A @ u
        v = np.zeros_like(u)
        for _ in range(n_dd):
            v = self.dd_step(v, r)
        return u + v
