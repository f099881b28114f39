"""Oracle: local Fourier analysis of the two-grid method (plain FP64, CPU).

TEST INFRASTRUCTURE ONLY (see oracle/fem.py).

Toy problem (Section 5): 1-D central differences D_{2,M}, coarse grid 2h,
linear interpolation / full weighting, exact shifted smoother A_s = A - i
alpha_s k^2.  Symbols of Section 5.2; the lemma of Section 5.5 (Eq. max_K11).

Finite elements (Section 6.1): Bloch-wave symbols
    sigma(P)(theta) = sum_beta exp(i theta . beta) P_{0,beta}      (Eq. symbol_sum)
computed from the blocks of a periodic assembly on a 3^d-cell torus (all
operators here reach at most one cell, so no block is aliased), with
    S = I - A_s^{-1} A,  K = I - omega_c I_P A_c^{-1} I_R A,  M = S^{n_s} K S^{n_s},
and rho = sup_theta rho(M(theta)).  The unit cell holds the fine nodes with
local index a in [0, p) and the coarse nodes with b in [0, p/2) per direction
(left/lower edges and the lower-left corner belong to the cell).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from . import fem, qsfem

# ----------------------------------------------------------------------------
# Toy 1-D problem (Section 5)
# ----------------------------------------------------------------------------


def central_difference_weights(M: int) -> np.ndarray:
    """Weights w_j, j = -M..M, of the order-2M central difference for -d^2/dx^2 (h = 1).

    Symmetric weights solved from the moment conditions on x^(2m), m = 0..M:
    sum_j w_j j^(2m) = -2 for m = 1 and 0 otherwise (the exact -d^2/dx^2 of x^2 is -2).
    """
    Amat = np.zeros((M + 1, M + 1))
    rhs = np.zeros(M + 1)
    for mm in range(M + 1):
        Amat[mm, 0] = 1.0 if mm == 0 else 0.0
        for j in range(1, M + 1):
            Amat[mm, j] = 2.0 * float(j) ** (2 * mm)
        rhs[mm] = -2.0 if mm == 1 else 0.0
    half = np.linalg.solve(Amat, rhs)      # (w_0, w_1, ..., w_M)
    return np.concatenate([half[:0:-1], half])


def toy_symbol(theta, k, eps, h, M):
    """tilde A(theta) = h^-2 sum_j w_j e^{i j theta} - (k^2 + i eps)."""
    w = central_difference_weights(M)
    js = np.arange(-M, M + 1)
    s = np.sum(w[:, None] * np.exp(1j * np.outer(js, np.atleast_1d(theta))), axis=0)
    return np.real(s) / h ** 2 - (k * k + 1j * eps)


def toy_M_hat(theta, k, eps, h, M, alpha_s, nu1=1, nu2=1, omega_c=1.0):
    """2x2 two-grid symbol M(theta) on span(e^{i theta x/h}, e^{i(theta+pi) x/h})."""
    A1 = toy_symbol(theta, k, eps, h, M)[0]
    A2 = toy_symbol(theta + math.pi, k, eps, h, M)[0]
    Ac = toy_symbol(2 * theta, k, eps, 2 * h, M)[0]
    As1 = A1 - 1j * alpha_s * k * k
    As2 = A2 - 1j * alpha_s * k * k
    S = np.diag([1 - A1 / As1, 1 - A2 / As2])
    IP = np.array([[0.5 + 0.5 * math.cos(theta)], [0.5 - 0.5 * math.cos(theta)]])
    IR = IP.T.copy()
    K = np.eye(2) - omega_c * (IP @ IR) * (1.0 / Ac) @ np.diag([A1, A2])
    return np.linalg.matrix_power(S, nu2) @ K @ np.linalg.matrix_power(S, nu1)


def toy_rho(k, eps, h, M, alpha_s, thetas=None, **kw):
    if thetas is None:
        thetas = np.linspace(-math.pi / 2, math.pi / 2, 2001, endpoint=False)
    return max(np.max(np.abs(np.linalg.eigvals(toy_M_hat(t, k, eps, h, M, alpha_s, **kw)))) for t in thetas)


def toy_bruteforce_rho(m, k, eps, h, M, alpha_s, nu1=1, nu2=1, omega_c=1.0):
    """Spectral radius of the explicit two-grid iteration matrix on m periodic points."""
    w = central_difference_weights(M)
    A = np.zeros((m, m), dtype=np.complex128)
    for i in range(m):
        for j, wj in zip(range(-M, M + 1), w):
            A[i, (i + j) % m] += wj / h ** 2
    A -= (k * k + 1j * eps) * np.eye(m)
    mc = m // 2
    Ac = np.zeros((mc, mc), dtype=np.complex128)
    for i in range(mc):
        for j, wj in zip(range(-M, M + 1), w):
            Ac[i, (i + j) % mc] += wj / (2 * h) ** 2
    Ac -= (k * k + 1j * eps) * np.eye(mc)
    P = np.zeros((m, mc))
    for J in range(mc):
        P[2 * J, J] = 1.0
        P[(2 * J + 1) % m, J] += 0.5
        P[(2 * J - 1) % m, J] += 0.5
    R = 0.5 * P.T                                   # full weighting [1/4, 1/2, 1/4]
    As = A - 1j * alpha_s * k * k * np.eye(m)
    S = np.eye(m) - np.linalg.solve(As, A)
    K = np.eye(m) - omega_c * P @ np.linalg.solve(Ac, R @ A)
    Mm = np.linalg.matrix_power(S, nu2) @ K @ np.linalg.matrix_power(S, nu1)
    return np.max(np.abs(np.linalg.eigvals(Mm)))


def toy_c(kh):
    """c = (1/4)(1 + cos kh)^2, the factor in Eq. K11hat_1."""
    return 0.25 * (1.0 + np.cos(kh)) ** 2


def lemma_max(c, R):
    """max_theta |f(theta)| = sqrt((1-c)^2 + (|cR|/2)^2) + cR/2   (Eq. max_K11)."""
    return math.sqrt((1 - c) ** 2 + (abs(c * R) / 2) ** 2) + c * R / 2


def lemma_f(theta, c, zeta_f, zeta_c, eps_t):
    return 1 - c * (theta - zeta_f - 1j * eps_t) / (theta - zeta_c - 1j * eps_t)


# ----------------------------------------------------------------------------
# Bloch-wave LFA of the finite-element two-grid method (Section 6)
# ----------------------------------------------------------------------------


def _unit_cell_fine(cell, p, mcells):
    """Global indices (periodic m-cell torus, 2-D) of the fine unit-cell nodes of `cell`."""
    m = mcells * p
    cy, cx = cell
    return np.array([((cy % mcells) * p + ay) * m + (cx % mcells) * p + ax
                     for ay in range(p) for ax in range(p)])


def _unit_cell_coarse(cell, p, mcells):
    q = p // 2
    m = mcells * q
    cy, cx = cell
    return np.array([((cy % mcells) * q + by) * m + (cx % mcells) * q + bx
                     for by in range(q) for bx in range(q)])


class BlochOperators:
    """Blocks P_{0,beta} of A, A_s, A_c, I_P, I_R for constant k, eps (2-D, Q_p, periodic).

    coarse = 'qsfem': A_c is the QSFEM operator of Section 3.3 ('opt');
    coarse = 'gal': A_c = I_R A_{alpha_c} I_P, standard Galerkin p-type coarsening
    of Section 4 (the comparison of Fig. 3 (a)), alpha_c shifting k^2 in the volume term."""

    def __init__(self, p, kh, eps_over_k2, alpha_s, coarse="qsfem", alpha_c=0.0):
        self.p = p
        mc = 3
        n = mc
        h = 1.0 / n
        k = kh / h
        kcell = np.full((n, n), k)
        ecell = np.full((n, n), eps_over_k2 * k * k)
        A = fem.assemble((n, n), p, h, fem.helmholtz_coefficient(kcell, ecell), kcell, (), True)
        As = fem.assemble((n, n), p, h, fem.shifted_coefficient(kcell, ecell, alpha_s), kcell, (), True)
        IP = fem.prolongation(n, p, 2, True)
        IR = IP.T.tocsr()
        if coarse == "qsfem":
            Ac = qsfem.assemble_coarse(n, p, kcell, ecell, (), True)
        elif coarse == "gal":
            Ash = fem.assemble((n, n), p, h, fem.shifted_coefficient(kcell, ecell, alpha_c), kcell, (), True)
            Ac = (IR @ Ash @ IP).tocsr()
        else:
            raise ValueError(coarse)
        betas = list(itertools.product((-1, 0, 1), repeat=2))
        f0 = _unit_cell_fine((0, 0), p, mc)
        c0 = _unit_cell_coarse((0, 0), p, mc)

        def blocks(Mat, rows0, colfn):
            D = Mat.toarray()
            return [(np.array(b), D[np.ix_(rows0, colfn(b))]) for b in betas]

        self.A = blocks(A, f0, lambda b: _unit_cell_fine(b, p, mc))
        self.As = blocks(As, f0, lambda b: _unit_cell_fine(b, p, mc))
        self.Ac = blocks(Ac, c0, lambda b: _unit_cell_coarse(b, p, mc))
        self.IP = blocks(IP, f0, lambda b: _unit_cell_coarse(b, p, mc))
        self.IR = blocks(IR, c0, lambda b: _unit_cell_fine(b, p, mc))

    @staticmethod
    def symbol(blocks, theta):
        th = np.asarray(theta, dtype=float)
        return sum(np.exp(1j * float(th @ b)) * B for b, B in blocks)

    def M_hat(self, theta, n_s=1, omega_c=1.0):
        A = self.symbol(self.A, theta)
        As = self.symbol(self.As, theta)
        Ac = self.symbol(self.Ac, theta)
        IP = self.symbol(self.IP, theta)
        IR = self.symbol(self.IR, theta)
        I = np.eye(A.shape[0])
        S = I - np.linalg.solve(As, A)
        K = I - omega_c * IP @ np.linalg.solve(Ac, IR @ A)
        Sn = np.linalg.matrix_power(S, n_s)
        return Sn @ K @ Sn

    def rho(self, thetas, n_s=1, omega_c=1.0):
        return max(np.max(np.abs(np.linalg.eigvals(self.M_hat(t, n_s, omega_c)))) for t in thetas)


def theta_grid(npts):
    t = -math.pi + 2 * math.pi * np.arange(npts) / npts
    return [np.array([a, b]) for a in t for b in t]


def lfa_rho(p, dofs_per_wavelength, D=0.01, alpha_s=0.2, n_s=1, omega_c=1.0, npts=48, coarse="qsfem", alpha_c=0.0):
    """sup_theta rho(M(theta)) with eps = D k^2 / pi (Section 6, Eq. epsilon_ksquare_D)."""
    kh = 2 * math.pi * p / dofs_per_wavelength
    ops = BlochOperators(p, kh, D / math.pi, alpha_s, coarse, alpha_c)
    return ops.rho(theta_grid(npts), n_s, omega_c)
