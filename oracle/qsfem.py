"""Oracle: dispersion-minimising coarse operator A_q (plain FP64, CPU).

TEST INFRASTRUCTURE ONLY (see oracle/fem.py).

Section 3.2, Eq. P_QSFEM: the compact 3x3 QSFEM stencil
    P0 = 4,
    P1 = 2 (c1 s1 - c2 s2) / den,   P2 = (c2 + s2 - c1 - s1) / den,
    den = c2 s2 (c1 + s1) - c1 s1 (c2 + s2),
    c1 = cos(eta cos(pi/16)), s1 = cos(eta sin(pi/16)),
    c2 = cos(eta cos(3pi/16)), s2 = cos(eta sin(3pi/16)),  eta = k h.
Eq. scaling_factor_QSFEM: N(eta) = -eta^2 / sigma_P(0), sigma_P(0) = P0 + 4 P1 + 4 P2.

Section 3.3, Eq. element_wise_qsfem and the 'quasi finite element' version:
per coarse cell c the contributions q_gamma(h k(c)),
    q_(0,0) = N P0 / 4,  q_edge = N P1 / 2,  q_diag = N P2,
minus i eps(c) times the Q1 cell mass, minus i k times the Q1 face mass on
absorbing boundary edges.

The coarse mesh has spacing 2h/p (Section 4.2), so n p / 2 cells per
direction; each coarse cell lies inside one fine cell and takes that fine
cell's k and eps (the paper states the coefficients are constant per cell).
"""
from __future__ import annotations

import functools
import math

import numpy as np
import scipy.sparse as sp

from . import fem

try:  # extended precision for the QSFEM ratios
    import mpmath as _mp
except ImportError:  # numpy long double is used instead
    _mp = None


def _stencil_scalar(eta: float):
    """(P0, P1, P2, N) at one eta, the formulas as printed, in 50-digit arithmetic.

    The printed ratios lose about eta^-6 units of the working precision (both
    numerators and the denominator vanish like eta^4, and sigma_P(0) like
    eta^2), so they are evaluated in extended precision and rounded once.
    """
    if _mp is not None:
        with _mp.workdps(50):
            e = _mp.mpf(eta)
            c1 = _mp.cos(e * _mp.cos(_mp.pi / 16))
            s1 = _mp.cos(e * _mp.sin(_mp.pi / 16))
            c2 = _mp.cos(e * _mp.cos(3 * _mp.pi / 16))
            s2 = _mp.cos(e * _mp.sin(3 * _mp.pi / 16))
            den = c2 * s2 * (c1 + s1) - c1 * s1 * (c2 + s2)
            P0 = _mp.mpf(4)
            P1 = 2 * (c1 * s1 - c2 * s2) / den
            P2 = (c2 + s2 - c1 - s1) / den
            N = -e * e / (P0 + 4 * P1 + 4 * P2)
            return float(P0), float(P1), float(P2), float(N)
    e = np.longdouble(eta)
    pi = np.longdouble(math.pi)
    c1, s1 = np.cos(e * np.cos(pi / 16)), np.cos(e * np.sin(pi / 16))
    c2, s2 = np.cos(e * np.cos(3 * pi / 16)), np.cos(e * np.sin(3 * pi / 16))
    den = c2 * s2 * (c1 + s1) - c1 * s1 * (c2 + s2)
    P1 = 2 * (c1 * s1 - c2 * s2) / den
    P2 = (c2 + s2 - c1 - s1) / den
    N = -e * e / (4 + 4 * P1 + 4 * P2)
    return 4.0, float(P1), float(P2), float(N)


@functools.lru_cache(maxsize=1 << 16)
def _stencil_cached(eta: float):
    return _stencil_scalar(eta)


def _stencil(eta):
    eta = np.asarray(eta, dtype=float)
    flat = [_stencil_cached(float(v)) for v in eta.reshape(-1)]
    out = np.array(flat).reshape(eta.shape + (4,)) if flat else np.zeros(eta.shape + (4,))
    return out[..., 0], out[..., 1], out[..., 2], out[..., 3]


def qsfem_stencil(eta):
    """(P0, P1, P2) of Eq. P_QSFEM, elementwise in eta."""
    P0, P1, P2, _ = _stencil(eta)
    return P0, P1, P2


def scaling_N(eta):
    """N(eta) = -eta^2 / sigma_P(0) (Eq. scaling_factor_QSFEM)."""
    return _stencil(eta)[3]


def symbol(eta, xi1, xi2):
    """sigma of the scaled operator N P at normalised wave vector (h xi1, h xi2)."""
    P0, P1, P2 = qsfem_stencil(eta)
    N = scaling_N(eta)
    return N * (P0 + 2 * P1 * (np.cos(xi1) + np.cos(xi2)) + 4 * P2 * np.cos(xi1) * np.cos(xi2))


def cell_q(eta):
    """(q00, q_edge, q_diag) = (N P0/4, N P1/2, N P2) for one coarse cell."""
    P0, P1, P2 = qsfem_stencil(eta)
    N = scaling_N(eta)
    return N * P0 / 4.0, N * P1 / 2.0, N * P2


def coarse_cell_fields(k_cell: np.ndarray, eps_cell: np.ndarray, p: int):
    """k, eps on the coarse cells: each fine cell holds (p/2)^d coarse cells."""
    q = p // 2
    kc = k_cell
    ec = eps_cell
    for ax in range(k_cell.ndim):
        kc = np.repeat(kc, q, axis=ax)
        ec = np.repeat(ec, q, axis=ax)
    return kc, ec


def assemble_coarse(n: int, p: int, k_cell: np.ndarray, eps_cell: np.ndarray,
                    robin_sides=(), periodic: bool = False) -> sp.csr_matrix:
    """A_q on the (n p/2)^2 coarse cells with spacing h_c = 2/(n p)  (2-D)."""
    assert k_cell.ndim == 2, "the 9-point scheme is two-dimensional"
    nc = n * p // 2
    hc = 1.0 / nc
    kc, ec = coarse_cell_fields(k_cell, eps_cell, p)
    m = nc + (0 if periodic else 1)
    rows, cols, vals = [], [], []
    Mq = np.array([[1.0 / 3.0, 1.0 / 6.0], [1.0 / 6.0, 1.0 / 3.0]])   # Q1 1-D mass on [0,1]
    for cy in range(nc):
        for cx in range(nc):
            q00, q1, q2 = cell_q(hc * kc[cy, cx])
            verts = [(jy, jx) for jy in (0, 1) for jx in (0, 1)]
            for (ay, ax) in verts:
                ga = ((cy + ay) % m) * m + (cx + ax) % m
                for (by, bx) in verts:
                    gb = ((cy + by) % m) * m + (cx + bx) % m
                    nd = abs(ay - by) + abs(ax - bx)
                    q = (q00, q1, q2)[nd]
                    mass = hc * hc * Mq[ay, by] * Mq[ax, bx]
                    rows.append(ga)
                    cols.append(gb)
                    vals.append(q - 1j * ec[cy, cx] * mass)
    for (axis, end) in robin_sides:
        # axis 0 = y (rows of cells), axis 1 = x
        for c in range(nc):
            if axis == 0:
                cy = 0 if end == 0 else nc - 1
                cx = c
                jy = 0 if end == 0 else 1
                pts = [((cy + jy), cx), ((cy + jy), cx + 1)]
            else:
                cx = 0 if end == 0 else nc - 1
                cy = c
                jx = 0 if end == 0 else 1
                pts = [(cy, cx + jx), (cy + 1, cx + jx)]
            kk = kc[cy, cx]
            for a in range(2):
                for b in range(2):
                    ga = pts[a][0] * m + pts[a][1]
                    gb = pts[b][0] * m + pts[b][1]
                    rows.append(ga)
                    cols.append(gb)
                    vals.append(-1j * kk * hc * Mq[a, b])
    A = sp.coo_matrix((np.array(vals), (np.array(rows), np.array(cols))), shape=(m * m, m * m)).tocsr()
    A.sum_duplicates()
    return A
