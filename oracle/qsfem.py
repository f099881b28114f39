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


# ----------------------------------------------------------------------------
# Three dimensions: a fitted 27-point stencil.  The paper only cites a 3-D
# dispersion-minimising scheme; this one is the project's own construction on
# the pattern of Eq. P_QSFEM (a reading, not the cited scheme):
#   sigma_P(xi) = P0 + 2 P1 sum_a cos xi_a + 4 P2 sum_{a<b} cos xi_a cos xi_b
#                 + 8 P3 cos xi_1 cos xi_2 cos xi_3,
# P0 = 8 and P1, P2, P3 chosen so that sigma_P vanishes at |xi| = eta along the
# three directions DIRS3 (the 2-D construction's exact zeros at pi/16 and
# 3 pi/16 are the midpoints of the halves of the symmetry-reduced arc [0, pi/4];
# here the directions are the images of the interior 3-point rule
# (2/3, 1/6, 1/6) of the symmetry-reduced spherical triangle with corners
# (0,0,1), (0,1,1)/sqrt2, (1,1,1)/sqrt3, normalised).  N = -eta^2 / sigma_P(0)
# as in Eq. scaling_factor_QSFEM.  The operator is h_c N P (the 3-D finite
# element forms scale with h), minus i eps h_c^3 times the Q1 mass and minus
# i k h_c^2 times the Q1 face mass on absorbing faces; per coarse cell the pair
# weights are N P0/8, N P1/4, N P2/2, N P3 by the number of coordinates in
# which the two vertices differ.
# ----------------------------------------------------------------------------

def _dirs3():
    V = np.array([[0.0, 0.0, 1.0], [0.0, 1.0, 1.0] / np.sqrt(2.0), [1.0, 1.0, 1.0] / np.sqrt(3.0)])
    out = []
    for w in ([2 / 3, 1 / 6, 1 / 6], [1 / 6, 2 / 3, 1 / 6], [1 / 6, 1 / 6, 2 / 3]):
        d = np.asarray(w) @ V
        out.append(d / np.linalg.norm(d))
    return np.array(out)


DIRS3 = _dirs3()


def _stencil27_scalar(eta: float):
    """(P0, P1, P2, P3, N) at one eta: the three zero conditions solved in 50 digits."""
    if _mp is not None:
        with _mp.workdps(50):
            e = _mp.mpf(eta)
            rows, rhs = [], []
            for d in DIRS3:
                c = [_mp.cos(e * _mp.mpf(float(x))) for x in d]
                rows.append([2 * (c[0] + c[1] + c[2]), 4 * (c[0] * c[1] + c[0] * c[2] + c[1] * c[2]),
                             8 * c[0] * c[1] * c[2]])
                rhs.append(-8)
            sol = _mp.lu_solve(_mp.matrix(rows), _mp.matrix(rhs))
            P1, P2, P3 = sol[0], sol[1], sol[2]
            s0 = 8 + 6 * P1 + 12 * P2 + 8 * P3
            return 8.0, float(P1), float(P2), float(P3), float(-e * e / s0)
    e = np.longdouble(eta)
    rows, rhs = [], []
    for d in DIRS3:
        c = np.cos(e * d.astype(np.longdouble))
        rows.append([2 * c.sum(), 4 * (c[0] * c[1] + c[0] * c[2] + c[1] * c[2]), 8 * c.prod()])
        rhs.append(-8.0)
    P1, P2, P3 = np.linalg.solve(np.array(rows, dtype=float), np.array(rhs))
    return 8.0, P1, P2, P3, -eta * eta / (8 + 6 * P1 + 12 * P2 + 8 * P3)


@functools.lru_cache(maxsize=1 << 16)
def _stencil27_cached(eta: float):
    return _stencil27_scalar(eta)


def stencil27(eta: float):
    """(P0, P1, P2, P3, N) of the fitted 27-point scheme at eta."""
    return _stencil27_cached(float(eta))


def symbol27(eta, xi):
    """N sigma_P(xi) of the fitted 27-point scheme (xi: 3 normalised wave-vector components)."""
    P0, P1, P2, P3, N = stencil27(eta)
    c = np.cos(np.asarray(xi, dtype=float))
    return N * (P0 + 2 * P1 * c.sum() + 4 * P2 * (c[0] * c[1] + c[0] * c[2] + c[1] * c[2]) + 8 * P3 * c.prod())


def cell_q27(eta):
    """(q_0, q_1, q_2, q_3) = (N P0/8, N P1/4, N P2/2, N P3) for one coarse cell."""
    P0, P1, P2, P3, N = stencil27(eta)
    return N * P0 / 8.0, N * P1 / 4.0, N * P2 / 2.0, N * P3


def assemble_coarse3(n: int, p: int, k_cell: np.ndarray, eps_cell: np.ndarray,
                     robin_sides=(), periodic: bool = False) -> sp.csr_matrix:
    """A_q on the (n p/2)^3 coarse cells with spacing h_c = 2/(n p)  (3-D, fitted 27-point)."""
    nc = n * p // 2
    hc = 1.0 / nc
    kc, ec = coarse_cell_fields(k_cell, eps_cell, p)
    m = nc + (0 if periodic else 1)
    Mq = np.array([[1.0 / 3.0, 1.0 / 6.0], [1.0 / 6.0, 1.0 / 3.0]])
    verts = [(a, b, c) for a in (0, 1) for b in (0, 1) for c in (0, 1)]
    rows, cols, vals = [], [], []
    gid = lambda z, y, x: ((z % m) * m + (y % m)) * m + (x % m)
    for cz in range(nc):
        for cy in range(nc):
            for cx in range(nc):
                q = cell_q27(hc * kc[cz, cy, cx])
                for va in verts:
                    ga = gid(cz + va[0], cy + va[1], cx + va[2])
                    for vb in verts:
                        gb = gid(cz + vb[0], cy + vb[1], cx + vb[2])
                        nd = sum(int(va[i] != vb[i]) for i in range(3))
                        mass = hc ** 3 * Mq[va[0], vb[0]] * Mq[va[1], vb[1]] * Mq[va[2], vb[2]]
                        rows.append(ga)
                        cols.append(gb)
                        vals.append(hc * q[nd] - 1j * ec[cz, cy, cx] * mass)
    for (axis, end) in robin_sides:
        j = 0 if end == 0 else 1
        c_axis = 0 if end == 0 else nc - 1
        for c1 in range(nc):
            for c2 in range(nc):
                cell = [0, 0, 0]
                others = [a for a in range(3) if a != axis]
                cell[axis] = c_axis
                cell[others[0]], cell[others[1]] = c1, c2
                kk = kc[tuple(cell)]
                face = []
                for a in (0, 1):
                    for b in (0, 1):
                        v = list(cell)
                        v[axis] += j
                        v[others[0]] += a
                        v[others[1]] += b
                        face.append((gid(*v), a, b))
                for (ga, a1, b1) in face:
                    for (gb, a2, b2) in face:
                        rows.append(ga)
                        cols.append(gb)
                        vals.append(-1j * kk * hc * hc * Mq[a1, a2] * Mq[b1, b2])
    A = sp.coo_matrix((np.array(vals), (np.array(rows), np.array(cols))), shape=(m ** 3, m ** 3)).tocsr()
    A.sum_duplicates()
    return A


def assemble_coarse(n: int, p: int, k_cell: np.ndarray, eps_cell: np.ndarray,
                    robin_sides=(), periodic: bool = False) -> sp.csr_matrix:
    """A_q on the (n p/2)^d coarse cells with spacing h_c = 2/(n p)."""
    if k_cell.ndim == 3:
        return assemble_coarse3(n, p, k_cell, eps_cell, robin_sides, periodic)
    assert k_cell.ndim == 2, "the coarse schemes are two- or three-dimensional"
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
