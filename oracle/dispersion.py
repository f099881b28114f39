"""Oracle: the dispersion error D_P of a compact 2-D stencil (plain FP64, CPU).

TEST INFRASTRUCTURE ONLY (see oracle/fem.py).

Section 3.2: a constant-coefficient stencil P on the grid h Z^2 multiplies the
plane wave e^{i x.xi} by its symbol sigma_P(xi) (Eq. symbol_sigma_P); its
propagating waves are the zero set Z_P of sigma_P, and its distance to the
true zero set {|xi| = k} is

    D_P = max_{t in [-pi, pi]} min_{xi in Z_P} || k (cos t, sin t) - xi || .

For the symmetric 3 x 3 stencils used here (corner P2, edge P1, centre P0)

    sigma_P(xi) = P0 + 2 P1 (cos h xi_1 + cos h xi_2) + 4 P2 cos h xi_1 cos h xi_2 ,

and the zero set does not depend on a common scale of P0, P1, P2.  Lengths
are in units of 1/h (z = h xi, eta = k h); the functions return D_P / k,
i.e. distances divided by eta.

Stencils (all for -Laplace - k^2 on a grid of spacing h, up to scale):
  * 'qsfem': the dispersion-minimising stencil of Eq. P_QSFEM (P0 = 4, P1, P2
    from the printed ratios, evaluated in 50-digit arithmetic by
    oracle.qsfem.cell_q);
  * 'q1':    the bilinear finite element, stiffness minus eta^2 times mass
    (the Q1 stencils of Section 3.3, Eq. fd_fe_constant1);
  * 'fd5':   the 5-point central difference, P = (4 - eta^2, -1, 0).

How Z_P is traced: along each polar direction s the nearest zero of sigma_P to
the origin, r(s), is bracketed on a grid of the ray and refined by bisection;
min over xi in Z_P is then a minimisation over s of |eta e_t - r(s) e_s|,
first on a dense grid of s around t, then refined by bounded scalar
minimisation (the zero curve is close to the circle, so the nearest point lies
near the ray of t).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq, minimize_scalar

from . import qsfem


def stencil(kind: str, eta: float):
    """(P0, P1, P2) of the named stencil at eta = k h."""
    if kind == "qsfem":
        q00, q1, q2 = qsfem.cell_q(eta)          # per-cell weights N P0/4, N P1/2, N P2
        return 4.0 * q00, 2.0 * q1, q2            # assembled: 4 cells, 2 cells, 1 cell
    if kind == "q1":
        e2 = eta * eta
        return 8.0 / 3.0 - 16.0 * e2 / 36.0, -1.0 / 3.0 - 4.0 * e2 / 36.0, -1.0 / 3.0 - e2 / 36.0
    if kind == "fd5":
        return 4.0 - eta * eta, -1.0, 0.0
    raise ValueError(kind)


def symbol(P, z1, z2):
    P0, P1, P2 = P
    return P0 + 2.0 * P1 * (np.cos(z1) + np.cos(z2)) + 4.0 * P2 * np.cos(z1) * np.cos(z2)


def radius(P, s: float, eta: float) -> float:
    """Smallest r > 0 with sigma_P(r cos s, r sin s) = 0 (the zero set along the ray)."""
    c, sn = math.cos(s), math.sin(s)
    f = lambda r: symbol(P, r * c, r * sn)
    rs = np.linspace(1e-3 * eta, 3.0 * max(eta, 0.5), 3001)
    v = f(rs)
    k = np.nonzero(np.sign(v[:-1]) != np.sign(v[1:]))[0]
    if k.size == 0:
        raise ValueError("no propagating zero along the ray")
    i = int(k[0])
    return brentq(f, rs[i], rs[i + 1], xtol=1e-15, rtol=1e-15, maxiter=200)


def distance(P, t: float, eta: float, width: float = 0.3, samples: int = 601) -> float:
    """min over xi in Z_P of |eta (cos t, sin t) - xi|, divided by eta."""
    def d2(s):
        # |eta e_t - r e_s|^2 written without cancellation
        r = radius(P, s, eta)
        return (r - eta) ** 2 + 4.0 * eta * r * math.sin(0.5 * (s - t)) ** 2

    ss = np.linspace(t - width, t + width, samples)
    vals = np.array([d2(s) for s in ss])
    i = int(np.argmin(vals))
    lo, hi = ss[max(i - 1, 0)], ss[min(i + 1, samples - 1)]
    res = minimize_scalar(d2, bounds=(lo, hi), method="bounded", options={"xatol": 1e-12})
    best = min(float(res.fun), float(vals[i]))
    return math.sqrt(max(best, 0.0)) / eta


def dispersion_error(kind: str, eta: float, nt: int = 64):
    """D_P / k over the directions t_j = -pi + 2 pi j / nt: (max, per-direction values)."""
    P = stencil(kind, eta)
    ts = -math.pi + 2.0 * math.pi * np.arange(nt) / nt
    d = np.array([distance(P, float(t), eta) for t in ts])
    return float(d.max()), d
