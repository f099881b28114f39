"""Pins of the dispersion-error oracle (oracle/dispersion.py, Section 3.2's D_P).

* 5-point differences: the zero set along the axes and the diagonals has a
  closed form, r = 2 asin(eta/2) and 2 sqrt(2) asin(eta / (2 sqrt(2))), and by
  symmetry the nearest zero to eta e_t lies on those rays.
* Bilinear elements: along the axes cos r = -(P0 + 2 P1) / (2 P1 + 4 P2).
* The QSFEM stencil vanishes exactly on |xi| = k along pi/16 and 3 pi/16
  (the construction of Eq. P_QSFEM), so D_P's inner minimum is 0 there; its
  D_P is far below the finite element's and the finite difference's.
* The minimum over the zero set, not the radial distance: checked against
  zero crossings of the symbol located on a fine Cartesian grid around the
  point (marching over grid edges), an independent route to Z_P.
"""
import math

import numpy as np
import pytest

from oracle import dispersion as D


@pytest.mark.parametrize("eta", [0.3, 1.0, 2 * math.pi / 5])
def test_fd5_axis_and_diagonal_closed_forms(eta):
    P = D.stencil("fd5", eta)
    ax = 2 * math.asin(eta / 2) / eta - 1
    dg = 2 * math.sqrt(2) * math.asin(eta / (2 * math.sqrt(2))) / eta - 1
    assert abs(D.distance(P, 0.0, eta) - ax) < 1e-12
    assert abs(D.distance(P, math.pi / 2, eta) - ax) < 1e-12
    assert abs(D.distance(P, math.pi / 4, eta) - dg) < 1e-12
    assert abs(D.distance(P, -3 * math.pi / 4, eta) - dg) < 1e-12


@pytest.mark.parametrize("eta", [0.5, 1.2])
def test_q1_axis_closed_form(eta):
    P0, P1, P2 = P = D.stencil("q1", eta)
    r = math.acos(-(P0 + 2 * P1) / (2 * P1 + 4 * P2))
    assert abs(D.distance(P, 0.0, eta) - abs(r - eta) / eta) < 1e-12
    # the stencil is the Q1 stiffness minus eta^2 times the Q1 mass of Section 3.3
    assert abs(P0 + 4 * P1 + 4 * P2 + eta ** 2) < 1e-14


@pytest.mark.parametrize("eta", [0.5, 1.0, 2 * math.pi / 5])
def test_qsfem_exact_zeros_and_symmetry(eta):
    P = D.stencil("qsfem", eta)
    for t in (math.pi / 16, 3 * math.pi / 16, 5 * math.pi / 16, -7 * math.pi / 16):
        assert D.distance(P, t, eta) < 1e-10
    for t in (0.1, 0.45):
        d = D.distance(P, t, eta)
        assert abs(D.distance(P, -t, eta) - d) < 1e-12
        assert abs(D.distance(P, math.pi / 2 - t, eta) - d) < 1e-12
    dq, _ = D.dispersion_error("qsfem", eta, nt=16)
    d1, _ = D.dispersion_error("q1", eta, nt=16)
    d5, _ = D.dispersion_error("fd5", eta, nt=16)
    assert dq < 1e-3 * d1 and d1 < d5


@pytest.mark.parametrize("kind,eta,t", [("q1", 1.0, 0.3), ("fd5", 1.3, 0.5), ("q1", 0.8, -2.0)])
def test_minimum_over_zero_set_matches_grid_crossings(kind, eta, t):
    P = D.stencil(kind, eta)
    d = D.distance(P, t, eta)
    x0 = np.array([math.cos(t), math.sin(t)]) * eta
    half = 2.0 * d * eta
    n = 2001
    g = np.linspace(-half, half, n)
    Z1, Z2 = np.meshgrid(x0[0] + g, x0[1] + g, indexing="ij")
    S = D.symbol(P, Z1, Z2)
    pts = []
    for ax in (0, 1):   # sign changes along grid edges, linear interpolation
        a = S[:-1, :] if ax == 0 else S[:, :-1]
        b = S[1:, :] if ax == 0 else S[:, 1:]
        m = np.sign(a) != np.sign(b)
        w = a[m] / (a[m] - b[m])
        if ax == 0:
            p1 = Z1[:-1, :][m] + w * (Z1[1:, :][m] - Z1[:-1, :][m])
            p2 = Z2[:-1, :][m]
        else:
            p1 = Z1[:, :-1][m]
            p2 = Z2[:, :-1][m] + w * (Z2[:, 1:][m] - Z2[:, :-1][m])
        pts.append(np.stack([p1, p2], 1))
    pts = np.concatenate(pts)
    dgrid = np.min(np.hypot(pts[:, 0] - x0[0], pts[:, 1] - x0[1])) / eta
    assert abs(dgrid - d) < 1e-6 * max(1.0, d), (dgrid, d)
    # and the radial distance is not the minimum (the check can tell them apart)
    r = D.radius(P, t, eta)
    assert abs(r - eta) / eta - d > 1e-6
