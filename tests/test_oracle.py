"""Pins of the FP64 CPU oracle against facts the paper and the mathematics fix.

Each test checks a property that a plausible mistake (dropped term, wrong
sign, transposed operand, wrong index) would break.  CPU only.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import dd, fem, krylov, lfa, qsfem, twogrid

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


# ---------------------------------------------------------------- 1-D element
@pytest.mark.parametrize("p", [1, 2, 3, 4, 6, 8])
def test_reference_matrices_polynomial_exactness(p):
    """x^i interpolated at the GLL nodes is exact; M, K integrate products exactly."""
    M, K = fem.reference_matrices(p)
    x = fem.gll_points(p)
    for i in range(p + 1):
        for j in range(p + 1):
            ci, cj = x ** i, x ** j
            assert abs(ci @ M @ cj - 1.0 / (i + j + 1)) < 1e-12
            dk = 0.0 if (i == 0 or j == 0) else i * j / (i + j - 1)
            assert abs(ci @ K @ cj - dk) < 1e-10 * max(1.0, dk)


def test_gll_points_are_lobatto():
    # the 5 GLL points on [-1,1] are 0, +-sqrt(3/7), +-1
    x = 2 * fem.gll_points(4) - 1
    assert np.allclose(x, [-1, -math.sqrt(3 / 7), 0, math.sqrt(3 / 7), 1], atol=1e-14)


# ------------------------------------------------------------- fine assembly
def test_q1_stencils_match_paper():
    g = _golden("q1_stencils.json")
    n, h = 3, 1.0 / 3
    ones = np.ones((n, n))
    S = fem.assemble((n, n), 1, h, 0 * ones, ones).toarray().real       # stiffness only
    Mm = -fem.assemble((n, n), 1, h, ones, 0 * ones).toarray().real + S  # mass (c = 1)
    m = n + 1
    c = 1 * m + 1
    assert abs(S[c, c] - g["stiffness_center"]) < 1e-14
    assert abs(S[c, c + 1] - g["stiffness_edge_neighbour"]) < 1e-14
    assert abs(S[c, c + m + 1] - g["stiffness_corner_neighbour"]) < 1e-14
    assert abs(Mm[c, c] / h ** 2 - g["mass_center_over_h2"]) < 1e-14
    assert abs(Mm[c, c + m] / h ** 2 - g["mass_edge_over_h2"]) < 1e-14
    assert abs(Mm[c, c + m + 1] / h ** 2 - g["mass_corner_over_h2"]) < 1e-14


def test_fine_matrices_complex_symmetric():
    w = synth.workload("square10_q4_n25")
    eps = synth.absorbing_layer(w["n"], 2, w["p"], w["k"])
    P = twogrid.Problem(w["n"], w["p"], w["k"], eps, coarse=True)
    for M in (P.A, P.As, P.Aq):
        d = abs(M - M.T).max()
        assert d <= 1e-13 * abs(M).max()


def _boundary_load(n, p, kk, g):
    """b_j = int_{boundary} g phi_j ds, Gauss quadrature on every boundary edge."""
    nodes = fem.gll_points(p)
    xq, wq = fem.gauss_legendre(p + 3)
    V = fem.lagrange_values(nodes, xq)
    h = 1.0 / n
    m = n * p + 1
    b = np.zeros(m * m, dtype=complex)
    for e in range(n):
        s = e * h + h * xq
        for (side, pts, idx) in (
            ("b", (s, 0 * s), [0 * m + e * p + a for a in range(p + 1)]),
            ("t", (s, 0 * s + 1), [(m - 1) * m + e * p + a for a in range(p + 1)]),
            ("l", (0 * s, s), [(e * p + a) * m for a in range(p + 1)]),
            ("r", (0 * s + 1, s), [(e * p + a) * m + m - 1 for a in range(p + 1)]),
        ):
            nrm = {"b": (0, -1), "t": (0, 1), "l": (-1, 0), "r": (1, 0)}[side]
            gv = g(pts[0], pts[1], nrm)
            b[idx] += h * (V.T @ (wq * gv))
    return b


@pytest.mark.parametrize("p", [2, 4])
def test_plane_wave_convergence_rate(p):
    """Robin data of an exact plane wave: L2 error decays like h^(p+1)."""
    kk = 4.0
    d = (math.cos(0.3), math.sin(0.3))

    def u(x, y):
        return np.exp(1j * kk * (d[0] * x + d[1] * y))

    def g(x, y, nrm):   # du/dn - i k u
        return 1j * kk * (d[0] * nrm[0] + d[1] * nrm[1] - 1.0) * u(x, y)

    errs = []
    ns = [2, 4, 8]
    for n in ns:
        kc = np.full((n, n), kk)
        A = fem.assemble((n, n), p, 1.0 / n, kc ** 2 + 0j, kc, fem.robin_set(2, "robin"))
        b = _boundary_load(n, p, kk, g)
        uh = spla.spsolve(A.tocsc(), b)
        errs.append(fem.l2_error_2d(n, p, uh, u))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(ns) - 1)]
    assert rates[-1] > p + 1 - 0.35, (errs, rates)


def test_robin_sign_gives_outgoing_wave():
    """With -i k on the boundary the 1-D problem -u'' - k^2 u = 0, u'(0) = -1 ... is solved by e^{ikx}."""
    # 2-D strip with Neumann top/bottom reduces to 1-D: plane wave along x, Robin at x=1 only
    # (outgoing), inhomogeneous Neumann at x=0.
    n, p, kk = 8, 4, 5.0
    kc = np.full((n, n), kk)
    A = fem.assemble((n, n), p, 1.0 / n, kc ** 2 + 0j, kc, [(1, 1)])
    m = n * p + 1
    # b = int_{x=0} (-du/dx) phi ds with u = e^{ikx}: -du/dx = -i k
    b = np.zeros(m * m, dtype=complex)
    nodes = fem.gll_points(p)
    Mref, _ = fem.reference_matrices(p)
    for e in range(n):
        idx = [(e * p + a) * m for a in range(p + 1)]
        b[idx] += (1.0 / n) * Mref.sum(axis=1) * (-1j * kk)
    uh = spla.spsolve(A.tocsc(), b)
    x = fem.node_coordinates_1d(n, p)
    ref = np.exp(1j * kk * x)
    got = uh.reshape(m, m)[m // 2]
    assert np.max(np.abs(got - ref)) < 1e-5


# ---------------------------------------------------------------------- QSFEM
@pytest.mark.parametrize("eta", [0.1, 0.3, 0.5, 1.0, 2 * math.pi / 5, 2.0])
def test_qsfem_exact_zeros_on_pi16_directions(eta):
    for j in (1, 3, 5, 7, 9, 11, 13, 15, 17, 19, 21, 23, 25, 27, 29, 31):
        t = j * math.pi / 16
        s = qsfem.symbol(eta, eta * math.cos(t), eta * math.sin(t))
        assert abs(s) < 1e-12 * eta ** 2 + 1e-13
    # and nonzero elsewhere on the circle (the stencil is not exact everywhere)
    assert abs(qsfem.symbol(eta, eta, 0.0)) > 1e-6 * eta ** 8      # error ~ 2.6e-6 eta^8 along theta = 0
    # sigma_{N P}(0) = -eta^2
    assert abs(qsfem.symbol(eta, 0.0, 0.0) + eta ** 2) < 1e-13 * eta ** 2


def test_coarse_operator_annihilates_dispersion_matched_wave():
    """Assembled periodic A_q (eps = 0) kills the discrete plane wave along pi/16."""
    n, p = 6, 4
    nc = n * p // 2
    hc = 1.0 / nc
    # choose k so that the wave is periodic on the torus along x only is impossible
    # for a generic direction; instead check the interior rows of a non-periodic
    # assembly on a wave of exact |xi| = k along 3 pi/16.
    kk = 2 * math.pi / (5 * hc)            # 5 coarse points per wavelength
    kc = np.full((n, n), kk)
    Aq = qsfem.assemble_coarse(n, p, kc, 0 * kc, (), False)
    m = nc + 1
    t = 3 * math.pi / 16
    X, Y = np.meshgrid(np.arange(m) * hc, np.arange(m) * hc)
    wave = np.exp(1j * kk * (math.cos(t) * X + math.sin(t) * Y)).reshape(-1)
    r = (Aq @ wave).reshape(m, m)
    interior = r[1:-1, 1:-1]
    scale = abs(Aq).max()
    assert np.max(np.abs(interior)) < 1e-12 * scale
    # and the boundary rows do not vanish (the natural condition is not exact)
    assert np.max(np.abs(r[0, :])) > 1e-6 * scale


def test_coarse_mass_term_matches_q1_mass():
    """The eps part of A_q is -i eps times the Q1 mass of the paper (Section 3.3)."""
    g = _golden("q1_stencils.json")
    n, p = 3, 4
    nc = n * p // 2
    hc = 1.0 / nc
    kc = np.full((n, n), 10.0)
    A0 = qsfem.assemble_coarse(n, p, kc, 0 * kc).toarray()
    A1 = qsfem.assemble_coarse(n, p, kc, 0 * kc + 1.0).toarray()
    Mm = (A0 - A1) / 1j            # = Q1 mass
    m = nc + 1
    c = 2 * m + 2
    assert abs(Mm[c, c] / hc ** 2 - g["mass_center_over_h2"]) < 1e-13
    assert abs(Mm[c, c + 1] / hc ** 2 - g["mass_edge_over_h2"]) < 1e-13
    assert abs(Mm[c, c + m + 1] / hc ** 2 - g["mass_corner_over_h2"]) < 1e-13


@pytest.mark.parametrize("side", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_coarse_absorbing_term_is_minus_ik_boundary_integral(side):
    """The Gamma_abs term of the 'quasi finite element' A_q (Section 3.3):
    adding an absorbing side adds the bilinear form -i int_side k phi_a phi_b ds
    with k constant per coarse cell.  Checked without the oracle's 1-D mass
    matrix: for nodal vectors v, w on the side, the Q1 basis represents the
    piecewise-linear interpolants I v, I w, whose product is quadratic on each
    cell and is integrated exactly by Simpson's rule.  A wrong scale (h_c^2
    for h_c), sign, mass entry or cell of k fails here."""
    n, p = 3, 4
    q = p // 2
    nc = n * q
    hc = 1.0 / nc
    m = nc + 1
    kf = synth.rng(17).uniform(3.0, 9.0, (n, n))           # k per fine cell [cy, cx]
    B0 = qsfem.assemble_coarse(n, p, kf, 0 * kf, ())
    B1 = qsfem.assemble_coarse(n, p, kf, 0 * kf, [side])
    D = (B1 - B0).toarray()
    axis, end = side
    grid = np.arange(m * m).reshape(m, m)                    # [iy, ix]
    j = 0 if end == 0 else m - 1
    nodes = grid[j, :] if axis == 0 else grid[:, j]          # ordered along the side
    fine_row = 0 if end == 0 else n - 1
    # k of the coarse cell c along the side: the fine cell that contains it
    ks = np.array([kf[fine_row, c // q] if axis == 0 else kf[c // q, fine_row] for c in range(nc)])
    off = np.ones(m * m, bool)
    off[nodes] = False
    assert np.all(D[off, :] == 0) and np.all(D[:, off] == 0)
    Ds = D[np.ix_(nodes, nodes)]
    r = synth.rng(18)
    for _ in range(4):
        v = r.standard_normal(m) + 1j * r.standard_normal(m)
        w = r.standard_normal(m) + 1j * r.standard_normal(m)
        fl, fr = v[:-1] * w[:-1], v[1:] * w[1:]
        fm = 0.25 * (v[:-1] + v[1:]) * (w[:-1] + w[1:])
        want = -1j * np.sum(ks * hc / 6.0 * (fl + 4.0 * fm + fr))
        assert abs(v @ Ds @ w - want) < 1e-13 * max(1.0, abs(want))
    # v = w = 1: the side integral of k
    assert abs(D.sum() + 1j * np.sum(ks) * hc) < 1e-13 * np.sum(ks)


# --------------------------------------------------------------- prolongation
@pytest.mark.parametrize("p", [2, 4, 6])
def test_prolongation_reproduces_half_degree_polynomials(p):
    n = 3
    q = p // 2
    IP = fem.prolongation(n, p, 2)
    xc = np.linspace(0, 1, n * q + 1)
    xf = fem.node_coordinates_1d(n, p)
    for a in range(q + 1):
        for b in range(q + 1):
            uc = np.outer(xc ** b, xc ** a).reshape(-1)       # y^b x^a
            uf = np.outer(xf ** b, xf ** a).reshape(-1)
            assert np.max(np.abs(IP @ uc - uf)) < 1e-13
    # degree q+1 is not reproduced (guards against an accidental identity)
    uc = np.outer(np.ones_like(xc), xc ** (q + 1)).reshape(-1)
    uf = np.outer(np.ones_like(xf), xf ** (q + 1)).reshape(-1)
    assert np.max(np.abs(IP @ uc - uf)) > 1e-6


# ------------------------------------------------------------------- smoother
def test_partition_sizes():
    assert dd.partition_1d(25, 2) == [(2 * i, 2) for i in range(12)] + [(24, 1)]
    assert [s for _, s in dd.partition_1d(25, 4)] == [4, 4, 4, 4, 3, 3, 3]
    assert dd.partition_1d(100, 2)[-1] == (98, 2)


def _small_problem(n=6, p=4, W=1.5, alpha_s=0.5, bc="robin", seed=3):
    k = synth.random_wavenumber(n, 2, W, seed=seed)
    eps = synth.absorbing_layer(n, 2, p, k, 6.0)
    return twogrid.Problem(n, p, k, eps, bc=bc, alpha_s=alpha_s)


def test_ddstep_fixed_point_is_shifted_solution():
    """If A_s u = f then DDStep(u, f) = u: checks the correction term and the averaging."""
    for bc in ("robin", "neumann", {(0, 0): "robin", (1, 1): "robin"}):
        P = _small_problem(bc=bc)
        S = dd.DDSmoother(P, 2)
        f = synth.random_complex(P.N, 7)
        u = spla.spsolve(P.As.tocsc(), f)
        v = S.dd_step(u, f)
        assert np.linalg.norm(v - u) < 1e-10 * np.linalg.norm(u)
        # and a generic u is not a fixed point
        u2 = synth.random_complex(P.N, 8)
        assert np.linalg.norm(S.dd_step(u2, f) - u2) > 1e-3 * np.linalg.norm(u2)


def test_single_subdomain_smoother_is_exact_shifted_solve():
    P = _small_problem(n=4)
    S = dd.DDSmoother(P, 4)
    assert len(S.subs) == 1
    f = synth.random_complex(P.N, 1)
    u = synth.random_complex(P.N, 2)
    got = S.smooth(u, f, n_dd=1)
    want = u + spla.spsolve(P.As.tocsc(), f - P.A @ u)
    assert np.linalg.norm(got - want) < 1e-11 * np.linalg.norm(want)


def test_subdomain_matrix_interior_rows_match_global():
    """Rows of A_s^(i) at dofs away from the internal boundary equal rows of A_s."""
    P = _small_problem(n=6)
    S = dd.DDSmoother(P, 2)
    As = P.As.toarray()
    for sd in S.subs:
        Al = sd.As.toarray()
        # dofs of U^(i) lie at least one cell inside Omega^(i) or on the true boundary
        for il in sd.u_local:
            g = sd.omega_dofs[il]
            row_g = As[g, sd.omega_dofs]
            assert np.allclose(Al[il], row_g, atol=1e-12 * abs(As).max())
            assert abs(As[g]).sum() - abs(row_g).sum() < 1e-10 * abs(As).max()


def test_multiplicity_counts():
    P = _small_problem(n=5)
    S = dd.DDSmoother(P, 2)
    m = 5 * 4 + 1
    L = S.L.reshape(m, m)
    assert L.min() == 1 and L.max() == 4
    # interfaces between blocks of 2 cells: x = 8, 16 (dof index)
    assert L[3, 8] == 2 and L[8, 8] == 4 and L[8, 3] == 2 and L[3, 3] == 1


# ------------------------------------------------------------------- two-grid
def test_two_grid_exact_solution_is_fixed_point():
    P = _small_problem()
    TG = twogrid.TwoGrid(P, l_dd=2)
    f = synth.random_complex(P.N, 11)
    u = spla.spsolve(P.A.tocsc(), f)
    assert np.linalg.norm(TG.step(u, f) - u) < 1e-9 * np.linalg.norm(u)


def test_banded_coarse_solve_matches_splu():
    P = _small_problem(n=8)
    B = twogrid.BandedSolver(P.Aq)
    b = synth.random_complex(P.Nc, 5)
    x1 = B.solve(b)
    x2 = spla.splu(P.Aq.tocsc()).solve(b)
    assert np.linalg.norm(x1 - x2) < 1e-11 * np.linalg.norm(x2)


@pytest.mark.parametrize("p,ppw,n_s,omega_c,coarse,alpha_c", [(4, 10, 1, 1.0, "qsfem", 0.0), (4, 8, 2, 0.8, "qsfem", 0.0),
                                                               (2, 12, 1, 1.0, "qsfem", 0.0), (4, 8, 1, 1.0, "gal", 0.0),
                                                               (6, 10, 1, 1.0, "gal", 0.05)])
def test_bruteforce_spectral_radius_equals_bloch_lfa(p, ppw, n_s, omega_c, coarse, alpha_c):
    """rho of the oracle's own TwoGridStep on a periodic torus (one subdomain = exact
    shifted smoother) equals sup over the torus' Bloch vectors of rho(M(theta)),
    for the QSFEM and the Galerkin coarse level."""
    mcells, D, alpha_s = 4, 0.01, 0.2
    kh = 2 * math.pi * p / ppw
    k = kh * mcells
    kc = np.full((mcells, mcells), k)
    ec = np.full((mcells, mcells), D * k * k / math.pi)
    P = twogrid.Problem(mcells, p, kc, ec, alpha_s=alpha_s, periodic=True, coarse_kind=coarse, alpha_c=alpha_c)
    TG = twogrid.TwoGrid(P, l_dd=mcells, n_s=n_s, omega_c=omega_c, coarse_solver="splu")
    N = P.N
    M = np.zeros((N, N), dtype=complex)
    z = np.zeros(N, dtype=complex)
    for j in range(N):
        e = np.zeros(N, dtype=complex)
        e[j] = 1.0
        M[:, j] = TG.step(e, z)
    rho_brute = np.max(np.abs(np.linalg.eigvals(M)))
    ops = lfa.BlochOperators(p, kh, D / math.pi, alpha_s, coarse, alpha_c)
    ths = [2 * math.pi * np.array([a, b]) / mcells for a in range(mcells) for b in range(mcells)]
    rho_lfa = ops.rho(ths, n_s, omega_c)
    assert abs(rho_brute - rho_lfa) < 1e-9 * max(1.0, rho_lfa)


def test_lfa_convergence_thresholds():
    """Section 6: order 4 converges at ~8+ dofs per wavelength, order 6 from 7."""
    assert lfa.lfa_rho(4, 10, npts=24) < 0.5
    assert lfa.lfa_rho(4, 6, npts=24) > 1.0
    assert lfa.lfa_rho(6, 7, npts=20) < 1.0
    assert lfa.lfa_rho(6, 6, npts=20) > 1.0


# ------------------------------------------------------------------------ toy
def test_toy_bruteforce_equals_lfa():
    m, ppw = 32, 10
    h = 1.0 / m
    k = 2 * math.pi / (ppw * h)
    eps = k * k * 0.01 / math.pi
    thetas = [2 * math.pi * j / m for j in range(-m // 4, m // 4)]
    for M in (1, 2):
        a = lfa.toy_bruteforce_rho(m, k, eps, h, M, 0.2)
        b = lfa.toy_rho(k, eps, h, M, 0.2, thetas=thetas)
        assert abs(a - b) < 1e-10 * max(1.0, a)


def test_toy_c_values_match_paper():
    g = _golden("toy_lfa_c.json")
    for ppw, c in zip(g["points_per_wavelength"], g["c_printed"]):
        assert abs(lfa.toy_c(2 * math.pi / ppw) - c) < 0.5 * 10 ** -g["printed_digits"]


def test_lemma_closed_form():
    for c, zf, zc, et in [(0.73, 0.7, 0.71, 0.002), (0.9, 0.5, 0.49, 0.01), (0.56, 1.0, 1.0005, 0.003)]:
        R = abs(zf - zc) / et
        th = zc + et * np.tan(np.linspace(-math.pi / 2 + 1e-7, math.pi / 2 - 1e-7, 400001))
        got = np.max(np.abs(lfa.lemma_f(th, c, zf, zc, et)))
        assert abs(got - lfa.lemma_max(c, R)) < 1e-6 * lfa.lemma_max(c, R)


def test_central_difference_symbols():
    w1 = lfa.central_difference_weights(1)
    assert np.allclose(w1, [-1, 2, -1])
    th = 0.3
    s = lfa.toy_symbol(th, 0.0, 0.0, 1.0, 1)[0]
    assert abs(s - 4 * math.sin(th / 2) ** 2) < 1e-14
    # order 4: symbol ~ theta^2 + O(theta^6)
    s2 = lfa.toy_symbol(0.01, 0.0, 0.0, 1.0, 2)[0]
    assert abs(s2 - 0.01 ** 2) < 1e-13


# --------------------------------------------------------------------- FGMRES
def test_fgmres_exact_preconditioner_one_iteration():
    P = _small_problem()
    lu = spla.splu(P.A.tocsc())
    f = synth.random_complex(P.N, 3)
    x, it, rr, _ = krylov.fgmres(lambda v: P.A @ v, lu.solve, f, tol=1e-10)
    assert it == 1 and rr < 1e-10


def test_fgmres_unpreconditioned_matches_direct():
    r = synth.rng(4)
    n = 40
    A = np.eye(n) * 4 + 0.3 * (r.standard_normal((n, n)) + 1j * r.standard_normal((n, n))) / math.sqrt(n)
    b = synth.random_complex(n, 9)
    x, it, rr, _ = krylov.fgmres(lambda v: A @ v, lambda v: v, b, tol=1e-12, restart=10, maxit=200)
    assert rr < 1e-12
    assert np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-10 * np.linalg.norm(x)


def test_small_workload_solve():
    """The method solves the 10-wavelength Q4 problem to 1e-8 in a modest number of cycles."""
    w = synth.workload("square10_q4_n25")
    P = twogrid.Problem(w["n"], w["p"], w["k"], w["eps"], alpha_s=0.2)
    TG = twogrid.TwoGrid(P, l_dd=4)
    x, it, rr, hist = krylov.fgmres(lambda v: P.A @ v, TG.precondition, w["f"], tol=1e-8)
    assert rr <= 1e-8
    xs = spla.spsolve(P.A.tocsc(), w["f"])
    assert np.linalg.norm(x - xs) < 1e-6 * np.linalg.norm(xs)
    t1 = _golden("table1a.json")
    # context: the paper reports 7 at an unstated tolerance; ours reaches 1e-6 in a similar count
    it6 = next(i for i, h in enumerate(hist) if h <= 1e-6)
    assert it6 <= 2 * max(t1["p4_ldd4_ndd1"])
