"""Oracle: fine-level finite-element discretisation (plain FP64, CPU).

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; only
the tests, `__graft_entry__.smoke()` and the benchmark's CPU-baseline arm use it.

What is computed (Section 2, Eq. bilin_form; Section 3.1):
    a(u, v) = int grad u . grad v - int (k^2 + i eps) u v - int_{Gamma_abs} i k u v
discretised with continuous Q_p elements on a uniform mesh of n^d cells of
side h = 1/n.  The basis is the nodal Lagrange basis on the Gauss-Lobatto-
Legendre (GLL) points of each cell (the paper's hierarchical basis spans the
same space).  k and eps are constant per cell.  Element matrices are
integrated exactly.  Dofs are numbered lexicographically on the global
(n p + 1)^d node grid, last array axis (x) fastest.  Cell arrays are indexed
[cy, cx] (2-D) or [cz, cy, cx] (3-D).

A boundary side is (axis, end) with `axis` the array axis (0 = slowest) and
end 0 (low) or 1 (high).  Robin sides carry -i k (unshifted) times the face
mass; all other sides are natural (Neumann).  `periodic=True` wraps the node
grid instead (used only by the Fourier-analysis cross-checks).
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.sparse as sp

# ----------------------------------------------------------------------------
# 1-D reference element on [0, 1]
# ----------------------------------------------------------------------------


def gll_points(p: int) -> np.ndarray:
    """GLL points on [0,1]: the end points and the roots of P_p' (Legendre)."""
    if p == 1:
        return np.array([0.0, 1.0])
    c = np.zeros(p + 1)
    c[p] = 1.0
    r = np.polynomial.legendre.legroots(np.polynomial.legendre.legder(c))
    x = np.concatenate([[-1.0], np.sort(np.real(r)), [1.0]])
    return 0.5 * (x + 1.0)


def gauss_legendre(nq: int):
    """nq-point Gauss-Legendre rule on [0,1] (exact for degree 2 nq - 1)."""
    x, w = np.polynomial.legendre.leggauss(nq)
    return 0.5 * (x + 1.0), 0.5 * w


def lagrange_values(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """V[q, a] = l_a(x_q), product formula."""
    x = np.atleast_1d(np.asarray(x, dtype=float))
    V = np.ones((x.size, nodes.size))
    for a in range(nodes.size):
        for b in range(nodes.size):
            if b != a:
                V[:, a] *= (x - nodes[b]) / (nodes[a] - nodes[b])
    return V


def lagrange_derivatives(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """D[q, a] = l_a'(x_q) = sum_{m != a} 1/(x_a - x_m) prod_{b != a, m} (x - x_b)/(x_a - x_b)."""
    x = np.atleast_1d(np.asarray(x, dtype=float))
    n = nodes.size
    D = np.zeros((x.size, n))
    for a in range(n):
        for m in range(n):
            if m == a:
                continue
            t = np.full(x.size, 1.0 / (nodes[a] - nodes[m]))
            for b in range(n):
                if b != a and b != m:
                    t *= (x - nodes[b]) / (nodes[a] - nodes[b])
            D[:, a] += t
    return D


def reference_matrices(p: int):
    """Exact 1-D mass M[a,b] = int l_a l_b and stiffness K[a,b] = int l_a' l_b' on [0,1]."""
    nodes = gll_points(p)
    xq, wq = gauss_legendre(p + 1)
    V = lagrange_values(nodes, xq)
    D = lagrange_derivatives(nodes, xq)
    M = V.T @ (wq[:, None] * V)
    K = D.T @ (wq[:, None] * D)
    return M, K


# ----------------------------------------------------------------------------
# Assembly
# ----------------------------------------------------------------------------


def _kron_all(mats):
    out = np.ones((1, 1))
    for m in mats:
        out = np.kron(out, m)
    return out


def element_matrices(p: int, h: float, dim: int):
    """(stiffness, mass) element matrices of a cell of side h, local lexicographic order."""
    M, K = reference_matrices(p)
    stiff = np.zeros(((p + 1) ** dim,) * 2)
    for ax in range(dim):
        stiff += _kron_all([K / h if b == ax else h * M for b in range(dim)])
    mass = _kron_all([h * M] * dim)
    return stiff, mass


def face_mass(p: int, h: float, dim: int, axis: int, end: int):
    """int_face l_alpha l_beta ds on the face {x_axis = end} of a cell of side h."""
    M, _ = reference_matrices(p)
    E = np.zeros((p + 1, p + 1))
    E[end * p, end * p] = 1.0
    return _kron_all([E if b == axis else h * M for b in range(dim)])


def grid_size(ncells, p, periodic=False):
    return [nc * p + (0 if periodic else 1) for nc in ncells]


def cell_dof_indices(ncells, p, periodic=False) -> np.ndarray:
    """gidx[cell, local] global dof index, cells and locals in C order."""
    dim = len(ncells)
    m = grid_size(ncells, p, periodic)
    strides = [int(np.prod(m[ax + 1:])) for ax in range(dim)]
    total = np.zeros([*ncells, *([p + 1] * dim)], dtype=np.int64)
    for ax in range(dim):
        g = np.arange(ncells[ax])[:, None] * p + np.arange(p + 1)[None, :]
        if periodic:
            g = g % m[ax]
        shape = [1] * (2 * dim)
        shape[ax] = ncells[ax]
        shape[dim + ax] = p + 1
        total = total + g.reshape(shape) * strides[ax]
    return total.reshape(int(np.prod(ncells)), (p + 1) ** dim)


def assemble(ncells, p: int, h: float, cvol: np.ndarray, kcell: np.ndarray,
             robin_sides=(), periodic: bool = False) -> sp.csr_matrix:
    """Global matrix of a(u,v) with volume coefficient `cvol` (k^2 + i eps, or shifted).

    sum over cells e of  [stiffness_e - cvol_e * mass_e]
      + sum over Robin faces f of  [-i k_e * facemass_f]          (Eq. bilin_form)
    """
    ncells = tuple(int(c) for c in ncells)
    dim = len(ncells)
    stiff, mass = element_matrices(p, h, dim)
    gidx = cell_dof_indices(ncells, p, periodic)
    cv = np.asarray(cvol, dtype=np.complex128).reshape(-1)
    data = stiff[None, :, :] - cv[:, None, None] * mass[None, :, :]
    L = gidx.shape[1]
    rows = np.broadcast_to(gidx[:, :, None], (gidx.shape[0], L, L))
    cols = np.broadcast_to(gidx[:, None, :], (gidx.shape[0], L, L))
    rows_l, cols_l, data_l = [rows.reshape(-1)], [cols.reshape(-1)], [data.reshape(-1)]
    kc = np.asarray(kcell, dtype=float).reshape(ncells)
    cell_ids = np.arange(int(np.prod(ncells))).reshape(ncells)
    for (axis, end) in robin_sides:
        fm = face_mass(p, h, dim, axis, end)
        sl = [slice(None)] * dim
        sl[axis] = 0 if end == 0 else ncells[axis] - 1
        cells = cell_ids[tuple(sl)].reshape(-1)
        kk = kc[tuple(sl)].reshape(-1)
        g = gidx[cells]
        d = (-1j * kk)[:, None, None] * fm[None, :, :]
        rows_l.append(np.broadcast_to(g[:, :, None], d.shape).reshape(-1))
        cols_l.append(np.broadcast_to(g[:, None, :], d.shape).reshape(-1))
        data_l.append(d.reshape(-1))
    N = int(np.prod(grid_size(ncells, p, periodic)))
    A = sp.coo_matrix((np.concatenate(data_l), (np.concatenate(rows_l), np.concatenate(cols_l))),
                      shape=(N, N)).tocsr()
    A.sum_duplicates()
    return A


def all_sides(dim):
    return [(ax, e) for ax in range(dim) for e in (0, 1)]


def robin_set(dim, bc):
    """bc: 'robin' | 'neumann' | 'dirichlet' | dict {(axis, end): 'robin'|'neumann'|'dirichlet'}."""
    if isinstance(bc, str):
        return [s for s in all_sides(dim)] if bc == "robin" else []
    return [s for s in all_sides(dim) if bc.get(s, "neumann") == "robin"]


def dirichlet_set(dim, bc):
    """The sides of Gamma_0 (Section 2: u = 0 there)."""
    if isinstance(bc, str):
        return [s for s in all_sides(dim)] if bc == "dirichlet" else []
    return [s for s in all_sides(dim) if bc.get(s, "neumann") == "dirichlet"]


def boundary_mask(m: int, dim: int, sides) -> np.ndarray:
    """Boolean mask over the m^dim node grid (lexicographic, last axis fastest) of
    the nodes on the given sides."""
    mask = np.zeros((m,) * dim, dtype=bool)
    for (axis, end) in sides:
        sl = [slice(None)] * dim
        sl[axis] = 0 if end == 0 else m - 1
        mask[tuple(sl)] = True
    return mask.reshape(-1)


def impose_dirichlet(A: sp.spmatrix, mask: np.ndarray) -> sp.csr_matrix:
    """The matrix of the space H^1_0(Omega; Gamma_0) (Section 2) kept on the full
    node grid: rows and columns of the Dirichlet nodes removed and replaced by
    the identity, so those unknowns are decoupled and equal their right-hand side."""
    if not mask.any():
        return A.tocsr()
    keep = sp.diags((~mask).astype(float))
    return (keep @ A @ keep + sp.diags(mask.astype(float))).tocsr()


def shifted_coefficient(k, eps, alpha_s):
    """k^2 + i alpha_s k^2 + i eps (Section 4.1, the complex-shifted operator A_s)."""
    return k * k + 1j * alpha_s * k * k + 1j * eps


def helmholtz_coefficient(k, eps):
    return k * k + 1j * eps


# ----------------------------------------------------------------------------
# Prolongation (Section 4.2): piecewise degree p/2 interpolation of the coarse
# vertex values, the coarse mesh having spacing 2h/p.
# ----------------------------------------------------------------------------


def prolongation_1d(n: int, p: int, periodic: bool = False) -> np.ndarray:
    """P[i_fine, J_coarse] = l^{eq, p/2}_b(xi_a) inside each cell (dense, small)."""
    assert p % 2 == 0
    q = p // 2
    nodes = gll_points(p)
    eq = np.linspace(0.0, 1.0, q + 1)
    V = lagrange_values(eq, nodes)          # V[a, b] = l^eq_b(xi_a)
    mf = n * p + (0 if periodic else 1)
    mc = n * q + (0 if periodic else 1)
    P = np.zeros((mf, mc))
    for e in range(n):
        for a in range(p + 1):
            i = (e * p + a) % mf
            for b in range(q + 1):
                J = (e * q + b) % mc
                P[i, J] = V[a, b]          # shared end points get identical values
    return P


def prolongation(n: int, p: int, dim: int, periodic: bool = False) -> sp.csr_matrix:
    P1 = sp.csr_matrix(prolongation_1d(n, p, periodic))
    P1.eliminate_zeros()
    out = P1
    for _ in range(dim - 1):
        out = sp.kron(out, P1, format="csr")
    return out


def interpolate_nodal(n: int, p: int, func, dim: int = 2) -> np.ndarray:
    """Nodal values of `func(x, y[, z])` at the global GLL node grid (lexicographic)."""
    nodes = gll_points(p)
    h = 1.0 / n
    x1 = np.concatenate([e * h + h * nodes[:-1] for e in range(n)] + [np.array([1.0])])
    grids = np.meshgrid(*([x1] * dim), indexing="ij")
    # grids[0] is the slowest axis; func takes (x, y[, z]) with x fastest.
    return np.asarray(func(*reversed(grids)), dtype=np.complex128).reshape(-1)


def node_coordinates_1d(n: int, p: int) -> np.ndarray:
    nodes = gll_points(p)
    h = 1.0 / n
    return np.concatenate([e * h + h * nodes[:-1] for e in range(n)] + [np.array([1.0])])


def l2_error_2d(n: int, p: int, uh: np.ndarray, exact, nq: int | None = None) -> float:
    """|| u_h - exact ||_{L2(unit square)} by Gauss quadrature on every cell."""
    nq = nq or p + 3
    nodes = gll_points(p)
    xq, wq = gauss_legendre(nq)
    V = lagrange_values(nodes, xq)            # V[q, a]
    h = 1.0 / n
    m = n * p + 1
    U = uh.reshape(m, m)
    err2 = 0.0
    for cy in range(n):
        for cx in range(n):
            loc = U[cy * p:cy * p + p + 1, cx * p:cx * p + p + 1]      # [ay, ax]
            vals = V @ loc @ V.T                                      # [qy, qx]
            X = cx * h + h * xq
            Y = cy * h + h * xq
            ex = exact(X[None, :], Y[:, None])
            err2 += np.sum((wq[:, None] * wq[None, :]) * np.abs(vals - ex) ** 2) * h * h
    return math.sqrt(err2)


def cells_iter(ncells):
    return itertools.product(*[range(c) for c in ncells])
