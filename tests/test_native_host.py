"""CPU checks of the native library: it builds, loads, exports the C ABI, and
its FP64 host set-up agrees with the oracle (no GPU needed)."""
import ctypes
import os
import re

import numpy as np

import synth
import pytest

from oracle import dd, fem, qsfem, twogrid
from tests.common import ensure_built, small_case, oracle_bc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def th():
    ensure_built()
    import paper_2509_17494_gb300 as th
    th.lib()
    return th


def test_exports_every_declared_symbol(th):
    hdrs = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]
    names = set()
    for h in hdrs:
        txt = open(h).read()
        names |= set(re.findall(r"^\s*(?:th_status|void|const char\*)\s+(th_\w+)\s*\(", txt, re.M))
    assert len(names) >= 19
    L = ctypes.CDLL(th.library_path())
    for nm in sorted(names):
        assert hasattr(L, nm), nm


@pytest.mark.parametrize("p", [2, 4, 6, 8])
def test_reference_matrices_match_oracle(th, p):
    nodes, M, K = th.host_reference_1d(p)
    M2, K2 = fem.reference_matrices(p)
    assert np.abs(nodes - fem.gll_points(p)).max() < 1e-14
    assert np.abs(M - M2).max() < 1e-14
    assert np.abs(K - K2).max() < 1e-12 * np.abs(K2).max()


@pytest.mark.parametrize("eta", [0.02, 0.05, 0.1, 0.19, 0.4, 1.0, 2 * np.pi / 5, 2.5])
def test_qsfem_cell_matches_oracle(th, eta):
    hc, eps = 0.02, 7.0
    d = th.host_qsfem_cell(eta / hc, eps, hc)
    q = qsfem.cell_q(eta)
    want = np.array([q[0] - 1j * eps * hc * hc / 9, q[1] - 1j * eps * hc * hc / 18, q[2] - 1j * eps * hc * hc / 36])
    assert np.abs(d - want).max() <= 5e-14 * np.abs(want).max()


@pytest.mark.parametrize("n,l_dd,bc", [(6, 2, "robin"), (7, 3, "neumann"),
                                        (5, 2, {"xlo": "robin", "yhi": "robin"}),
                                        (6, 2, {"xlo": "dirichlet", "ylo": "dirichlet", "xhi": "robin", "yhi": "robin"}),
                                        (5, 3, "dirichlet")])
def test_inverse_rows_match_oracle(th, n, l_dd, bc):
    p = 4
    k, eps = small_case(n=n, p=p)
    P = twogrid.Problem(n, p, k, eps, bc=oracle_bc(bc), alpha_s=0.5)
    S = dd.DDSmoother(P, l_dd)
    for sub, sd in enumerate(S.subs):
        box, W, Lu, Lw = th.host_inverse_rows(n, p, k, eps, sub, bc=bc, alpha_s=0.5, l_dd=l_dd)
        inv = np.linalg.inv(sd.As.toarray())
        rows = inv[sd.u_local, :] / S.L[sd.u_dofs][:, None]
        ox, oy, wx, wy, ux, uy, vx, vy = box[:8]
        assert box[8:] == [0, 1, 0, 1]
        Wr = np.zeros((vx * vy, wx * wy), complex)
        for ry in range(vy):
            for rx in range(vx):
                Wr[ry * vx + rx] = W[ry * Lu + rx].reshape(Lw, Lw)[:wy, :wx].reshape(-1)
        assert np.abs(Wr - rows).max() <= 1e-12 * np.abs(rows).max(), sub
        # padding beyond the boxes is exactly zero
        Wfull = W.reshape(Lu, Lu, Lw, Lw)
        assert np.all(Wfull[vy:] == 0) and np.all(Wfull[:, vx:] == 0)
        assert np.all(Wfull[..., wy:, :] == 0) and np.all(Wfull[..., wx:] == 0)


@pytest.mark.parametrize("n,l_dd", [(4, 2), (5, 2)])
def test_inverse_rows_match_oracle_3d(th, n, l_dd):
    p = 2
    k = 2 * np.pi * 1.5 / synth.random_velocity(n, 3, 9)
    eps = synth.absorbing_layer(n, 3, p, k, width_dofs=2)
    P = twogrid.Problem(n, p, k, eps, dim=3, alpha_s=0.5, coarse=False)
    S = dd.DDSmoother(P, l_dd)
    for sub, sd in enumerate(S.subs):
        box, W, Lu, Lw = th.host_inverse_rows(n, p, k, eps, sub, bc="robin", alpha_s=0.5, l_dd=l_dd, dim=3)
        ox, oy, wx, wy, ux, uy, vx, vy, oz, wz, uz, vz = box
        inv = np.linalg.inv(sd.As.toarray())
        rows = inv[sd.u_local, :] / S.L[sd.u_dofs][:, None]
        Wr = np.zeros((vx * vy * vz, wx * wy * wz), complex)
        for rz in range(vz):
            for ry in range(vy):
                for rx in range(vx):
                    Wr[(rz * vy + ry) * vx + rx] = W[(rz * Lu + ry) * Lu + rx].reshape(Lw, Lw, Lw)[:wz, :wy, :wx].reshape(-1)
        assert np.abs(Wr - rows).max() <= 1e-12 * np.abs(rows).max(), sub


@pytest.mark.parametrize("eta", [0.05, 0.1, 0.3, 1.0, 1.57, 2.2])
def test_qsfem27_cell_matches_oracle(th, eta):
    """The library's weights against the oracle's 50-digit solve of the zero
    conditions.  The weight of the corner pairs is fixed by the O(eta^6)
    differences between the fitted directions, so the library (a long double
    solve: 64-bit significand on x86) loses about eta^-4 of its unit roundoff:
    1e-13 from eta = 0.1 on, 2e-12 at eta = 0.05."""
    from oracle import qsfem
    hc, eps = 0.025, 3.0
    d = th.host_qsfem27_cell(eta / hc, eps, hc)
    q = np.array(qsfem.cell_q27(eta))
    mass = np.array([1 / 27, 1 / 54, 1 / 108, 1 / 216]) * hc ** 3
    want = hc * q - 1j * eps * mass
    tol = 1e-13 if eta >= 0.1 else 2e-12
    assert np.abs(d - want).max() <= tol * np.abs(want).max(), (d, want)


def test_workspace_size_and_argument_errors(th):
    a = th.workspace_size(25, 4, l_dd=2)
    b = th.workspace_size(25, 4, l_dd=2, nrhs_max=4)
    c = th.workspace_size(25, 4, l_dd=2, prec="bf16", extra_prec=("fp64",))
    assert 0 < a < b and a < c
    # Dirichlet sides are built in 2-D only
    assert th.workspace_size(10, 4, bc="dirichlet") > 0
    for kw, code in [(dict(n=25, p=3), 1), (dict(n=0, p=4), 1), (dict(n=4, p=2, bc="dirichlet", dim=3), 8)]:
        with pytest.raises(th.ThError) as e:
            th.workspace_size(**kw)
        assert e.value.code == code
    with pytest.raises(th.ThError):
        th.workspace_size(10, 4, l_dd=0)
    with pytest.raises(th.ThError):
        th.workspace_size(10, 4, restart=0)
    # the coarse partition's chunk count: 2 P - 1 <= m_c (m_c = 21 here)
    assert th.workspace_size(10, 4, coarse_chunks=11) > 0
    for bad in (12, -1):
        with pytest.raises(th.ThError) as e:
            th.workspace_size(10, 4, coarse_chunks=bad)
        assert e.value.code == 1


def _stencil_matrix(sten, mc, q):
    import scipy.sparse as sp
    S = 2 * q + 1
    rows, cols, vals = [], [], []
    for node in range(mc * mc):
        y, x = divmod(node, mc)
        for a in range(S):
            for b in range(S):
                v = sten[node, a, b]
                if v == 0:
                    continue
                yy, xx = y + a - q, x + b - q
                assert 0 <= yy < mc and 0 <= xx < mc
                rows.append(node)
                cols.append(yy * mc + xx)
                vals.append(v)
    return sp.csr_matrix((vals, (rows, cols)), shape=(mc * mc, mc * mc))


@pytest.mark.parametrize("n,p,bc,alpha_c", [(5, 4, "robin", 0.0), (4, 6, {"xlo": "robin", "yhi": "robin"}, 0.05),
                                            (3, 8, "neumann", 0.2), (6, 2, "robin", 0.02)])
def test_galerkin_setup_matches_oracle(th, n, p, bc, alpha_c):
    """Galerkin p-coarsening: the set-up's stencil equals I_P^T A_{alpha_c} I_P of
    the oracle, and its block sweep solves A_c x = b."""
    k, eps = small_case(n=n, p=p)
    P = twogrid.Problem(n, p, k, eps, bc=oracle_bc(bc), coarse_kind="gal", alpha_c=alpha_c)
    q = p // 2
    mc = n * q + 1
    b = synth.random_complex(mc * mc, 8)
    sten, x = th.host_galerkin(n, p, k.reshape(-1), eps.reshape(-1), bc=bc, alpha_c=alpha_c, b=b)
    A = _stencil_matrix(sten, mc, q)
    assert abs(A - P.Aq).max() <= 1e-12 * abs(P.Aq).max()
    import scipy.sparse.linalg as spla
    want = spla.spsolve(P.Aq.tocsc(), b)
    assert np.abs(x - want).max() <= 1e-9 * np.abs(want).max()


@pytest.mark.parametrize("n,P,bc", [(25, 3, "robin"), (13, 4, "robin"),
                                    (13, 3, {"xlo": "dirichlet", "ylo": "dirichlet", "xhi": "robin", "yhi": "robin"})])
def test_reduced_separator_inverse_is_block_of_coarse_inverse(th, n, P, bc):
    """The explicit inverse of the reduced separator system (the Schur complement
    of A_q on the separator rows) equals the separator block of A_q^{-1}, here
    the oracle's A_q inverted densely.  mc = 51 and 27 coarse rows: not multiples
    of the 16-column tasks the set-up computes the inverse in, with K = 2 and 3
    separator blocks."""
    p = 4
    k, eps = small_case(n=n, p=p, W=n / 5.0)
    sep, Sinv = th.host_coarse_separators(n, p, k, eps, bc=bc, P=P)
    mc = n * p // 2 + 1
    assert len(sep) == P - 1 and np.all(np.diff(sep) > 1) and sep[0] > 0 and sep[-1] < mc - 1
    Aq = twogrid.Problem(n, p, k, eps, bc=oracle_bc(bc), alpha_s=0.5).Aq.toarray()
    Ainv = np.linalg.inv(Aq)
    idx = np.concatenate([np.arange(s * mc, (s + 1) * mc) for s in sep])
    want = Ainv[np.ix_(idx, idx)]
    assert np.abs(Sinv - want).max() < 1e-10 * np.abs(want).max()
