"""Oracle: flexible GMRES (plain FP64, CPU).

TEST INFRASTRUCTURE ONLY (see oracle/fem.py).

The paper uses the two-grid step as a preconditioner (Section 4) without
naming the Krylov method; the outer solver here is right-preconditioned
flexible GMRES(m) (Saad 1993): Arnoldi with modified Gram-Schmidt on
A z_j, z_j = B(v_j), Givens rotations on the Hessenberg matrix, x = x0 + Z y.
Stops when the Givens residual estimate falls below tol * ||b||; the true
relative residual ||b - A x|| / ||b|| is recomputed at the end.
"""
from __future__ import annotations

import numpy as np


def fgmres(apply_A, precond, b, x0=None, tol=1e-8, restart=60, maxit=500):
    """Returns (x, iterations, relres, history)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0, [0.0]
    hist = []
    it = 0
    while True:
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta <= tol * bnorm or it >= maxit:
            break
        m = restart
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m, dtype=np.complex128)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        j_done = 0
        for j in range(m):
            z = precond(V[j])
            Z.append(z)
            w = apply_A(z)
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            V.append(w / H[j + 1, j] if H[j + 1, j] != 0 else w)
            # unitary rotations G_i = [[conj(c_i), conj(s_i)], [-s_i, c_i]]
            for i in range(j):
                t = np.conj(cs[i]) * H[i, j] + np.conj(sn[i]) * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a, c = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(c) ** 2)
            cs[j] = a / den if den != 0 else 1.0
            sn[j] = c / den if den != 0 else 0.0
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            it += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= tol * bnorm or it >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        for i in range(j_done):
            x = x + y[i] * Z[i]
        if abs(g[j_done]) <= tol * bnorm or it >= maxit:
            break
    relres = np.linalg.norm(b - apply_A(x)) / bnorm
    return x, it, relres, hist
