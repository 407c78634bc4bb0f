"""Flexible GMRES in FP64 (oracle, test infrastructure).

The paper solves Eq. (dbem4) with flexible GMRES (Sec. 3.1 and Sec. 4): a
right-preconditioned GMRES in which the preconditioner may change from one
iteration to the next (Saad 1993), so the preconditioned directions
z_j = P_j(v_j) are stored next to the Arnoldi basis v_j and the update is
x = x0 + Z y.  Restarted, modified Gram-Schmidt with one re-orthogonalisation,
Givens rotations for the small least-squares problem.  Convergence is judged
on the true residual ||b - A x|| / ||b|| at every restart and at the end.
"""
from __future__ import annotations

import numpy as np


def fgmres(apply_A, b, tol=1e-8, restart=40, maxit=2000, precond=None, x0=None):
    """Solve A x = b.  apply_A, precond: callables on complex vectors.

    Returns (x, info) with info = dict(iters, relres (true), history).
    """
    b = np.asarray(b, dtype=np.complex128)
    n = b.size
    x = np.zeros(n, np.complex128) if x0 is None else np.array(x0, np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros(n, np.complex128), dict(iters=0, relres=0.0, history=[0.0])
    P = (lambda v: v) if precond is None else precond
    hist = []
    it = 0
    r = b - apply_A(x)
    rel = np.linalg.norm(r) / bnorm
    hist.append(rel)
    while rel > tol and it < maxit:
        m = restart
        V = np.zeros((m + 1, n), np.complex128)
        Z = np.zeros((m, n), np.complex128)
        H = np.zeros((m + 1, m), np.complex128)
        cs = np.zeros(m, np.complex128)
        sn = np.zeros(m, np.complex128)
        g = np.zeros(m + 1, np.complex128)
        beta = np.linalg.norm(r)
        V[0] = r / beta
        g[0] = beta
        j_done = 0
        for j in range(m):
            Z[j] = P(V[j])
            w = apply_A(Z[j])
            for _ in range(2):                      # MGS + one re-orthogonalisation
                for i in range(j + 1):
                    h = np.vdot(V[i], w)
                    H[i, j] += h
                    w = w - h * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                      # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + np.conj(cs[i]) * H[i + 1, j]
                H[i, j] = t
            a, bb = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            if den == 0:
                cs[j], sn[j] = 1.0, 0.0
            elif abs(a) == 0:
                cs[j], sn[j] = 0.0, 1.0
            else:
                cs[j] = abs(a) / den
                sn[j] = (a / abs(a)) * np.conj(bb) / den
            H[j, j] = cs[j] * a + sn[j] * bb
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) / bnorm <= tol or it >= maxit:
                break
        y = np.zeros(j_done, np.complex128)
        for i in range(j_done - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:j_done] @ y[i + 1:j_done]) / H[i, i]
        x = x + Z[:j_done].T @ y
        r = b - apply_A(x)
        rel = np.linalg.norm(r) / bnorm
    return x, dict(iters=it, relres=float(rel), history=hist)
