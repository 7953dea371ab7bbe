"""Right-preconditioned flexible GMRES (oracle).

The outer solver of the paper is GMRES (Saad and Schultz) preconditioned by one multigrid
V-cycle per iteration (Sec. 3), stopped when ||r_k|| / ||r_0|| < tol on the full residual
[r_u; r_lambda] (Eq. ch7_linearstoppingcriterion, Sec. 6.1).  The flexible variant keeps
the preconditioned directions Z_j = M^{-1} v_j, so the V-cycle may change between
iterations (needed once the cycle runs in lower precision).  Arnoldi uses modified
Gram-Schmidt, the least-squares problem is solved with Givens rotations; x_0 = 0.
"""
from __future__ import annotations

import numpy as np


def fgmres(A, b: np.ndarray, precond, tol: float = 1e-8, restart: int = 50, maxit: int = 1000):
    """Solve A x = b.  Returns (x, iterations, relative residual history list)."""
    n = b.size
    x = np.zeros(n)
    r0 = np.linalg.norm(b)
    hist = [1.0]
    if r0 == 0.0:
        return x, 0, hist
    it = 0
    r = b.copy()
    while it < maxit:
        beta = np.linalg.norm(r)
        m = restart
        V = np.zeros((m + 1, n))
        Zs = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        converged = False
        for j in range(m):
            Zs[j] = precond(V[j])
            w = A @ Zs[j]
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / r0)
            if abs(g[j + 1]) / r0 < tol or it >= maxit:
                converged = abs(g[j + 1]) / r0 < tol
                break
        y = np.zeros(j_done)
        for i in range(j_done - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:j_done] @ y[i + 1:j_done]) / H[i, i]
        x = x + Zs[:j_done].T @ y
        r = b - A @ x
        if converged:
            break
    return x, it, hist
