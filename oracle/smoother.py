"""CheapSIMPLE block smoother (oracle).

SIMPLE (Algorithm 4, Eq. ch6_ASIMPLE) in its "cheap" form (Sec. 5.2): the predictor solve
with K is replaced by damped Jacobi sweeps, and the corrector solve with the approximate
Schur complement uses the inverse of its nodal 3x3 block diagonal.  One sweep, given the
current (u, lambda) and the right-hand side (f, g) of [K B1; B2 -Z]:

  1. predictor:  u_half = u + omega_J D_K^{-1} (f - K u - B1 lambda), repeated nu_J times
  2. corrector:  -S_hat dlam = g - B2 u_half + Z lambda
  3. update:     lambda += alpha dlam,   u = u_half - alpha A_tilde^{-1} B1 dlam

with A_tilde = diag(K) (SIMPLE) or the absolute row sums of K (SIMPLEC, Eq. ch6_simplecapprox),
S_hat = Z + B2 A_tilde^{-1} B1 (the paper's default Schur approximation with the alpha
factor taken out, so that alpha acts as a damping of the correction), and the corrector
inverse taken on the nodal 3x3 diagonal blocks of S_hat.  With the exact S_hat inverse and
alpha = 1 the constraint row is satisfied exactly after the sweep (Eq. ch6_errormatsimple_special).

The step lambda += alpha dlam is damped Jacobi on S_hat preconditioned by its block diagonal
S_bd; it contracts only while alpha * rho(S_bd^{-1} S_hat) < 2.  Where a slave mesh is much finer
than its master, each master node couples many slave nodes and rho grows far beyond 2, so the
optional Schur damping replaces alpha by min(alpha, (4/3) / rho) with rho estimated by
``schur_rho`` (the same (4/3)/lambda_max rule the Jacobi predictor uses).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def atilde_diag(K: sp.csr_matrix, simplec: bool) -> np.ndarray:
    if simplec:
        return np.asarray(abs(K).sum(axis=1)).ravel()
    return K.diagonal().copy()


def schur_blocks(B1: sp.csr_matrix, B2: sp.csr_matrix, Z: np.ndarray, at_inv: np.ndarray) -> np.ndarray:
    """Nodal 3x3 diagonal blocks of S_hat = Z + B2 A_tilde^{-1} B1."""
    S = (B2 @ sp.diags(at_inv) @ B1).tocsr()
    nl = Z.shape[0]
    out = Z.copy()
    for l in range(nl):
        out[l] += S[3 * l:3 * l + 3, 3 * l:3 * l + 3].toarray()
    return out


def cheap_simple_sweep(K, B1, B2, Z_full, u, lam, f, g, dinv, omega_j, nu_j, at_inv, S_inv_apply, alpha):
    """One CheapSIMPLE sweep; S_inv_apply(r) returns S_hat^{-1} r."""
    for _ in range(nu_j):
        r_u = f - K @ u - B1 @ lam
        u = u + omega_j * dinv * r_u
    r_l = g - B2 @ u + Z_full @ lam
    dlam = -S_inv_apply(r_l)
    lam = lam + alpha * dlam
    u = u - alpha * at_inv * (B1 @ dlam)
    return u, lam


def schur_rho(B1: sp.csr_matrix, B2: sp.csr_matrix, Z: np.ndarray, at_inv: np.ndarray, S_inv: np.ndarray,
              steps: int = 30) -> float:
    """Power-iteration estimate of the spectral radius of S_bd^{-1} S_hat, S_hat = Z + B2 A~^{-1} B1.

    Start from the normalised ones vector; each step forms y = S_bd^{-1} S_hat x, takes
    rho = ||y|| and continues from y / rho.  Returns the last rho."""
    nl = Z.shape[0]
    x = np.full(3 * nl, 1.0 / np.sqrt(3 * nl))
    rho = 0.0
    for _ in range(steps):
        r = np.einsum("lij,lj->li", Z, x.reshape(-1, 3)).ravel() + B2 @ (at_inv * (B1 @ x))
        y = np.einsum("lij,lj->li", S_inv, r.reshape(-1, 3)).ravel()
        rho = float(np.linalg.norm(y))
        x = y / rho
    return rho
