"""Block smoothers of Sec. 5.1 besides CheapSIMPLE, and the inner solvers of their cheap variants
(Sec. 5.2).  Oracle: plain FP64 CPU code, test infrastructure only (imported by the tests, never
by the product path).

Each smoother is the iteration x <- x + M^{-1} (b - A x) of Eq. ch6_commonblocksmoothing, with a
block preconditioning matrix M approximating A = [K B1; B2 -Z] and right-hand side (f, g), and is
carried out in the predictor-corrector form the paper gives:

* Uzawa (Eq. ch6_Uzawa, Algorithm 2), M = (1/omega) [K 0; B2 -S_hat]:
    predictor   K du = f - K u - B1 lam
    corrector   -S_hat dlam = g - B2 u + Z lam - B2 du
    update      u += omega du,   lam += omega dlam
* Braess-Sarazin (Eq. ch6_ABraessSarazin, Algorithm 3), M = [omega A~ B1; B2 -Z]:
    predictor   u_h = u + (1/omega) A~^{-1} (f - K u - B1 lam)
    corrector   -(Z + (1/omega) B2 A~^{-1} B1) dlam = g + Z lam - B2 u_h
    update      lam += dlam,   u = u_h - (1/omega) A~^{-1} B1 dlam
* SIMPLE (Eq. ch6_ASIMPLE, Algorithm 4), M = [K 0; B2 -S_hat] [I A~^{-1} B1; 0 (1/omega) I]:
    predictor   K u_h = f - B1 lam
    corrector   -S_hat dlam = g + Z lam - B2 u_h
    update      lam += omega dlam,   u = u_h - omega A~^{-1} B1 dlam

The exact variants solve the predictor and corrector systems.  The cheap variants (Sec. 5.2)
replace the K solve by damped symmetric Gauss-Seidel sweeps and the Schur solve by an
incomplete LU factorisation without fill (ILU(0)) of the assembled Schur approximation, the
inner solvers of the paper's experiments (Sec. 6.1).  The ILU(0) works on the nodal 3 x 3 blocks
of the multipliers: with Cartesian multipliers a tangential row of an active node (-Z = T) can
have a zero diagonal entry, while its nodal block (normal and tangents) is invertible.  A~ is diag(K), or for SIMPLEC the absolute
row sums of K (Eq. ch6_simplecapprox); S_hat = Z + B2 A~^{-1} B1 unless a caller passes another
Schur solve.
"""
from __future__ import annotations

from typing import Callable, Tuple

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import spsolve_triangular

Solve = Callable[[np.ndarray], np.ndarray]


# ------------------------------------------------------------------ inner solvers (Sec. 5.2)
def sgs(K: sp.spmatrix, b: np.ndarray, x: np.ndarray, sweeps: int = 1, omega: float = 1.0) -> np.ndarray:
    """Damped symmetric Gauss-Seidel from x: each sweep is one forward and one backward
    Gauss-Seidel pass with relaxation omega.  With K = D + L + U (diagonal, strictly lower and
    strictly upper parts) the forward pass solves (D/omega + L) x' = b - (U + (1 - 1/omega) D) x
    and the backward pass (D/omega + U) x'' = b - (L + (1 - 1/omega) D) x'."""
    K = sp.csr_matrix(K)
    d = K.diagonal()
    lo = sp.tril(K, k=-1, format="csr")
    up = sp.triu(K, k=1, format="csr")
    fwd = (sp.diags(d / omega) + lo).tocsr()
    bwd = (sp.diags(d / omega) + up).tocsr()
    rest = sp.diags((1.0 - 1.0 / omega) * d)
    x = np.array(x, dtype=np.float64, copy=True)
    for _ in range(sweeps):
        x = spsolve_triangular(fwd, b - (up + rest) @ x, lower=True)
        x = spsolve_triangular(bwd, b - (lo + rest) @ x, lower=False)
    return x


def jp_coloring(G: sp.spmatrix, seed: int = 0x5EED) -> np.ndarray:
    """Colour of every node of the symmetric graph G (diagonal ignored) by Jones-Plassmann rounds:
    an uncoloured node whose priority (the MIS-2 key, fmix32(i ^ seed) * 2^32 + i) exceeds that
    of every uncoloured neighbour takes the smallest colour none of its coloured neighbours has.
    The rounds are data parallel, so a GPU can reproduce the colouring exactly."""
    from .aggregate import priorities
    G = sp.csr_matrix(G)
    n = G.shape[0]
    key = priorities(n, seed)
    color = -np.ones(n, dtype=np.int64)
    nbrs = [G.indices[G.indptr[i]:G.indptr[i + 1]] for i in range(n)]
    nbrs = [nb[nb != i] for i, nb in enumerate(nbrs)]
    while (color < 0).any():
        pick = [i for i in np.nonzero(color < 0)[0]
                if all(color[j] >= 0 or key[j] < key[i] for j in nbrs[i])]
        new = {}
        for i in pick:
            used = {int(color[j]) for j in nbrs[i] if color[j] >= 0}
            c = 0
            while c in used:
                c += 1
            new[i] = c
        for i, c in new.items():
            color[i] = c
    return color


def colored_block_sgs(K: sp.spmatrix, color: np.ndarray, bs: int = 3):
    """Damped symmetric block Gauss-Seidel over nodal bs x bs blocks in colour order, prepared for
    K and a colouring of its nodes: returns apply(b, x, sweeps, omega).  Each sweep visits the
    colours ascending, then descending; within a colour every node i (no two adjacent) takes
    x_i <- x_i + omega K_ii^{-1} (b_i - sum_j K_ij x_j) from the current x (the nodes of one colour
    are updated together, as they do not couple)."""
    K = sp.csr_matrix(K)
    rows = _blocks(K, bs)
    ncol = int(color.max()) + 1 if color.size else 0
    parts = []
    for c in range(ncol):
        nodes = np.nonzero(color == c)[0]
        idx = (nodes[:, None] * bs + np.arange(bs)[None, :]).ravel()
        inv = np.array([np.linalg.inv(rows[i][i]) for i in nodes]).reshape(-1, bs, bs)
        ri = np.repeat(np.arange(nodes.size * bs), bs)
        ci = (np.arange(nodes.size)[:, None, None] * bs + np.zeros((1, bs, 1), dtype=np.int64)
              + np.arange(bs)[None, None, :]).ravel()
        dinv = sp.csr_matrix((inv.ravel(), (ri, ci)), shape=(nodes.size * bs, nodes.size * bs))
        parts.append((idx, K[idx, :].tocsr(), dinv))
    order = list(range(ncol)) + list(range(ncol - 1, -1, -1))

    def apply(b: np.ndarray, x: np.ndarray, sweeps: int = 1, omega: float = 1.0) -> np.ndarray:
        x = np.array(x, dtype=np.float64, copy=True)
        b = np.asarray(b, dtype=np.float64)
        for _ in range(sweeps):
            for c in order:
                idx, Kc, dinv = parts[c]
                x[idx] = x[idx] + omega * (dinv @ (b[idx] - Kc @ x))
        return x
    return apply


def block_sgs_colored(K: sp.spmatrix, b: np.ndarray, x: np.ndarray, color: np.ndarray, bs: int = 3,
                      sweeps: int = 1, omega: float = 1.0) -> np.ndarray:
    """One-off form of colored_block_sgs."""
    return colored_block_sgs(K, color, bs)(b, x, sweeps, omega)


def _blocks(S: sp.csr_matrix, bs: int):
    """Rows of S as {block column: bs x bs array} per block row (the block pattern of S)."""
    nb = S.shape[0] // bs
    C = S.tocoo()
    rows = [dict() for _ in range(nb)]
    for i, j, v in zip(C.row, C.col, C.data):
        blk = rows[i // bs].setdefault(j // bs, np.zeros((bs, bs)))
        blk[i % bs, j % bs] += v
    return rows


def ilu0(S: sp.spmatrix, bs: int = 1):
    """Incomplete LU factorisation without fill on the block pattern of S (bs x bs blocks; bs = 1
    is the pointwise ILU(0)): row-wise block Gaussian elimination, A_ik <- A_ik A_kk^{-1} and
    A_ij <- A_ij - A_ik A_kj for the blocks (i, j) of the pattern only.  Returns the rows of the
    factors as {block column: block}: L strictly below the diagonal (its diagonal blocks are the
    identity), U on and above it."""
    S = sp.csr_matrix(S, dtype=np.float64)
    if S.shape[0] % bs:
        raise ValueError("ILU(0): size not a multiple of the block size")
    rows = _blocks(S, bs)
    for i, ri in enumerate(rows):
        for k in sorted(c for c in ri if c < i):
            piv = rows[k].get(k)
            if piv is None or not np.all(np.isfinite(piv)) or abs(np.linalg.det(piv)) == 0.0:
                raise np.linalg.LinAlgError(f"ILU(0): singular pivot block {k}")
            ri[k] = ri[k] @ np.linalg.inv(piv)
            a = ri[k]
            for j, v in rows[k].items():
                if j > k and j in ri:
                    ri[j] = ri[j] - a @ v
        d = ri.get(i)
        if d is None or abs(np.linalg.det(d)) == 0.0:
            raise np.linalg.LinAlgError(f"ILU(0): singular pivot block {i}")
    L = [{j: v for j, v in ri.items() if j < i} for i, ri in enumerate(rows)]
    U = [{j: v for j, v in ri.items() if j >= i} for i, ri in enumerate(rows)]
    return L, U


def ilu0_matrices(S: sp.spmatrix, bs: int = 1) -> Tuple[sp.csr_matrix, sp.csr_matrix]:
    """The ILU(0) factors as sparse matrices: L with unit diagonal blocks, U."""
    L, U = ilu0(S, bs)
    n = S.shape[0]

    def assemble(rows, unit):
        I, J, V = [], [], []
        for bi, ri in enumerate(rows):
            items = list(ri.items()) + ([(bi, np.eye(bs))] if unit else [])
            for bj, blk in items:
                for a in range(bs):
                    for c in range(bs):
                        I.append(bi * bs + a); J.append(bj * bs + c); V.append(blk[a, c])
        return sp.csr_matrix((V, (I, J)), shape=(n, n))
    return assemble(L, True), assemble(U, False)


def ilu0_solver(S: sp.spmatrix, bs: int = 1) -> Solve:
    """r -> U^{-1} L^{-1} r with the ILU(0) factors of S (block forward and back substitution)."""
    L, U = ilu0(S, bs)
    Uinv = [np.linalg.inv(ri[i]) for i, ri in enumerate(U)]
    nb = len(L)

    def solve(r: np.ndarray) -> np.ndarray:
        y = np.array(r, dtype=np.float64).reshape(nb, bs)
        for i in range(nb):
            for j, blk in L[i].items():
                y[i] -= blk @ y[j]
        x = np.zeros_like(y)
        for i in range(nb - 1, -1, -1):
            t = y[i].copy()
            for j, blk in U[i].items():
                if j > i:
                    t -= blk @ x[j]
            x[i] = Uinv[i] @ t
        return x.ravel()
    return solve


def schur_approx(B1: sp.spmatrix, B2: sp.spmatrix, Z_full: sp.spmatrix, at_inv: np.ndarray,
                 scale: float = 1.0) -> sp.csr_matrix:
    """Z + scale * B2 A~^{-1} B1, assembled."""
    return (sp.csr_matrix(Z_full) + scale * (sp.csr_matrix(B2) @ sp.diags(at_inv) @ sp.csr_matrix(B1))).tocsr()


# ------------------------------------------------------------------ block smoothers (Sec. 5.1)
def uzawa_sweep(K, B1, B2, Z_full, u, lam, f, g, omega: float, k_solve: Solve, s_solve: Solve):
    """One Uzawa sweep (Algorithm 2).  k_solve(r) approximates K^{-1} r from a zero guess;
    s_solve(r) approximates S_hat^{-1} r."""
    du = k_solve(f - K @ u - B1 @ lam)
    dlam = -s_solve(g - B2 @ u + Z_full @ lam - B2 @ du)
    return u + omega * du, lam + omega * dlam


def braess_sarazin_sweep(K, B1, B2, Z_full, u, lam, f, g, omega: float, at_inv: np.ndarray, s_solve: Solve):
    """One Braess-Sarazin sweep (Algorithm 3).  s_solve(r) approximates
    (Z + (1/omega) B2 A~^{-1} B1)^{-1} r."""
    uh = u + (at_inv / omega) * (f - K @ u - B1 @ lam)
    dlam = -s_solve(g + Z_full @ lam - B2 @ uh)
    return uh - (at_inv / omega) * (B1 @ dlam), lam + dlam


def simple_sweep(K, B1, B2, Z_full, u, lam, f, g, omega: float, k_solve: Callable[[np.ndarray, np.ndarray], np.ndarray],
                 at_inv: np.ndarray, s_solve: Solve):
    """One SIMPLE sweep (Algorithm 4).  k_solve(rhs, x0) approximates K^{-1} rhs starting from x0
    (the current u); s_solve(r) approximates S_hat^{-1} r."""
    uh = k_solve(f - B1 @ lam, u)
    dlam = -s_solve(g + Z_full @ lam - B2 @ uh)
    return uh - omega * at_inv * (B1 @ dlam), lam + omega * dlam
