"""Transfer operators and Galerkin products (oracle).

* Tentative prolongator for the displacements (Sec. 3.1.2): per aggregate, the rows of the
  level's nullspace B belonging to the aggregate's nodes (ascending node id, DOF-minor) are
  factorised B_agg = Q R (thin QR, R with positive diagonal); Q is the aggregate's block of
  P-hat and R becomes the coarse node's block of the coarse nullspace, so P-hat B_c = B.
* Tentative prolongator for the multipliers (Sec. 4.1, Eq. ch6_segregatedtransfers): the
  multiplier nullspace is one constant per Cartesian component; per multiplier aggregate the
  nullspace entries b_l of its nodes give P-hat^lambda[(l,c),(L,c)] = b_l / ||b_L|| and the
  coarse entry ||b_L||.
* Smoothed prolongator (Eq. ProlongatorSmoothing): P = P-hat - omega D^{-1} K P-hat with D the
  pointwise diagonal of K and omega = (4/3)/lambda_max(D^{-1}K).  lambda_max comes from 20
  power-iteration steps on D^{-1}K from the normalised all-ones vector followed by the
  generalised Rayleigh quotient (x^T K x)/(x^T D x).
* Restriction R = P^T (Sec. 3.1.2 and Sec. 6.2 setup) and the block Galerkin products of the
  segregated transfers (Sec. 4.1): K_c = P^T K P, B1_c = P^T B1 P^lambda,
  B2_c = P^lambda^T B2 P, Z_c = P^lambda^T Z P^lambda.  Patterns are structural products.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .saddle import BlockMat, pattern, sym_product


def tentative_prolongator(agg: np.ndarray, n_agg: int, B: np.ndarray, bu: int):
    """P-hat (BlockMat, bu x 6 blocks) and coarse nullspace (6 n_agg, 6)."""
    nn = agg.size
    rows, cols, vals = [], [], []
    Bc = np.zeros((6 * n_agg, 6))
    order = np.argsort(agg, kind="stable")           # nodes grouped by aggregate, ascending id
    starts = np.searchsorted(agg[order], np.arange(n_agg + 1))
    for a in range(n_agg):
        nodes = order[starts[a]:starts[a + 1]]
        dof = (nodes[:, None] * bu + np.arange(bu)[None, :]).ravel()
        Q, R = np.linalg.qr(B[dof], mode="reduced")
        if Q.shape[1] < 6:
            raise np.linalg.LinAlgError("aggregate has fewer than 6 DOFs")
        s = np.sign(np.diag(R))
        if np.any(s == 0) or np.min(np.abs(np.diag(R))) < 1e-12 * np.max(np.abs(np.diag(R))):
            raise np.linalg.LinAlgError("rank-deficient nullspace on an aggregate")
        Q = Q * s[None, :]
        R = R * s[:, None]
        Bc[6 * a:6 * a + 6] = R
        rr = np.repeat(dof, 6)
        cc = np.tile(6 * a + np.arange(6), dof.size)
        rows.append(rr); cols.append(cc); vals.append(Q.ravel())
    V = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nn * bu, n_agg * 6))
    V.sort_indices()
    return BlockMat(V, pattern(np.arange(nn), agg, (nn, n_agg)), bu, 6), Bc


def tentative_lagmult(lagg: np.ndarray, n_lagg: int, Bl: np.ndarray):
    """P-hat^lambda (BlockMat, 3x3 diagonal blocks) and coarse multiplier nullspace."""
    nl = lagg.size
    norm = np.sqrt(np.bincount(lagg, weights=Bl * Bl, minlength=n_lagg))
    w = Bl / norm[lagg]
    rows = (np.arange(nl)[:, None] * 3 + np.arange(3)[None, :]).ravel()
    cols = (lagg[:, None] * 3 + np.arange(3)[None, :]).ravel()
    V = sp.csr_matrix((np.repeat(w, 3), (rows, cols)), shape=(3 * nl, 3 * n_lagg))
    V.sort_indices()
    return BlockMat(V, pattern(np.arange(nl), lagg, (nl, n_lagg)), 3, 3), norm


def lambda_max(K: sp.csr_matrix, iters: int = 20) -> float:
    """Largest eigenvalue estimate of D^{-1} K (power iteration, then Rayleigh quotient)."""
    d = K.diagonal()
    n = K.shape[0]
    x = np.ones(n) / np.sqrt(n)
    for _ in range(iters):
        y = (K @ x) / d
        x = y / np.linalg.norm(y)
    return float(x @ (K @ x)) / float(x @ (d * x))


def smoothed_prolongator(K: BlockMat, Phat: BlockMat, omega: float) -> BlockMat:
    """P = P-hat - omega D^{-1} K P-hat with its structural pattern."""
    d = K.val.diagonal()
    KP = (K.val @ Phat.val).tocsr()
    V = (Phat.val - sp.diags(omega / d) @ KP).tocsr()
    V.sort_indices()
    pat = sym_product(K.pat, Phat.pat)
    pat = ((pat + Phat.pat) > 0).astype(np.float64).tocsr()
    pat.sort_indices()
    return BlockMat(V, pat, Phat.br, Phat.bc)


def transpose(A: BlockMat) -> BlockMat:
    V = A.val.T.tocsr(); V.sort_indices()
    P = A.pat.T.tocsr(); P.sort_indices()
    return BlockMat(V, P, A.bc, A.br)


def galerkin(K: BlockMat, B1: BlockMat, B2: BlockMat, Z: np.ndarray,
             P: BlockMat, Pl: BlockMat, lagg: np.ndarray, n_lagg: int):
    """Coarse blocks (K_c, B1_c, B2_c, Z_c) of the segregated Galerkin product."""
    R = transpose(P)
    Rl = transpose(Pl)
    Kc = BlockMat((R.val @ K.val @ P.val).tocsr(), sym_product(R.pat, K.pat, P.pat), 6, 6)
    B1c = BlockMat((R.val @ B1.val @ Pl.val).tocsr(), sym_product(R.pat, B1.pat, Pl.pat), 6, 3)
    B2c = BlockMat((Rl.val @ B2.val @ P.val).tocsr(), sym_product(Rl.pat, B2.pat, P.pat), 3, 6)
    w = np.asarray(Pl.val.sum(axis=1)).ravel()[0::3]      # P^lambda weight per fine node
    Zc = np.zeros((n_lagg, 3, 3))
    np.add.at(Zc, lagg, (w * w)[:, None, None] * Z)
    for M in (Kc, B1c, B2c):
        M.val.sort_indices()
    return Kc, B1c, B2c, Zc
