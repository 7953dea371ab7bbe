"""The linearised saddle-point operator A = [K B1; B2 -Z] (oracle).

Follows the block system of Sec. 2.3 (Eq. ch6_finalsaddlepointsystem and its compact form
Eq. ch6_finalsaddlepointsystem_comprehensive) for frictionless contact with Cartesian
multipliers:

* B1 (displacements x multipliers) is the transposed mortar operator: slave rows carry
  D^T, master rows carry -M^T, each entry times the 3x3 identity.
* B2 (multipliers x displacements): for an active slave node j the normal row is the
  linearised weighted gap n_j^T (D_jj u_s - sum_l M_jl u_m); its two tangential rows have
  no displacement entries.  Inactive rows have no displacement entries either.
* -Z: for an active node the normal row is zero and the tangential rows are the frictionless
  sliding conditions tau^T lambda_j = 0 (the T block); for an inactive node it is the
  identity row lambda_j = 0.

Block matrices are kept as scalar scipy CSR matrices for values plus node-level CSR
"patterns" (structural, never pruned) for the bit-exact comparison of sparsity.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


@dataclass
class BlockMat:
    """Scalar CSR values plus the node-level structural pattern (0/1 CSR)."""
    val: sp.csr_matrix
    pat: sp.csr_matrix
    br: int
    bc: int

    def blocks(self) -> np.ndarray:
        """Block values aligned with ``pat`` (row-major blocks, (nnzb, br, bc))."""
        P = self.pat.tocsr()
        P.sort_indices()
        rows = np.repeat(np.arange(P.shape[0], dtype=np.int64), np.diff(P.indptr))
        cols = P.indices.astype(np.int64)
        V = self.val.tocsr()
        V.sort_indices()
        ncol = np.int64(V.shape[1])
        vkeys = np.repeat(np.arange(V.shape[0], dtype=np.int64), np.diff(V.indptr)) * ncol + V.indices
        out = np.zeros((rows.size, self.br, self.bc))
        for a in range(self.br):
            for b in range(self.bc):
                k = (rows * self.br + a) * ncol + cols * self.bc + b
                pos = np.minimum(np.searchsorted(vkeys, k), max(vkeys.size - 1, 0))
                hit = vkeys[pos] == k if vkeys.size else np.zeros(k.size, bool)
                out[:, a, b] = np.where(hit, V.data[pos] if vkeys.size else 0.0, 0.0)
        return out


def pattern(rows, cols, shape) -> sp.csr_matrix:
    P = sp.csr_matrix((np.ones(len(rows)), (np.asarray(rows), np.asarray(cols))), shape=shape)
    P.data[:] = 1.0
    P.sort_indices()
    return P


def sym_product(*pats: sp.csr_matrix) -> sp.csr_matrix:
    """Structural product of node patterns (entries are positive counts: no cancellation)."""
    out = pats[0].astype(np.float64)
    for q in pats[1:]:
        out = (out @ q.astype(np.float64)).tocsr()
    out.data[:] = 1.0
    out.sort_indices()
    return out


def bsr_to_scalar(rowptr, col, val, n_brow, n_bcol) -> sp.csr_matrix:
    br, bc = val.shape[1], val.shape[2]
    rows = np.repeat(np.arange(n_brow), np.diff(rowptr))
    r = (rows[:, None, None] * br + np.arange(br)[None, :, None]) + 0 * np.arange(bc)[None, None, :]
    c = (np.asarray(col)[:, None, None] * bc + np.arange(bc)[None, None, :]) + 0 * np.arange(br)[None, :, None]
    A = sp.csr_matrix((val.ravel(), (r.ravel(), c.ravel())), shape=(n_brow * br, n_bcol * bc))
    A.sort_indices()
    return A


def block_diag3(Z: np.ndarray) -> sp.csr_matrix:
    """Scalar CSR of the nodal block-diagonal matrix with 3x3 blocks Z (n, 3, 3)."""
    n = Z.shape[0]
    r = (np.arange(n)[:, None, None] * 3 + np.arange(3)[None, :, None]) + 0 * np.arange(3)[None, None, :]
    c = (np.arange(n)[:, None, None] * 3 + np.arange(3)[None, None, :]) + 0 * np.arange(3)[None, :, None]
    M = sp.csr_matrix((Z.ravel(), (r.ravel(), c.ravel())), shape=(3 * n, 3 * n))
    M.sort_indices()
    return M


@dataclass
class Saddle:
    """Fine-level blocks of A = [K B1; B2 -Z] with nodal 3x3 blocks."""
    K: BlockMat
    B1: BlockMat
    B2: BlockMat
    Z: np.ndarray          # (n_s, 3, 3)
    n_nodes: int
    n_s: int

    def full(self) -> sp.csr_matrix:
        Zs = block_diag3(self.Z)
        return sp.bmat([[self.K.val, self.B1.val], [self.B2.val, -Zs]], format="csr")


def build_saddle(prob) -> Saddle:
    """Assemble the blocks of Eq. ch6_finalsaddlepointsystem_comprehensive from (K, D, M, triads, active)."""
    nn = prob.n_nodes
    ns = prob.n_s
    Kval = bsr_to_scalar(prob.K_rowptr, prob.K_col, prob.K_val, nn, nn)
    Kpat = pattern(np.repeat(np.arange(nn), np.diff(prob.K_rowptr)), prob.K_col, (nn, nn))
    I3 = np.eye(3)
    # B1: column j (multiplier node) has D_jj I3 at the slave node's row and -M_jl I3 at master rows
    r1, c1, v1 = [], [], []
    for j in range(ns):
        r1.append(prob.slave_node[j]); c1.append(j); v1.append(prob.D[j] * I3)
        for q in range(prob.M_rowptr[j], prob.M_rowptr[j + 1]):
            r1.append(prob.master_node[prob.M_col[q]]); c1.append(j); v1.append(-prob.M_val[q] * I3)
    # B2 / Z rows per multiplier node
    r2, c2, v2 = [], [], []
    Z = np.zeros((ns, 3, 3))
    for j in range(ns):
        n = prob.triad[j, 0]
        if prob.active[j]:
            row = np.zeros((3, 3)); row[0] = n
            r2.append(j); c2.append(prob.slave_node[j]); v2.append(prob.D[j] * row)
            for q in range(prob.M_rowptr[j], prob.M_rowptr[j + 1]):
                r2.append(j); c2.append(prob.master_node[prob.M_col[q]]); v2.append(-prob.M_val[q] * row)
            # -Z = [0; tau_xi^T; tau_eta^T]
            Z[j, 1] = -prob.triad[j, 1]
            Z[j, 2] = -prob.triad[j, 2]
        else:
            Z[j] = -I3
    B1 = _coo_blocks(r1, c1, v1, nn, ns, 3, 3)
    B2 = _coo_blocks(r2, c2, v2, ns, nn, 3, 3)
    return Saddle(K=BlockMat(Kval, Kpat, 3, 3), B1=B1, B2=B2, Z=Z, n_nodes=nn, n_s=ns)


def _coo_blocks(rows, cols, vals, nbr, nbc, br, bc) -> BlockMat:
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    if rows.size == 0:
        return BlockMat(sp.csr_matrix((nbr * br, nbc * bc)), sp.csr_matrix((nbr, nbc)), br, bc)
    vals = np.asarray(vals).reshape(-1, br, bc)
    rr = rows[:, None, None] * br + np.arange(br)[None, :, None] + 0 * np.arange(bc)[None, None, :]
    cc = cols[:, None, None] * bc + np.arange(bc)[None, None, :] + 0 * np.arange(br)[None, :, None]
    V = sp.csr_matrix((vals.ravel(), (rr.ravel(), cc.ravel())), shape=(nbr * br, nbc * bc))
    V.sum_duplicates()
    V.sort_indices()
    return BlockMat(V, pattern(rows, cols, (nbr, nbc)), br, bc)
