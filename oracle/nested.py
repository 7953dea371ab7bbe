"""Nested multigrid approach (Sec. 3.2, Fig. mgmphmodelsA) as a comparison preconditioner (oracle;
test infrastructure only, never imported by the product path).

The coupling between displacements and multipliers is treated only on the finest level, by an
outer SIMPLE iteration (Algorithm 4); single-field multigrid serves as the inner solver of the
displacement block:

    predictor   u_h = u + V_K (f - K u - B1 lam)          (one AMG V-cycle on K alone)
    corrector   -S_hat dlam = g + Z lam - B2 u_h          (S_hat = Z + B2 A~^{-1} B1, exact)
    update      lam += omega dlam,   u = u_h - omega A~^{-1} B1 dlam

The displacement hierarchy is built from K alone with the same components as the fully coupled
one: MIS-2 aggregates of K's node graph without inter-body couplings, tentative transfers from
the rigid-body modes, optionally smoothed (SA, omega = (4/3)/lambda_max), R = P^T and Galerkin
products; damped Jacobi pre- and post-smoothing with omega_J = (4/3)/lambda_max(D^{-1} K), and
LU on the coarsest level.  The multiplier field is small on these problems, so its Schur
approximation is solved directly (the limiting case of a nested solver for it).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .aggregate import aggregate_nodes, aggregation_graph
from .saddle import BlockMat, block_diag3, build_saddle, sym_product
from .smoother import atilde_diag
from .transfer import lambda_max, smoothed_prolongator, tentative_prolongator, transpose


@dataclass
class KLevel:
    K: BlockMat
    body: np.ndarray
    B: np.ndarray
    bu: int
    P: Optional[BlockMat] = None
    R: Optional[BlockMat] = None
    dinv: Optional[np.ndarray] = None
    omega_j: float = 0.0
    lu: Optional[tuple] = None


class KHierarchy:
    """Single-field AMG for the displacement block K."""

    def __init__(self, levels: List[KLevel], sweeps: int):
        self.levels = levels
        self.sweeps = sweeps

    def vcycle(self, b: np.ndarray, level: int = 0) -> np.ndarray:
        L = self.levels[level]
        if level == len(self.levels) - 1:
            return sla.lu_solve(L.lu, b)
        K = L.K.val
        x = np.zeros_like(b)
        for _ in range(self.sweeps):
            x = x + L.omega_j * L.dinv * (b - K @ x)
        x = x + L.P.val @ self.vcycle(L.R.val @ (b - K @ x), level + 1)
        for _ in range(self.sweeps):
            x = x + L.omega_j * L.dinv * (b - K @ x)
        return x


def k_hierarchy(K: BlockMat, body: np.ndarray, B: np.ndarray, levels_max: int = 10, coarse_max_rows: int = 5000,
                transfer: int = 1, sa_omega: float = 4.0 / 3.0, seed: int = 0x5EED, sweeps: int = 1) -> KHierarchy:
    levels = [KLevel(K=K, body=body, B=B, bu=K.br)]
    while len(levels) < levels_max and levels[-1].K.val.shape[0] >= coarse_max_rows:
        L = levels[-1]
        agg, roots = aggregate_nodes(aggregation_graph(L.K.pat, L.body), seed)
        n_agg = roots.size
        Phat, Bc = tentative_prolongator(agg, n_agg, L.B, L.bu)
        P = smoothed_prolongator(L.K, Phat, sa_omega / lambda_max(L.K.val)) if transfer == 1 else Phat
        R = transpose(P)
        Kc = BlockMat((R.val @ L.K.val @ P.val).tocsr(), sym_product(R.pat, L.K.pat, P.pat), 6, 6)
        Kc.val.sort_indices()
        L.P, L.R = P, R
        levels.append(KLevel(K=Kc, body=L.body[roots], B=Bc, bu=6))
        if Kc.val.shape[0] >= L.K.val.shape[0]:
            levels.pop()
            break
    for L in levels[:-1]:
        L.dinv = 1.0 / L.K.val.diagonal()
        L.omega_j = (4.0 / 3.0) / lambda_max(L.K.val)
    levels[-1].lu = sla.lu_factor(levels[-1].K.val.toarray())
    return KHierarchy(levels, sweeps)


class NestedPreconditioner:
    """Outer SIMPLE sweeps on the fine level with the K hierarchy's V-cycle as predictor."""

    def __init__(self, prob, outer_sweeps: int = 1, omega: float = 0.8, simplec: bool = False, **k_opts):
        S = build_saddle(prob)
        self.K = S.K.val.tocsr()
        self.B1 = S.B1.val.tocsr()
        self.B2 = S.B2.val.tocsr()
        self.Zf = block_diag3(S.Z).tocsr()
        self.nu = self.K.shape[0]
        self.kh = k_hierarchy(S.K, prob.body_id.astype(np.int64), prob.nullspace.copy(), **k_opts)
        self.at_inv = 1.0 / atilde_diag(self.K, simplec)
        Sh = (self.Zf + self.B2 @ sp.diags(self.at_inv) @ self.B1).toarray()
        self.s_lu = sla.lu_factor(Sh)
        self.sweeps = outer_sweeps
        self.omega = omega

    def A(self) -> sp.csr_matrix:
        return sp.bmat([[self.K, self.B1], [self.B2, -self.Zf]], format="csr")

    def apply(self, r: np.ndarray) -> np.ndarray:
        f, g = r[:self.nu], r[self.nu:]
        u = np.zeros(self.nu)
        lam = np.zeros(r.size - self.nu)
        for _ in range(self.sweeps):
            uh = u + self.kh.vcycle(f - self.K @ u - self.B1 @ lam)
            dlam = -sla.lu_solve(self.s_lu, g + self.Zf @ lam - self.B2 @ uh)
            lam = lam + self.omega * dlam
            u = uh - self.omega * self.at_inv * (self.B1 @ dlam)
        return np.concatenate([u, lam])
