"""Fully coupled block-AMG hierarchy and V-cycle (oracle).

Setup (Sec. 3.1.2, Sec. 4, Algorithm 1): on every level but the coarsest,
  1. node graph of K without inter-body couplings, MIS-2 displacement aggregates;
  2. multiplier aggregates by Algorithm 1 through the pattern of the level's D coupling
     (level 0: the diagonal dual-mortar D between slave node j and multiplier node j;
     coarser levels: the structural pattern of P-hat^T D P-hat^lambda, which couples coarse
     multiplier node L only to the displacement aggregate it was derived from);
  3. tentative transfers, optionally smoothed displacement prolongator (SA), R = P^T;
  4. segregated Galerkin products for K, B1, B2, Z;
  5. CheapSIMPLE data: omega_J, D_K^{-1}, A_tilde^{-1} and the inverted nodal blocks of S_hat
     (optionally the Schur-step damping min(alpha, (4/3)/rho(S_bd^{-1} S_hat)), Sec. 5.2).
Coarsening stops at ``levels_max`` levels or once the saddle system has fewer than
``coarse_max_rows`` rows (Sec. 6.2 setup); the coarsest level is merged into one dense
matrix [K_c B1_c; B2_c -Z_c] and solved by LU with partial pivoting (Sec. 6.2 setup).

V-cycle (Fig. mgalgorithm), zero initial guess on every level: pre-smooth, residual,
restrict, recurse, prolongate and add, post-smooth; coarsest level: direct solve.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .aggregate import aggregate_nodes, aggregation_graph, lagmult_aggregation
from .saddle import BlockMat, block_diag3, build_saddle
from .blocksmoothers import (braess_sarazin_sweep, colored_block_sgs, ilu0_solver, jp_coloring, schur_approx,
                             simple_sweep, uzawa_sweep)
from .blocksmoothers import sgs as sgs_point
from .smoother import atilde_diag, cheap_simple_sweep, schur_blocks, schur_rho
from .transfer import galerkin, lambda_max, smoothed_prolongator, tentative_lagmult, tentative_prolongator, transpose


@dataclass
class Options:
    levels_max: int = 10
    coarse_max_rows: int = 5000
    transfer: int = 0            # 0 = PA (tentative), 1 = SA (smoothed displacement prolongator)
    sa_omega: float = 4.0 / 3.0
    smoother_sweeps: int = 1     # CheapSIMPLE sweeps, pre and post
    jacobi_sweeps: int = 1       # Jacobi sweeps in the predictor
    jacobi_omega: float = 0.0    # <= 0: (4/3)/lambda_max(D^{-1}K)
    simple_alpha: float = 0.8
    simplec: int = 0             # 0: A_tilde = diag(K), 1: absolute row sums (SIMPLEC)
    seed: int = 0x5EED
    schur_damping: int = 0       # 1: alpha -> min(alpha, (4/3)/rho(S_bd^-1 S_hat)) per level
    # level smoother: "cheap_simple" (the default above), or a cheap block smoother of Sec. 5.1 /
    # 5.2 with SGS for K and nodal-block ILU(0) for its Schur approximation: "uzawa",
    # "braess_sarazin", "simple_sgs" (SIMPLE, or SIMPLEC with simplec = 1)
    smoother: str = "cheap_simple"
    # coarsest level: "lu" (merged dense matrix, LU with partial pivoting) or "smoother" (the level
    # smoother's sweeps from a zero guess, no merged matrix; the paper's alternative, Sec. 6.2)
    coarse_solver: str = "lu"
    block_omega: float = 0.7     # damping of the block smoother (the paper's omega)
    sgs_sweeps: int = 1
    sgs_omega: float = 0.7
    sgs_kind: str = "point"      # "point": natural-order pointwise SGS; "colored_block": nodal-block
                                 # SGS in Jones-Plassmann colour order (the data-parallel form)
    fgmres_restart: int = 50
    fgmres_maxit: int = 1000
    tol: float = 1e-8


@dataclass
class Level:
    K: BlockMat
    B1: BlockMat
    B2: BlockMat
    Z: np.ndarray
    body: np.ndarray
    B: np.ndarray            # displacement nullspace (bu*nn, 6)
    Bl: np.ndarray           # multiplier nullspace entry per multiplier node
    lm_dnode: np.ndarray     # multiplier node -> displacement node it couples to through D
    bu: int
    # transfer to the next level
    agg: Optional[np.ndarray] = None
    n_agg: int = 0
    lagg: Optional[np.ndarray] = None
    n_lagg: int = 0
    Phat: Optional[BlockMat] = None
    P: Optional[BlockMat] = None
    Pl: Optional[BlockMat] = None
    R: Optional[BlockMat] = None
    Rl: Optional[BlockMat] = None
    # smoother
    lam_max: float = 0.0
    omega_j: float = 0.0
    dinv: Optional[np.ndarray] = None
    at_inv: Optional[np.ndarray] = None
    S_blocks: Optional[np.ndarray] = None
    S_inv: Optional[np.ndarray] = None
    alpha: float = 0.0           # damping of the multiplier correction on this level
    schur_rho: float = 0.0
    # coarsest
    lu: Optional[tuple] = None
    extra: dict = field(default_factory=dict)

    @property
    def nn(self) -> int:
        return self.body.size

    @property
    def nl(self) -> int:
        return self.Z.shape[0]

    @property
    def nu_dofs(self) -> int:
        return self.bu * self.nn

    @property
    def rows(self) -> int:
        return self.bu * self.nn + 3 * self.nl

    def Z_full(self) -> sp.csr_matrix:
        return block_diag3(self.Z)

    def A(self) -> sp.csr_matrix:
        return sp.bmat([[self.K.val, self.B1.val], [self.B2.val, -self.Z_full()]], format="csr")


def d_rows(level: Level):
    """Rows of the level's D coupling as (slave DOF, [multiplier DOFs]) in ascending DOF order."""
    out = []
    order = np.argsort(level.lm_dnode, kind="stable")
    for l in order:
        k = int(level.lm_dnode[l])
        for r in range(level.bu):
            if level.extra.get("fine", False):
                js = [3 * int(l) + r]                      # D (x) I3 on the fine level
            else:
                js = [3 * int(l) + c for c in range(3)]     # full 6x3 coupling block
            out.append((level.bu * k + r, js))
    out.sort(key=lambda t: t[0])
    return out


class Hierarchy:
    def __init__(self, levels: List[Level], opts: Options):
        self.levels = levels
        self.opts = opts

    @property
    def n_levels(self) -> int:
        return len(self.levels)

    def operator_complexity(self) -> float:
        nnz = [L.A().nnz for L in self.levels]
        return float(sum(nnz)) / float(nnz[0])

    # ---------------------------------------------------------------- V-cycle
    def smooth(self, L: Level, u, lam, f, g):
        o = self.opts
        Zf = L.Z_full()
        K, B1, B2 = L.K.val, L.B1.val, L.B2.val
        if o.smoother != "cheap_simple":
            return self._block_smooth(L, u, lam, f, g, Zf)

        def s_inv(r):
            return np.einsum("lij,lj->li", L.S_inv, r.reshape(-1, 3)).ravel()
        for _ in range(o.smoother_sweeps):
            u, lam = cheap_simple_sweep(K, B1, B2, Zf, u, lam, f, g, L.dinv,
                                        L.omega_j, o.jacobi_sweeps, L.at_inv, s_inv, L.alpha)
        return u, lam

    def _block_smooth(self, L: Level, u, lam, f, g, Zf):
        """Cheap Uzawa, Braess-Sarazin or SIMPLE(C) sweeps (Algorithms 2-4, Sec. 5.2): SGS for K,
        ILU(0) on the nodal 3 x 3 blocks of the Schur approximation (built on first use)."""
        o = self.opts
        K, B1, B2 = L.K.val, L.B1.val, L.B2.val
        w = o.block_omega
        if "block_s_solve" not in L.extra:
            if L.nl == 0:
                L.extra["block_s_solve"] = lambda r: r
            else:
                scale = 1.0 / w if o.smoother == "braess_sarazin" else 1.0
                L.extra["block_s_solve"] = ilu0_solver(schur_approx(B1, B2, Zf, L.at_inv, scale), 3)
        s_solve = L.extra["block_s_solve"]
        zero = np.zeros(L.nu_dofs)
        sgs = sgs_point
        if o.sgs_kind == "colored_block":
            if "colored_sgs" not in L.extra:
                col = jp_coloring(aggregation_graph(L.K.pat, np.zeros(L.nn, dtype=np.int64)), o.seed)
                L.extra["colored_sgs"] = colored_block_sgs(K, col, L.bu)
            prepared = L.extra["colored_sgs"]

            def sgs(K, r, x0, sweeps, omega):
                return prepared(r, x0, sweeps, omega)
        for _ in range(o.smoother_sweeps):
            if o.smoother == "uzawa":
                u, lam = uzawa_sweep(K, B1, B2, Zf, u, lam, f, g, w,
                                     lambda r: sgs(K, r, zero, o.sgs_sweeps, o.sgs_omega), s_solve)
            elif o.smoother == "braess_sarazin":
                u, lam = braess_sarazin_sweep(K, B1, B2, Zf, u, lam, f, g, w, L.at_inv, s_solve)
            elif o.smoother == "simple_sgs":
                u, lam = simple_sweep(K, B1, B2, Zf, u, lam, f, g, w,
                                      lambda r, x0: sgs(K, r, x0, o.sgs_sweeps, o.sgs_omega), L.at_inv, s_solve)
            else:
                raise ValueError(f"unknown smoother {o.smoother!r}")
        return u, lam

    def residual(self, L: Level, u, lam, f, g):
        ru = f - L.K.val @ u - L.B1.val @ lam
        rl = g - L.B2.val @ u + L.Z_full() @ lam
        return ru, rl

    def vcycle(self, b: np.ndarray, level: int = 0) -> np.ndarray:
        L = self.levels[level]
        nu = L.nu_dofs
        if level == self.n_levels - 1:
            if self.opts.coarse_solver == "smoother" and self.n_levels > 1:
                u, lam = self.smooth(L, np.zeros(nu), np.zeros(b.size - nu), b[:nu], b[nu:])
                return np.concatenate([u, lam])
            return sla.lu_solve(L.lu, b)
        f, g = b[:nu], b[nu:]
        u = np.zeros(nu)
        lam = np.zeros(b.size - nu)
        u, lam = self.smooth(L, u, lam, f, g)
        ru, rl = self.residual(L, u, lam, f, g)
        rc = np.concatenate([L.R.val @ ru, L.Rl.val @ rl])
        c = self.vcycle(rc, level + 1)
        nuc = self.levels[level + 1].nu_dofs
        u = u + L.P.val @ c[:nuc]
        lam = lam + L.Pl.val @ c[nuc:]
        u, lam = self.smooth(L, u, lam, f, g)
        return np.concatenate([u, lam])

    def A0(self) -> sp.csr_matrix:
        return self.levels[0].A()


def setup(prob, opts: Optional[Options] = None, reuse: Optional[Hierarchy] = None) -> Hierarchy:
    """Build the hierarchy for a ContactProblem (all FP64).

    reuse: a hierarchy of the same problem under another active set.  Only the constraint blocks
    B2 and Z depend on the active set; the aggregates, the transfers, lambda_max and the coarse K
    (the expensive parts of the setup) are taken from it, and the coarse B1, B2, Z, the smoother
    data and the coarsest factorisation are formed anew.
    """
    o = opts or Options()
    S = build_saddle(prob)
    L0 = Level(K=S.K, B1=S.B1, B2=S.B2, Z=S.Z, body=prob.body_id.astype(np.int64),
               B=prob.nullspace.copy(), Bl=np.ones(prob.n_s), lm_dnode=prob.slave_node.astype(np.int64), bu=3)
    L0.extra["fine"] = True
    levels = [L0]
    if reuse is not None:
        for Lr in reuse.levels[:-1]:
            L = levels[-1]
            for name in ("agg", "n_agg", "lagg", "n_lagg", "Phat", "P", "Pl", "R", "Rl", "lam_max"):
                setattr(L, name, getattr(Lr, name))
            _, B1c, B2c, Zc = galerkin(L.K, L.B1, L.B2, L.Z, L.P, L.Pl, L.lagg, L.n_lagg)
            nxt = reuse.levels[len(levels)]
            levels.append(Level(K=nxt.K, B1=B1c, B2=B2c, Z=Zc, body=nxt.body, B=nxt.B, Bl=nxt.Bl,
                                lm_dnode=nxt.lm_dnode, bu=nxt.bu))
    while reuse is None and len(levels) < o.levels_max and levels[-1].rows >= o.coarse_max_rows:
        L = levels[-1]
        G = aggregation_graph(L.K.pat, L.body)
        agg, roots = aggregate_nodes(G, o.seed)
        n_agg = roots.size
        lagg_d, dmap, n_lagg = lagmult_aggregation(agg, d_rows(L), L.bu)
        lagg = np.array([lagg_d[l] for l in range(L.nl)], dtype=np.int64)
        Phat, Bc = tentative_prolongator(agg, n_agg, L.B, L.bu)
        Pl, Blc = tentative_lagmult(lagg, n_lagg, L.Bl)
        L.lam_max = lambda_max(L.K.val)
        P = smoothed_prolongator(L.K, Phat, o.sa_omega / L.lam_max) if o.transfer == 1 else Phat
        Kc, B1c, B2c, Zc = galerkin(L.K, L.B1, L.B2, L.Z, P, Pl, lagg, n_lagg)
        L.agg, L.n_agg, L.lagg, L.n_lagg = agg, n_agg, lagg, n_lagg
        L.Phat, L.P, L.Pl = Phat, P, Pl
        L.R, L.Rl = transpose(P), transpose(Pl)
        body_c = L.body[roots]
        inv_d = {v: k for k, v in dmap.items()}
        lm_dnode_c = np.array([inv_d[Lc] for Lc in range(n_lagg)], dtype=np.int64)
        levels.append(Level(K=Kc, B1=B1c, B2=B2c, Z=Zc, body=body_c, B=Bc, Bl=Blc,
                            lm_dnode=lm_dnode_c, bu=6))
    # smoother data on all but the coarsest level (on all levels when it smooths the coarsest)
    smoothed = levels if (o.coarse_solver == "smoother" and len(levels) > 1) else levels[:-1]
    for L in smoothed:
        if L.lam_max == 0.0:
            L.lam_max = lambda_max(L.K.val)
        L.omega_j = o.jacobi_omega if o.jacobi_omega > 0 else (4.0 / 3.0) / L.lam_max
        L.dinv = 1.0 / L.K.val.diagonal()
        L.at_inv = 1.0 / atilde_diag(L.K.val, bool(o.simplec))
        L.S_blocks = schur_blocks(L.B1.val, L.B2.val, L.Z, L.at_inv)
        L.S_inv = np.linalg.inv(L.S_blocks)
        L.alpha = o.simple_alpha
        if o.schur_damping and L.nl > 0:
            L.schur_rho = schur_rho(L.B1.val, L.B2.val, L.Z, L.at_inv, L.S_inv)
            L.alpha = min(o.simple_alpha, (4.0 / 3.0) / L.schur_rho)
    Lc = levels[-1]
    Lc.lu = sla.lu_factor(Lc.A().toarray())
    return Hierarchy(levels, o)
