"""Primal-dual active set strategy for the frictionless contact problem (oracle; test
infrastructure only, never imported by the product path).

The discrete contact conditions of Sec. 2 (Eqs. ch4_discretenormalcontact,
ch4_discretefrictionless) ask, at every slave node j, for a weighted gap g_j >= 0, a normal
multiplier lambda_n,j >= 0 with g_j lambda_n,j = 0, and zero tangential multipliers.  The primal-
dual active set strategy (PDASS, Sec. 2.2), a semi-smooth Newton method, finds the active set by
solving the linear saddle point system of the current set (active nodes: normal row g_j = 0 and
tangential rows T lambda_j = 0; inactive nodes: lambda_j = 0) and updating

    active_j  <=>  lambda_n,j - c g_j > 0

until the set no longer changes; the problem being linear here, the stop means that the
conditions hold.  Conventions of this package: n_j is the slave normal pointing to the master, so
that a compressive contact force gives lambda_j = lambda_n,j n_j with lambda_n,j > 0, and with a
geometric initial gap g0_j the weighted gap of the displaced configuration is

    g_j(u) = D_jj g0_j - n_j^T (D_jj u_s,j - sum_l M_jl u_m,l),

whose active rows are the normal rows of B2 with right-hand side D_jj g0_j.
"""
from __future__ import annotations

import copy
from typing import Callable, List, Optional

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .saddle import block_diag3, build_saddle


def assemble(prob):
    """A = [K B1; B2 -Z] of the problem's current active set."""
    S = build_saddle(prob)
    return sp.bmat([[S.K.val, S.B1.val], [S.B2.val, -block_diag3(S.Z)]], format="csr")


def weighted_gap(prob, g0: np.ndarray, u: np.ndarray) -> np.ndarray:
    """g_j(u) for every slave node j (the normal-row formula, whatever the node's status)."""
    ns = prob.n_s
    out = prob.D * g0
    for j in range(ns):
        n = prob.triad[j, 0]
        s = prob.slave_node[j]
        v = prob.D[j] * u[3 * s:3 * s + 3]
        for q in range(prob.M_rowptr[j], prob.M_rowptr[j + 1]):
            m = prob.master_node[prob.M_col[q]]
            v = v - prob.M_val[q] * u[3 * m:3 * m + 3]
        out[j] -= n @ v
    return out


def with_active_set(prob, g0: np.ndarray, active: np.ndarray):
    """A copy of the problem with the given active set and its constraint right-hand side."""
    p = copy.copy(prob)
    p.active = active.astype(np.uint8)
    g = np.zeros(3 * prob.n_s)
    g[0::3] = np.where(active, prob.D * g0, 0.0)
    p.g = g
    return p


def pdass(prob, g0: np.ndarray, c: float = 1.0, active0: Optional[np.ndarray] = None, max_steps: int = 50,
          solve: Optional[Callable] = None):
    """Runs the PDASS from active0 (default: every slave node active).  solve(p, A, b) returns the
    solution of A x = b for the step's problem p (default: sparse direct).  Returns the final
    problem, its solution and the list of active sets visited."""
    active = np.ones(prob.n_s, bool) if active0 is None else np.asarray(active0, bool).copy()
    history: List[np.ndarray] = []
    for _ in range(max_steps):
        p = with_active_set(prob, g0, active)
        A = assemble(p)
        b = p.rhs
        x = solve(p, A, b) if solve is not None else spla.spsolve(A.tocsc(), b)
        history.append(active.copy())
        nu = 3 * prob.n_nodes
        lam = x[nu:].reshape(-1, 3)
        lam_n = np.einsum("jk,jk->j", prob.triad[:, 0], lam)
        gap = weighted_gap(prob, g0, x[:nu])
        new_active = lam_n - c * gap > 0.0
        if np.array_equal(new_active, active):
            return p, x, history
        active = new_active
    raise RuntimeError("PDASS: active set did not settle")
