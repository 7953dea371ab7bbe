"""Differentiable solves through the amgc C-ABI (marshalling only; the work runs in libamgc).

``SaddleSolve`` wraps amgc_solve in a ``torch.autograd.Function``: x = A(K)^{-1} b, and its
backward solves the transposed system with the transposed hierarchy (amgc_solve_transposed)
and scatters -adj (x) x onto the stored blocks of K (amgc_grad_scatter), giving the gradients
with respect to the stiffness values and the right-hand side.

``contact_gradients`` evaluates the contact objective
    J = sum over active slave nodes of the normal multiplier n_j . lambda_j
        + 0.5 * sum over master interface nodes of |u_m|^2
and its gradients with respect to the element moduli E_e (K = sum_e E_e Khat_e, f = -K_fD u_D)
and the uniform prescribed top displacement, through one adjoint solve and amgc_grad_elements.
"""
from __future__ import annotations

import copy

import numpy as np
import torch

from . import amgc


def _device_problem(prob, K_val: torch.Tensor):
    p = copy.copy(prob)
    p.K_val = K_val.detach().contiguous()
    return p


class SaddleSolve(torch.autograd.Function):
    """The forward hierarchy is kept for the backward pass only: it is released as soon as no
    gradient is needed (forward without grad) or once the backward pass has used it.  A second
    backward pass through the same graph (retain_graph=True) sets the hierarchy up again."""

    @staticmethod
    def forward(ctx, K_val, b, prob, opts, adj_tol):
        h = amgc.setup(_device_problem(prob, K_val), opts)
        x = torch.zeros_like(b)
        h.solve(b.detach().contiguous(), x)
        ctx.adj_tol = adj_tol
        ctx.rebuild = (prob, K_val.detach(), opts)
        if any(ctx.needs_input_grad[:2]):
            ctx.h = h
        else:
            h.close()
            ctx.h = None
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        h = ctx.h
        if h is None:
            prob, K_val, opts = ctx.rebuild
            h = amgc.setup(_device_problem(prob, K_val), opts)
        ctx.h = None
        try:
            adj = torch.zeros_like(gx)
            h.solve_transposed(gx.contiguous(), adj, tol=ctx.adj_tol)
            gK = torch.empty((h.export(0, "k_col").size, 3, 3), dtype=torch.float64, device=x.device)
            h.grad_scatter(adj, x, gK)
        finally:
            h.close()
        return gK, adj, None, None, None


def saddle_solve(K_val: torch.Tensor, b: torch.Tensor, prob, opts=None, adj_tol: float = 1e-10):
    """x = A^{-1} b with A assembled from prob's structure and the stiffness values K_val."""
    return SaddleSolve.apply(K_val, b, prob, opts if opts is not None else amgc.default_options(), adj_tol)


def objective_gradient(prob, x: torch.Tensor):
    """J(x) and dJ/dx for the contact objective (slave normal multipliers + master-face energy)."""
    dev = x.device
    n_u = prob.n_u
    c = torch.zeros_like(x)
    act = torch.from_numpy(np.nonzero(prob.active)[0]).to(dev)
    nrm = torch.from_numpy(prob.triad[:, 0, :]).to(dev)
    lam = x[n_u:].view(-1, 3)
    J = (lam[act] * nrm[act]).sum()
    c[n_u:].view(-1, 3)[act] = nrm[act]
    mn = torch.from_numpy(prob.master_node.astype(np.int64)).to(dev)
    u = x[:n_u].view(-1, 3)
    J = J + 0.5 * (u[mn] ** 2).sum()
    c[:n_u].view(-1, 3)[mn] = u[mn]
    return J, c


class ElementTables:
    """Device copies of the element data amgc_grad_elements reads (from keep_full problems)."""

    def __init__(self, prob, device="cuda"):
        e = prob.extra
        t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(device)  # noqa: E731
        self.conn = t(e["conn"], np.int32)
        self.shape = t(e["elem_shape"], np.int32)
        self.Khat = t(e["Khat"], np.float64)
        self.node_free = t(e["node_free"], np.int32)
        self.uD = t(e["u_D"], np.float64)
        self.E = t(e["E_elem"], np.float64)
        self.top = t(e["top_mask"], np.uint8)
        self.ne = int(self.conn.shape[0])


def contact_gradients(prob, h, x: torch.Tensor, tables: ElementTables, adj_tol: float = 1e-10):
    """(J, dJ/dE (ne), dJ/dt (3), adjoint, adjoint iterations) for the solution x of hierarchy h."""
    J, c = objective_gradient(prob, x)
    adj = torch.zeros_like(x)
    it, _, _ = h.solve_transposed(c, adj, tol=adj_tol)
    gE = torch.empty(tables.ne, dtype=torch.float64, device=x.device)
    gt = torch.empty(3, dtype=torch.float64, device=x.device)
    amgc.grad_elements(tables.conn, tables.shape, tables.Khat, tables.node_free, adj, x, tables.uD, tables.E, gE,
                       lift_mask=tables.top, gt=gt)
    return J, gE, gt, adj, it
