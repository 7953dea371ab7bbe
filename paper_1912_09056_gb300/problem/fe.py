"""Trilinear hex8 linear-elasticity assembly on structured bricks (input generation).

The paper's systems come from a finite element discretisation of each solid body
(Sec. 2.2: nodal displacement DOFs, first-order Lagrange elements).  This module
produces the stiffness block K of those systems for the synthetic workloads:
isotropic linear elasticity, 2x2x2 Gauss quadrature, assembled into a node-blocked
(3x3) sparse matrix.  It holds none of the multigrid method's arithmetic.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

# Local node order of the hex8 element in natural coordinates.
HEX8_XI = np.array(
    [[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
     [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], dtype=np.float64)

_G = 1.0 / np.sqrt(3.0)
GAUSS_2x2x2 = np.array([[a, b, c] for c in (-_G, _G) for b in (-_G, _G) for a in (-_G, _G)])


def hex8_dN_dxi(p: np.ndarray) -> np.ndarray:
    """Derivatives of the 8 trilinear shape functions at natural point p -> (8, 3)."""
    t = 1.0 + HEX8_XI * p[None, :]                      # (8,3) factors (1 + xi_a xi)
    d = np.empty((8, 3))
    d[:, 0] = 0.125 * HEX8_XI[:, 0] * t[:, 1] * t[:, 2]
    d[:, 1] = 0.125 * HEX8_XI[:, 1] * t[:, 0] * t[:, 2]
    d[:, 2] = 0.125 * HEX8_XI[:, 2] * t[:, 0] * t[:, 1]
    return d


def elasticity_matrix(E: float, nu: float) -> np.ndarray:
    """Isotropic Hooke matrix, Voigt order (xx, yy, zz, xy, yz, zx), engineering shear."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[0, 0] = C[1, 1] = C[2, 2] = lam + 2.0 * mu
    C[3, 3] = C[4, 4] = C[5, 5] = mu
    return C


def hex8_stiffness(X: np.ndarray, E: np.ndarray, nu: float) -> np.ndarray:
    """Element stiffness matrices for elements with nodal coordinates X (ne, 8, 3).

    E is the per-element Young's modulus (ne,), nu the Poisson ratio of the body.
    Returns (ne, 24, 24) with DOF order (node, component).
    """
    ne = X.shape[0]
    C1 = elasticity_matrix(1.0, nu)
    Ke = np.zeros((ne, 24, 24))
    B = np.zeros((ne, 6, 24))
    for p in GAUSS_2x2x2:
        dNdxi = hex8_dN_dxi(p)                           # (8,3)
        J = np.einsum("na,enb->eab", dNdxi, X)           # J_ab = d x_b / d xi_a
        detJ = np.linalg.det(J)
        if np.any(detJ <= 0):
            raise ValueError("inverted hex8 element")
        Jinv = np.linalg.inv(J)
        dNdx = np.einsum("eab,nb->ena", Jinv, dNdxi)     # (ne,8,3)
        B[:] = 0.0
        B[:, 0, 0::3] = dNdx[:, :, 0]
        B[:, 1, 1::3] = dNdx[:, :, 1]
        B[:, 2, 2::3] = dNdx[:, :, 2]
        B[:, 3, 0::3] = dNdx[:, :, 1]
        B[:, 3, 1::3] = dNdx[:, :, 0]
        B[:, 4, 1::3] = dNdx[:, :, 2]
        B[:, 4, 2::3] = dNdx[:, :, 1]
        B[:, 5, 0::3] = dNdx[:, :, 2]
        B[:, 5, 2::3] = dNdx[:, :, 0]
        CB = np.einsum("ij,ejb->eib", C1, B)
        Ke += np.matmul(B.transpose(0, 2, 1), CB) * (detJ * E)[:, None, None]
    return Ke


def brick_mesh(nx: int, ny: int, nz: int, lo, hi):
    """Structured brick [lo, hi] with nx*ny*nz hex8 elements.

    Returns (coords (nn,3), conn (ne,8), ijk (nn,3)).  Node id = i + (nx+1)(j + (ny+1)k).
    """
    xs = np.linspace(lo[0], hi[0], nx + 1)
    ys = np.linspace(lo[1], hi[1], ny + 1)
    zs = np.linspace(lo[2], hi[2], nz + 1)
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    i = i.ravel(); j = j.ravel(); k = k.ravel()
    coords = np.stack([xs[i], ys[j], zs[k]], axis=1)
    ijk = np.stack([i, j, k], axis=1)
    ek, ej, ei = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ei = ei.ravel(); ej = ej.ravel(); ek = ek.ravel()

    def nid(a, b, c):
        return a + (nx + 1) * (b + (ny + 1) * c)
    conn = np.stack([nid(ei, ej, ek), nid(ei + 1, ej, ek), nid(ei + 1, ej + 1, ek), nid(ei, ej + 1, ek),
                     nid(ei, ej, ek + 1), nid(ei + 1, ej, ek + 1), nid(ei + 1, ej + 1, ek + 1),
                     nid(ei, ej + 1, ek + 1)], axis=1).astype(np.int64)
    return coords, conn, ijk


def block_pattern(conn: np.ndarray, n_nodes: int):
    """Node-graph CSR (sorted columns, diagonal included) of the elements' couplings: the
    structure of E^T E for the element-node incidence matrix E.  Returns (rowptr, cols, keys)
    with keys = row * n_nodes + col in ascending order."""
    ne = conn.shape[0]
    inc = sp.csr_matrix((np.ones(ne * 8), (np.repeat(np.arange(ne, dtype=np.int64), 8), conn.ravel())),
                        shape=(ne, n_nodes))
    G = (inc.T.tocsr() @ inc).tocsr()
    G.sort_indices()
    rowptr = G.indptr.astype(np.int64)
    cols = G.indices.astype(np.int64)
    keys = np.repeat(np.arange(n_nodes, dtype=np.int64), np.diff(rowptr)) * n_nodes + cols
    return rowptr, cols, keys


def assemble_bsr(coords, conn, E_elem, nu, n_nodes):
    """Assemble K as node-blocked CSR: (rowptr, col, val (nnzb,3,3)).

    Elements that are translates of the body's last element (all but the jittered ones on a
    structured brick) share its unit-modulus matrix, scaled by their own E.  Contributions are
    added one local node pair (a, b) at a time: on a brick every node is local node a of at
    most one element, so the blocks of one pair land on distinct positions.
    """
    rowptr, cols, keys = block_pattern(conn, n_nodes)
    val = np.zeros((keys.size, 3, 3))
    rel = coords[conn] - coords[conn[:, :1]]
    h = np.abs(rel[-1]).max()
    same = np.abs(rel - rel[-1][None]).max(axis=(1, 2)) <= 1e-12 * h
    K_ref = hex8_stiffness(coords[conn[-1:]], np.ones(1), nu)[0]
    others = np.nonzero(~same)[0]
    K_oth = hex8_stiffness(coords[conn[others]], E_elem[others], nu) if others.size else None
    distinct = all(np.unique(conn[:, a]).size == conn.shape[0] for a in range(8))
    Es = E_elem[same]
    for a in range(8):
        for b in range(8):
            pos = np.searchsorted(keys, conn[:, a] * n_nodes + conn[:, b])
            blk = K_ref[3 * a:3 * a + 3, 3 * b:3 * b + 3]
            if distinct:
                val[pos[same]] += Es[:, None, None] * blk[None]
                if others.size:
                    val[pos[others]] += K_oth[:, 3 * a:3 * a + 3, 3 * b:3 * b + 3]
            else:
                np.add.at(val, pos[same], Es[:, None, None] * blk[None])
                if others.size:
                    np.add.at(val, pos[others], K_oth[:, 3 * a:3 * a + 3, 3 * b:3 * b + 3])
    return rowptr, cols, val


def element_shapes(coords, conn, nu):
    """Distinct unit-modulus element matrices of a brick: (shape id per element, Khat (ns,24,24)).

    Elements that are translates of the last element share shape 0; every other element gets
    its own shape (on the structured bricks these are the jittered interface elements).
    """
    rel = coords[conn] - coords[conn[:, :1]]
    h = np.abs(rel[-1]).max()
    same = np.abs(rel - rel[-1][None]).max(axis=(1, 2)) <= 1e-12 * h
    others = np.nonzero(~same)[0]
    shape = np.zeros(conn.shape[0], dtype=np.int32)
    shape[others] = 1 + np.arange(others.size, dtype=np.int32)
    Khat = np.empty((1 + others.size, 24, 24))
    Khat[0] = hex8_stiffness(coords[conn[-1:]], np.ones(1), nu)[0]
    if others.size:
        Khat[1:] = hex8_stiffness(coords[conn[others]], np.ones(others.size), nu)
    return shape, Khat
