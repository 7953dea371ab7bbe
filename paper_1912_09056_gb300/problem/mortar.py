"""Segment-based dual-mortar coupling matrices D and M on a flat interface (input generation).

The paper's contact force uses two mortar matrices D (slave x slave) and M (slave x
master) built from the Lagrange-multiplier basis on the slave surface (Sec. 2.2); with
dual (biorthogonal) multiplier shape functions D is diagonal (Sec. 2.3).  The paper
defers the integration itself to the mortar literature, so this module states the
construction used for the synthetic workloads:

* slave surface: bilinear quad4 faces (in-plane jittered nodes allowed), master
  surface: an axis-aligned structured grid of quad4 faces, both lying in one plane,
  so the projection onto the slave auxiliary plane is the identity;
* dual basis per slave face e: psi_j = sum_k a_jk N_k with A_e = D_e M_e^{-1},
  D_e = diag(int_e N_j), M_e = (int_e N_j N_k)  (3x3 Gauss on the face);
* each slave/master face pair is clipped (Sutherland-Hodgman), the overlap polygon is
  split into triangles about its vertex centroid and integrated with the 7-point
  degree-5 triangle rule (Radon); slave parameters come from a Newton inverse of
  the bilinear map;
* M_jl = sum over segments of int psi_j N^m_l, and D_jj = sum over segments of
  int psi_j, i.e. the same quadrature, so that sum_l M_jl = D_jj holds to rounding
  wherever the master covers the slave (the mortar patch condition).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

# Quad4 local corners (xi, eta) in counter-clockwise order.
QUAD_XI = np.array([[-1.0, -1.0], [1.0, -1.0], [1.0, 1.0], [-1.0, 1.0]])

_G3 = np.array([-np.sqrt(0.6), 0.0, np.sqrt(0.6)])
_W3 = np.array([5.0, 8.0, 5.0]) / 9.0

# Radon's 7-point degree-5 rule on the reference triangle, barycentric coordinates,
# weights relative to the triangle area.
_s15 = np.sqrt(15.0)
_a1 = (6.0 - _s15) / 21.0
_a2 = (6.0 + _s15) / 21.0
TRI7_BARY = np.array([
    [1 / 3, 1 / 3, 1 / 3],
    [_a1, _a1, 1 - 2 * _a1], [_a1, 1 - 2 * _a1, _a1], [1 - 2 * _a1, _a1, _a1],
    [_a2, _a2, 1 - 2 * _a2], [_a2, 1 - 2 * _a2, _a2], [1 - 2 * _a2, _a2, _a2]])
TRI7_W = np.array([9 / 40] + [(155 - _s15) / 1200] * 3 + [(155 + _s15) / 1200] * 3)


def quad_N(xi: np.ndarray, eta: np.ndarray) -> np.ndarray:
    """Bilinear shape functions, (..., 4)."""
    return 0.25 * (1 + QUAD_XI[:, 0] * xi[..., None]) * (1 + QUAD_XI[:, 1] * eta[..., None])


def quad_map(X: np.ndarray, xi, eta):
    """Physical point and Jacobian of the bilinear map of corners X (4,2)."""
    N = quad_N(xi, eta)
    x = N @ X
    dxi = 0.25 * QUAD_XI[:, 0] * (1 + QUAD_XI[:, 1] * eta[..., None])
    deta = 0.25 * QUAD_XI[:, 1] * (1 + QUAD_XI[:, 0] * xi[..., None])
    J = np.stack([dxi @ X, deta @ X], axis=-2)          # (...,2,2): rows d/dxi, d/deta
    return x, J


def quad_inverse_map(X: np.ndarray, pts: np.ndarray, iters: int = 30, tol: float = 1e-14):
    """Newton inverse of the bilinear map for points pts (n,2) -> (xi, eta)."""
    xi = np.zeros(pts.shape[0])
    eta = np.zeros(pts.shape[0])
    for _ in range(iters):
        x, J = quad_map(X, xi, eta)
        r = pts - x
        # solve J^T d = r  (x = x0 + d_xi * dx/dxi + d_eta * dx/deta)
        a, b = J[:, 0, 0], J[:, 1, 0]
        c, d = J[:, 0, 1], J[:, 1, 1]
        det = a * d - b * c
        dxi = (d * r[:, 0] - b * r[:, 1]) / det
        deta = (-c * r[:, 0] + a * r[:, 1]) / det
        xi += dxi
        eta += deta
        if np.max(np.abs(dxi) + np.abs(deta)) < tol:
            break
    return xi, eta


def dual_coefficients(X: np.ndarray) -> np.ndarray:
    """A_e = D_e M_e^{-1} for one slave face with corners X (4,2)."""
    xi, eta = np.meshgrid(_G3, _G3, indexing="ij")
    w = np.outer(_W3, _W3).ravel()
    xi = xi.ravel(); eta = eta.ravel()
    N = quad_N(xi, eta)                                   # (9,4)
    _, J = quad_map(X, xi, eta)
    detJ = J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
    wd = w * detJ
    De = N.T @ wd
    Me = (N * wd[:, None]).T @ N
    return np.diag(De) @ np.linalg.inv(Me)


def clip_polygon_rect(poly: np.ndarray, x0, x1, y0, y1) -> np.ndarray:
    """Sutherland-Hodgman clip of polygon (n,2) against the rectangle [x0,x1]x[y0,y1]."""
    def clip(P, axis, bound, keep_ge):
        if len(P) == 0:
            return P
        out = []
        n = len(P)
        for i in range(n):
            cur = P[i]
            prv = P[i - 1]
            cin = (cur[axis] >= bound) if keep_ge else (cur[axis] <= bound)
            pin = (prv[axis] >= bound) if keep_ge else (prv[axis] <= bound)
            if cin:
                if not pin:
                    t = (bound - prv[axis]) / (cur[axis] - prv[axis])
                    out.append(prv + t * (cur - prv))
                out.append(cur)
            elif pin:
                t = (bound - prv[axis]) / (cur[axis] - prv[axis])
                out.append(prv + t * (cur - prv))
        return np.array(out) if out else np.zeros((0, 2))
    P = np.asarray(poly, dtype=np.float64)
    P = clip(P, 0, x0, True)
    P = clip(P, 0, x1, False)
    P = clip(P, 1, y0, True)
    P = clip(P, 1, y1, False)
    return P


def polygon_area(P: np.ndarray) -> float:
    x, y = P[:, 0], P[:, 1]
    return 0.5 * float(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))


def quad_inverse_map_batched(X: np.ndarray, pts: np.ndarray, iters: int = 30, tol: float = 1e-14):
    """Newton inverse of the bilinear maps of corners X (n,4,2), one map per point pts (n,2);
    every point iterates until its own step is below tol (at most `iters` steps)."""
    n = pts.shape[0]
    xi = np.zeros(n)
    eta = np.zeros(n)
    live = np.arange(n)
    for _ in range(iters):
        if live.size == 0:
            break
        Xl = X[live]
        N = quad_N(xi[live], eta[live])                              # (m,4)
        x = np.einsum("mk,mkc->mc", N, Xl)
        dxi_w = 0.25 * QUAD_XI[:, 0] * (1 + QUAD_XI[:, 1] * eta[live][:, None])
        deta_w = 0.25 * QUAD_XI[:, 1] * (1 + QUAD_XI[:, 0] * xi[live][:, None])
        a, b = np.einsum("mk,mk->m", dxi_w, Xl[:, :, 0]), np.einsum("mk,mk->m", deta_w, Xl[:, :, 0])
        c, d = np.einsum("mk,mk->m", dxi_w, Xl[:, :, 1]), np.einsum("mk,mk->m", deta_w, Xl[:, :, 1])
        r = pts[live] - x
        det = a * d - b * c
        dxi = (d * r[:, 0] - b * r[:, 1]) / det
        deta = (-c * r[:, 0] + a * r[:, 1]) / det
        xi[live] += dxi
        eta[live] += deta
        live = live[np.abs(dxi) + np.abs(deta) >= tol]
    return xi, eta


def dual_mortar(slave_xy: np.ndarray, slave_faces: np.ndarray,
                master_origin, master_h, master_n):
    """Assemble D (diagonal, per slave node) and M (slave x master CSR).

    slave_xy (ns,2) in-plane slave node coordinates, slave_faces (nf,4) CCW corner ids;
    the master surface is the structured grid with origin (x0,y0), spacing (hx,hy),
    (mx, my) faces; master node (a,b) has id a + (mx+1) b.
    Returns D (ns,), M (scipy CSR ns x nm).

    Every (slave face, master face) pair with an overlap is clipped and triangulated first;
    the quadrature of all segments (inverse maps, dual basis, products) then runs batched.
    """
    x0, y0 = master_origin
    hx, hy = master_h
    mx, my = master_n
    ns = slave_xy.shape[0]
    nm = (mx + 1) * (my + 1)
    nf = slave_faces.shape[0]
    A_all = np.empty((nf, 4, 4))
    seg_face, seg_r0, seg_mids, seg_npts = [], [], [], []
    pts_all, wts_all = [], []
    for f in range(nf):
        ids = slave_faces[f]
        X = slave_xy[ids]
        if polygon_area(X) <= 0:
            raise ValueError("slave face is not counter-clockwise")
        A_all[f] = dual_coefficients(X)
        bx0, by0 = X.min(axis=0)
        bx1, by1 = X.max(axis=0)
        a0 = max(int(np.floor((bx0 - x0) / hx)) - 1, 0)
        a1 = min(int(np.floor((bx1 - x0) / hx)) + 1, mx - 1)
        b0 = max(int(np.floor((by0 - y0) / hy)) - 1, 0)
        b1 = min(int(np.floor((by1 - y0) / hy)) + 1, my - 1)
        for b in range(b0, b1 + 1):
            for a in range(a0, a1 + 1):
                rx0, rx1 = x0 + a * hx, x0 + (a + 1) * hx
                ry0, ry1 = y0 + b * hy, y0 + (b + 1) * hy
                P = clip_polygon_rect(X, rx0, rx1, ry0, ry1)
                if len(P) < 3 or polygon_area(P) <= 1e-14 * hx * hy:
                    continue
                c = P.mean(axis=0)
                npts = 0
                for t in range(len(P)):
                    p1, p2 = P[t], P[(t + 1) % len(P)]
                    area = 0.5 * ((p1[0] - c[0]) * (p2[1] - c[1]) - (p2[0] - c[0]) * (p1[1] - c[1]))
                    if area <= 0:
                        continue
                    pts_all.append(TRI7_BARY[:, 0:1] * c + TRI7_BARY[:, 1:2] * p1 + TRI7_BARY[:, 2:3] * p2)
                    wts_all.append(TRI7_W * area)
                    npts += TRI7_W.size
                seg_face.append(f)
                seg_r0.append((rx0, ry0))
                seg_mids.append((a + (mx + 1) * b, a + 1 + (mx + 1) * b, a + 1 + (mx + 1) * (b + 1),
                                 a + (mx + 1) * (b + 1)))
                seg_npts.append(npts)
    seg_face = np.asarray(seg_face, dtype=np.int64)
    seg_npts = np.asarray(seg_npts, dtype=np.int64)
    seg_r0 = np.asarray(seg_r0)
    seg_mids = np.asarray(seg_mids, dtype=np.int64)
    pts = np.concatenate(pts_all)
    wts = np.concatenate(wts_all)
    seg_of_pt = np.repeat(np.arange(seg_face.size), seg_npts)
    face_of_pt = seg_face[seg_of_pt]
    xi, eta = quad_inverse_map_batched(slave_xy[slave_faces[face_of_pt]], pts)
    psi = np.einsum("pk,pjk->pj", quad_N(xi, eta), A_all[face_of_pt])         # psi_j at the points
    r0 = seg_r0[seg_of_pt]
    Nm = quad_N(2.0 * (pts[:, 0] - r0[:, 0]) / hx - 1.0, 2.0 * (pts[:, 1] - r0[:, 1]) / hy - 1.0)
    pw = psi * wts[:, None]
    starts = np.concatenate([[0], np.cumsum(seg_npts)[:-1]])
    Mloc = np.add.reduceat(pw[:, :, None] * Nm[:, None, :], starts, axis=0)    # (nseg,4,4)
    D = np.zeros(ns)
    np.add.at(D, slave_faces[face_of_pt].ravel(), pw.ravel())
    rows = np.repeat(slave_faces[seg_face], 4, axis=1).ravel()
    cols = np.tile(seg_mids, (1, 4)).ravel()
    M = sp.coo_matrix((Mloc.reshape(-1), (rows, cols)), shape=(ns, nm)).tocsr()
    M.sum_duplicates()
    M.sort_indices()
    return D, M
