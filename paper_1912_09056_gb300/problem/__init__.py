"""Seeded synthetic inputs: two-block frictionless mortar-contact saddle-point systems.

These generators build the linearised system of Sec. 2.3 (Eq. ch6_finalsaddlepointsystem)
for two hex8 bricks in linear elasticity touching on a flat, possibly tilted interface:
the stiffness block K, the dual-mortar matrices D and M, the slave-node triads, the
active set, the rigid-body nullspace and the right-hand side.  Nothing in here is part
of the multigrid method; both the CUDA library and the oracle consume these arrays.

Random draws use NumPy's PCG64 generator (``numpy.random.default_rng(seed)``).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from .fe import assemble_bsr, brick_mesh
from .mortar import dual_mortar


@dataclass
class ContactProblem:
    """One linearised contact system with fully prescribed nodes eliminated."""
    name: str
    n_nodes: int                 # free displacement nodes = block rows of K
    K_rowptr: np.ndarray         # int32 (n_nodes+1)
    K_col: np.ndarray            # int32 (nnzb)
    K_val: np.ndarray            # float64 (nnzb,3,3), row-major blocks
    body_id: np.ndarray          # int32 (n_nodes): 0 = master body, 1 = slave body
    coords: np.ndarray           # float64 (n_nodes,3), current (tilted) coordinates
    nullspace: np.ndarray        # float64 (3 n_nodes, 6): t_x t_y t_z r_x r_y r_z
    slave_node: np.ndarray       # int32 (n_s): slave interface node -> K block row
    master_node: np.ndarray      # int32 (n_m): master interface node -> K block row
    D: np.ndarray                # float64 (n_s): diagonal dual-mortar matrix
    M_rowptr: np.ndarray         # int32 (n_s+1)  M is n_s x n_m
    M_col: np.ndarray            # int32
    M_val: np.ndarray            # float64
    triad: np.ndarray            # float64 (n_s,3,3): rows n, tau_xi, tau_eta
    active: np.ndarray           # uint8 (n_s)
    f: np.ndarray                # float64 (3 n_nodes): lifted displacement rhs
    g: np.ndarray                # float64 (3 n_s): constraint rhs (weighted gap, 0 here)
    extra: dict = field(default_factory=dict)

    @property
    def n_u(self) -> int:
        return 3 * self.n_nodes

    @property
    def n_s(self) -> int:
        return int(self.D.shape[0])

    @property
    def n_lam(self) -> int:
        return 3 * self.n_s

    @property
    def n(self) -> int:
        return self.n_u + self.n_lam

    @property
    def rhs(self) -> np.ndarray:
        return np.concatenate([self.f, self.g])


def rotation_x(deg: float) -> np.ndarray:
    t = np.deg2rad(deg)
    c, s = np.cos(t), np.sin(t)
    return np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])


def rigid_body_modes(coords: np.ndarray) -> np.ndarray:
    """Six rigid-body modes at the given nodes, rotations about the nodes' centroid."""
    d = coords - coords.mean(axis=0)
    n = coords.shape[0]
    B = np.zeros((n, 3, 6))
    B[:, 0, 0] = 1.0
    B[:, 1, 1] = 1.0
    B[:, 2, 2] = 1.0
    # r_x = e_x x d, r_y = e_y x d, r_z = e_z x d
    B[:, 1, 3] = -d[:, 2]; B[:, 2, 3] = d[:, 1]
    B[:, 0, 4] = d[:, 2];  B[:, 2, 4] = -d[:, 0]
    B[:, 0, 5] = -d[:, 1]; B[:, 1, 5] = d[:, 0]
    return B.reshape(3 * n, 6)


def two_block_problem(name: str = "two_block",
                      master_n=(8, 8, 8), slave_n=(7, 7, 7),
                      master_box=((0.0, 0.0, 0.0), (1.0, 1.0, 1.0)),
                      slave_box=((0.0, 0.0, 1.0), (1.0, 1.0, 2.0)),
                      E_master: float = 1.0, E_slave: float = 1.0,
                      nu_master: float = 0.3, nu_slave: float = 0.3,
                      tilt_deg: float = 0.0, jitter: float = 0.2, seed: int = 0,
                      active_fraction: float = 1.0, top_disp=(0.0, 0.0, -0.01),
                      log_E_sigma: float = 0.0, E_elem: Optional[np.ndarray] = None,
                      keep_full: bool = False) -> ContactProblem:
    """Master brick below, slave brick on top, touching on the plane z = master top.

    Bottom face of the master is clamped, the slave's top face is moved by top_disp
    (all three components prescribed).  Interior slave-interface nodes are jittered
    in-plane by U(+-jitter*h), edge nodes only along their edge, corners not at all.
    The whole model is then rotated about the x-axis through the interface centre.
    E_elem, if given, replaces the moduli of all elements (master elements first).
    """
    rng = np.random.default_rng(seed)
    mx, my, mz = master_n
    sx, sy, sz = slave_n
    cm, conn_m, ijk_m = brick_mesh(mx, my, mz, master_box[0], master_box[1])
    cs, conn_s, ijk_s = brick_mesh(sx, sy, sz, slave_box[0], slave_box[1])
    if abs(master_box[1][2] - slave_box[0][2]) > 1e-14:
        raise ValueError("bricks must touch")
    nm_nodes = cm.shape[0]
    # in-plane jitter of the slave interface nodes
    hx = (slave_box[1][0] - slave_box[0][0]) / sx
    hy = (slave_box[1][1] - slave_box[0][1]) / sy
    iface_s = np.nonzero(ijk_s[:, 2] == 0)[0]
    if jitter > 0:
        i, j = ijk_s[iface_s, 0], ijk_s[iface_s, 1]
        dx = rng.uniform(-jitter * hx, jitter * hx, size=iface_s.size)
        dy = rng.uniform(-jitter * hy, jitter * hy, size=iface_s.size)
        dx[(i == 0) | (i == sx)] = 0.0
        dy[(j == 0) | (j == sy)] = 0.0
        cs[iface_s, 0] += dx
        cs[iface_s, 1] += dy
    coords = np.concatenate([cm, cs])
    conn_s_g = conn_s + nm_nodes
    # interface in-plane data (before rotation)
    iface_m = np.nonzero(ijk_m[:, 2] == mz)[0]
    slave_xy = cs[iface_s, :2].copy()
    fi, fj = np.meshgrid(np.arange(sx), np.arange(sy), indexing="xy")
    fi = fi.ravel(); fj = fj.ravel()
    faces = np.stack([fi + (sx + 1) * fj, fi + 1 + (sx + 1) * fj,
                      fi + 1 + (sx + 1) * (fj + 1), fi + (sx + 1) * (fj + 1)], axis=1)
    hmx = (master_box[1][0] - master_box[0][0]) / mx
    hmy = (master_box[1][1] - master_box[0][1]) / my
    D, M = dual_mortar(slave_xy, faces, (master_box[0][0], master_box[0][1]), (hmx, hmy), (mx, my))
    # active set: all, or the nodes nearest to a jittered interface centre
    ns = iface_s.size
    if active_fraction >= 1.0:
        active = np.ones(ns, dtype=np.uint8)
    else:
        c0 = np.array([0.5 * (slave_box[0][0] + slave_box[1][0]), 0.5 * (slave_box[0][1] + slave_box[1][1])])
        c0 = c0 + rng.uniform(-0.05, 0.05, size=2)
        dist = np.hypot(slave_xy[:, 0] - c0[0], slave_xy[:, 1] - c0[1])
        order = np.lexsort((np.arange(ns), dist))
        n_act = int(round(active_fraction * ns))
        active = np.zeros(ns, dtype=np.uint8)
        active[order[:n_act]] = 1
    # material field
    E_m = np.full(conn_m.shape[0], E_master)
    E_s = np.full(conn_s.shape[0], E_slave)
    if log_E_sigma > 0:
        E_m *= np.exp(rng.normal(0.0, log_E_sigma, size=E_m.size))
        E_s *= np.exp(rng.normal(0.0, log_E_sigma, size=E_s.size))
    if E_elem is not None:
        E_elem = np.asarray(E_elem, dtype=np.float64)
        E_m = E_elem[:conn_m.shape[0]].copy()
        E_s = E_elem[conn_m.shape[0]:].copy()
    # rigid rotation about the x-axis through the interface centre
    R = rotation_x(tilt_deg)
    ctr = np.array([0.5 * (master_box[0][0] + master_box[1][0]),
                    0.5 * (master_box[0][1] + master_box[1][1]), master_box[1][2]])
    coords = (coords - ctr) @ R.T + ctr
    n_all = coords.shape[0]
    # stiffness of both bodies (no coupling between them)
    rp_m, col_m, val_m = assemble_bsr(coords[:nm_nodes], conn_m, E_m, nu_master, nm_nodes)
    rp_s, col_s, val_s = assemble_bsr(coords[nm_nodes:], conn_s, E_s, nu_slave, n_all - nm_nodes)
    rowptr = np.concatenate([rp_m, rp_s[1:] + rp_m[-1]])
    col = np.concatenate([col_m, col_s + nm_nodes])
    val = np.concatenate([val_m, val_s])
    # Dirichlet data
    u_D = np.zeros((n_all, 3))
    presc = np.zeros(n_all, dtype=bool)
    bot = np.nonzero(ijk_m[:, 2] == 0)[0]
    top = np.nonzero(ijk_s[:, 2] == sz)[0] + nm_nodes
    presc[bot] = True
    presc[top] = True
    u_D[top] = R @ np.asarray(top_disp, dtype=np.float64)
    free = np.nonzero(~presc)[0]
    newid = -np.ones(n_all, dtype=np.int64)
    newid[free] = np.arange(free.size)
    rows_all = np.repeat(np.arange(n_all), np.diff(rowptr))
    keep = (~presc[rows_all]) & (~presc[col])
    lift = (~presc[rows_all]) & presc[col]
    f = np.zeros((n_all, 3))
    np.add.at(f, rows_all[lift], -np.einsum("bij,bj->bi", val[lift], u_D[col[lift]]))
    f = f[free].ravel()
    # lifting map of a uniform top displacement t given in the unrotated frame: f = L t
    top_lift = np.zeros((n_all, 3, 3))
    on_top = presc[col] & (col >= nm_nodes) & lift
    blk = val[on_top] @ R                                     # K_fD (R e_c) per block
    np.add.at(top_lift, rows_all[on_top], -blk)
    top_lift = top_lift[free].reshape(-1, 3)
    kr = newid[rows_all[keep]]
    kc = newid[col[keep]]
    K_val = val[keep]
    K_rowptr = np.zeros(free.size + 1, dtype=np.int64)
    np.add.at(K_rowptr, kr + 1, 1)
    K_rowptr = np.cumsum(K_rowptr)
    body = np.zeros(n_all, dtype=np.int32)
    body[nm_nodes:] = 1
    slave_node = newid[iface_s + nm_nodes]
    master_node = newid[iface_m]
    if np.any(slave_node < 0) or np.any(master_node < 0):
        raise ValueError("interface node is prescribed")
    n_vec = R @ np.array([0.0, 0.0, -1.0])
    t1 = R @ np.array([1.0, 0.0, 0.0])
    t2 = R @ np.array([0.0, 1.0, 0.0])
    triad = np.broadcast_to(np.stack([n_vec, t1, t2]), (ns, 3, 3)).copy()
    extra = dict(tilt_deg=tilt_deg, R=R, n_all_nodes=n_all, n_dofs_total=3 * n_all, top_lift=top_lift,
                 n_elements=conn_m.shape[0] + conn_s.shape[0])
    if keep_full:
        from .fe import element_shapes
        sh_m, Kh_m = element_shapes(coords[:nm_nodes], conn_m, nu_master)
        sh_s, Kh_s = element_shapes(coords[nm_nodes:], conn_s, nu_slave)
        node_free = newid.astype(np.int32)
        top_mask = np.zeros(n_all, dtype=np.uint8)
        top_mask[top] = 1
        extra.update(elem_shape=np.concatenate([sh_m, sh_s + Kh_m.shape[0]]).astype(np.int32),
                     Khat=np.concatenate([Kh_m, Kh_s]), node_free=node_free, top_mask=top_mask,
                     top_disp=np.asarray(top_disp, dtype=np.float64))
        extra.update(full_rowptr=rowptr, full_col=col, full_val=val, full_coords=coords,
                     prescribed=presc, u_D=u_D, free=free, body_all=body,
                     conn=np.concatenate([conn_m, conn_s_g]), E_elem=np.concatenate([E_m, E_s]),
                     nu_elem=np.concatenate([np.full(E_m.size, nu_master), np.full(E_s.size, nu_slave)]),
                     iface_slave_all=iface_s + nm_nodes, iface_master_all=iface_m,
                     ijk_m=ijk_m, ijk_s=ijk_s)
    return ContactProblem(
        name=name, n_nodes=int(free.size),
        K_rowptr=K_rowptr.astype(np.int32), K_col=kc.astype(np.int32), K_val=np.ascontiguousarray(K_val),
        body_id=body[free].astype(np.int32), coords=coords[free].copy(),
        nullspace=rigid_body_modes(coords[free]),
        slave_node=slave_node.astype(np.int32), master_node=master_node.astype(np.int32),
        D=D, M_rowptr=M.indptr.astype(np.int32), M_col=M.indices.astype(np.int32),
        M_val=M.data.astype(np.float64), triad=triad, active=active,
        f=f, g=np.zeros(3 * ns), extra=extra)


# The five synthetic workloads.  Sizes follow the workload descriptions: config 0 is the
# tiny case, 1 the medium SA case, 2 the large FP32-vs-FP64 case, 3 the batched set and
# 4 the adjoint case.
WORKLOADS = {
    0: dict(name="tiny_8x8x8_7x7x7", master_n=(8, 8, 8), slave_n=(7, 7, 7), seed=0),
    1: dict(name="medium_48^3_41^3", master_n=(48, 48, 48), slave_n=(41, 41, 41), E_master=1.0,
            E_slave=10.0, tilt_deg=5.0, seed=1, active_fraction=0.6),
    2: dict(name="large_110x110x55_97x97x49", master_n=(110, 110, 55), slave_n=(97, 97, 49),
            master_box=((0.0, 0.0, 0.0), (1.0, 1.0, 0.5)), slave_box=((0.1, 0.1, 0.5), (0.9, 0.9, 0.9)),
            E_master=1.0, E_slave=100.0, nu_master=0.3, nu_slave=0.45, seed=2),
    4: dict(name="adjoint_58^3_50^3", master_n=(58, 58, 58), slave_n=(50, 50, 50), E_master=1.0,
            E_slave=10.0, tilt_deg=5.0, seed=4, active_fraction=0.6, log_E_sigma=0.5),
}


def workload(cfg: int, keep_full: bool = False, **overrides) -> ContactProblem:
    kw = dict(WORKLOADS[cfg])
    kw.update(overrides)
    return two_block_problem(keep_full=keep_full, **kw)


def batched_workloads(count: int = 64, seed: int = 3, lo: int = 8, hi: int = 32, scale: Optional[float] = None):
    """Instance parameters of the batched set: uneven bricks, random material/tilt/active set."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        nmst = int(rng.integers(lo, hi + 1))
        nslv = int(rng.integers(lo, hi + 1))
        out.append(dict(name=f"batch_{b}", master_n=(nmst,) * 3, slave_n=(nslv,) * 3,
                        E_master=1.0, E_slave=float(rng.uniform(1.0, 100.0)),
                        nu_master=float(rng.uniform(0.2, 0.45)), nu_slave=float(rng.uniform(0.2, 0.45)),
                        tilt_deg=float(rng.uniform(0.0, 10.0)), active_fraction=float(rng.uniform(0.3, 1.0)),
                        seed=int(rng.integers(0, 2**31 - 1)),
                        top_amps=rng.uniform(-0.02, 0.0, size=4).tolist()))
    return out


def concat_problems(probs, name: str = "batch"):
    """Block-diagonal concatenation of independent problems (K rows, slave and master nodes).

    Returns (problem, node_ptr, lm_ptr): instance q owns K block rows [node_ptr[q],
    node_ptr[q+1]) and slave / multiplier nodes [lm_ptr[q], lm_ptr[q+1]).  Bodies of instance q
    get ids 2q and 2q + 1.
    """
    node_ptr = np.cumsum([0] + [p.n_nodes for p in probs]).astype(np.int32)
    lm_ptr = np.cumsum([0] + [p.n_s for p in probs]).astype(np.int32)
    m_ptr = np.cumsum([0] + [p.master_node.size for p in probs])
    kptr = np.cumsum([0] + [p.K_col.size for p in probs])
    mnz = np.cumsum([0] + [p.M_col.size for p in probs])
    K_rowptr = np.concatenate([probs[0].K_rowptr[:1]] + [p.K_rowptr[1:] + kptr[q] for q, p in enumerate(probs)])
    M_rowptr = np.concatenate([probs[0].M_rowptr[:1]] + [p.M_rowptr[1:] + mnz[q] for q, p in enumerate(probs)])
    cat = ContactProblem(
        name=name, n_nodes=int(node_ptr[-1]),
        K_rowptr=K_rowptr.astype(np.int32),
        K_col=np.concatenate([p.K_col + node_ptr[q] for q, p in enumerate(probs)]).astype(np.int32),
        K_val=np.concatenate([p.K_val for p in probs]),
        body_id=np.concatenate([p.body_id + 2 * q for q, p in enumerate(probs)]).astype(np.int32),
        coords=np.concatenate([p.coords for p in probs]),
        nullspace=np.concatenate([p.nullspace for p in probs]),
        slave_node=np.concatenate([p.slave_node + node_ptr[q] for q, p in enumerate(probs)]).astype(np.int32),
        master_node=np.concatenate([p.master_node + node_ptr[q] for q, p in enumerate(probs)]).astype(np.int32),
        D=np.concatenate([p.D for p in probs]),
        M_rowptr=M_rowptr.astype(np.int32),
        M_col=np.concatenate([p.M_col + m_ptr[q] for q, p in enumerate(probs)]).astype(np.int32),
        M_val=np.concatenate([p.M_val for p in probs]),
        triad=np.concatenate([p.triad for p in probs]),
        active=np.concatenate([p.active for p in probs]),
        f=np.concatenate([p.f for p in probs]),
        g=np.concatenate([p.g for p in probs]),
        extra=dict(n_inst=len(probs)))
    return cat, node_ptr, lm_ptr


# prescribed-displacement patterns of the batched workload (unrotated frame, scaled by the
# instance's seeded amplitudes): compression, and compression with x, y and diagonal shear
BATCH_PATTERNS = np.array([[0.0, 0.0, 1.0], [0.3, 0.0, 1.0], [0.0, 0.3, 1.0], [0.3, 0.3, 1.0]])


def batched_rhs(probs, params, cat, node_ptr, lm_ptr):
    """(nrhs, rows) right-hand sides: per instance f = L (a_k d_k), g = 0, in the concatenated order."""
    n_u = cat.n_u
    nrhs = BATCH_PATTERNS.shape[0]
    out = np.zeros((nrhs, cat.n))
    for q, (p, prm) in enumerate(zip(probs, params)):
        L = p.extra["top_lift"]
        for k in range(nrhs):
            out[k, 3 * node_ptr[q]:3 * node_ptr[q + 1]] = L @ (prm["top_amps"][k] * BATCH_PATTERNS[k])
    return out


def batched_workload(count: int = 64, seed: int = 3, lo: int = 8, hi: int = 32):
    """The batched set: `count` uneven instances, concatenated, with four right-hand sides each."""
    params = batched_workloads(count, seed, lo, hi)
    probs = []
    for prm in params:
        kw = {k: v for k, v in prm.items() if k != "top_amps"}
        probs.append(two_block_problem(**kw))
    cat, node_ptr, lm_ptr = concat_problems(probs)
    return cat, node_ptr, lm_ptr, batched_rhs(probs, params, cat, node_ptr, lm_ptr), probs, params
