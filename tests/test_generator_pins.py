"""Pins of the seeded input generator against facts the paper and the mechanics fix."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from paper_1912_09056_gb300.problem import rigid_body_modes, two_block_problem, workload
from paper_1912_09056_gb300.problem.fe import brick_mesh
from paper_1912_09056_gb300.problem.mortar import dual_mortar

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _full_K(p):
    e = p.extra
    n = e["n_all_nodes"]
    rows = np.repeat(np.arange(n), np.diff(e["full_rowptr"]))
    br = (rows[:, None, None] * 3 + np.arange(3)[None, :, None]) + 0 * np.arange(3)[None, None, :]
    bc = (e["full_col"][:, None, None] * 3 + np.arange(3)[None, None, :]) + 0 * np.arange(3)[None, :, None]
    return sp.csr_matrix((e["full_val"].ravel(), (br.ravel(), bc.ravel())), shape=(3 * n, 3 * n))


def test_weak_scaling_dof_counts_match_paper_table():
    """Table ScalingStudyMeshRefinement: DOF counts of the 2k x 2k x k brick family."""
    rows = np.loadtxt(os.path.join(GOLDEN, "weak_scaling_dofs.txt"), dtype=np.int64)
    for k, nu, nl, nt in rows:
        cm, _, _ = brick_mesh(2 * k, 2 * k, k, (0, 0, 0), (1, 1, 0.5))
        cs, _, ijk = brick_mesh(2 * k, 2 * k, k, (0.1, 0.1, 0.5), (0.9, 0.9, 0.9))
        n_iface = int(np.sum(ijk[:, 2] == 0))
        assert 3 * (cm.shape[0] + cs.shape[0]) == nu
        assert 3 * n_iface == nl
        assert nu + nl == nt
    # full generation of the smallest member
    k = 20
    p = two_block_problem(master_n=(2 * k, 2 * k, k), slave_n=(2 * k, 2 * k, k),
                          master_box=((0, 0, 0), (1, 1, 0.5)), slave_box=((0.1, 0.1, 0.5), (0.9, 0.9, 0.9)),
                          jitter=0.0)
    assert p.extra["n_dofs_total"] == rows[0, 1]
    assert p.n_lam == rows[0, 2]
    assert abs(p.D.sum() - 0.64) < 1e-12          # slave interface area 0.8 x 0.8


def test_workload_sizes():
    p = workload(0)
    assert p.n_u == 3288 and p.n_lam == 192 and p.extra["n_dofs_total"] == 3723


def test_stiffness_symmetric_and_rigid_modes(cfg0):
    K = _full_K(cfg0)
    assert abs(K - K.T).max() <= 1e-14 * abs(K).max()
    coords = cfg0.extra["full_coords"]
    body = cfg0.extra["body_all"]
    for b in (0, 1):
        sel = body == b
        B = rigid_body_modes(coords[sel])
        Bf = np.zeros((3 * coords.shape[0], 6))
        idx = (np.nonzero(sel)[0][:, None] * 3 + np.arange(3)).ravel()
        Bf[idx] = B
        assert np.abs(K @ Bf).max() <= 1e-12 * abs(K).max()
    # a stretch is not a null mode
    u = np.zeros(3 * coords.shape[0]); u[0::3] = coords[:, 0]
    assert np.abs(K @ u).max() > 1e-3 * abs(K).max()


def test_mortar_patch_condition(cfg0):
    """Row sums of M equal the diagonal of D under dual shape functions (non-matching, jittered)."""
    rs = np.add.reduceat(cfg0.M_val, cfg0.M_rowptr[:-1])
    assert np.abs(rs - cfg0.D).max() <= 1e-13 * cfg0.D.max()
    assert abs(cfg0.D.sum() - 1.0) <= 1e-13


def _grid(n, jitter=0.0, seed=0):
    x = np.linspace(0, 1, n + 1)
    X, Y = np.meshgrid(x, x, indexing="xy")
    xy = np.stack([X.ravel(), Y.ravel()], 1)
    rng = np.random.default_rng(seed)
    if jitter:
        i = np.tile(np.arange(n + 1), n + 1); j = np.repeat(np.arange(n + 1), n + 1)
        d = rng.uniform(-jitter / n, jitter / n, size=xy.shape)
        d[(i == 0) | (i == n), 0] = 0; d[(j == 0) | (j == n), 1] = 0
        xy = xy + d
    fi, fj = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    fi = fi.ravel(); fj = fj.ravel()
    faces = np.stack([fi + (n + 1) * fj, fi + 1 + (n + 1) * fj, fi + 1 + (n + 1) * (fj + 1), fi + (n + 1) * (fj + 1)], 1)
    return xy, faces


def test_mortar_matching_meshes_give_M_equal_D():
    """Coincident slave and master grids: biorthogonality makes M = diag(D) exactly."""
    xy, faces = _grid(5)
    D, M = dual_mortar(xy, faces, (0.0, 0.0), (0.2, 0.2), (5, 5))
    Md = M.toarray()
    assert np.abs(Md - np.diag(D)).max() <= 1e-14
    # D_jj = integral of N_j: h^2/4 per adjacent face
    i = np.tile(np.arange(6), 6); j = np.repeat(np.arange(6), 6)
    nfaces = (np.where((i == 0) | (i == 5), 1, 2) * np.where((j == 0) | (j == 5), 1, 2))
    assert np.abs(D - nfaces * 0.04 / 4).max() <= 1e-15


def test_mortar_D_equals_integral_of_N_for_jittered_faces():
    """D_jj = int psi_j = int N_j (biorthogonality), up to the segment quadrature error."""
    from paper_1912_09056_gb300.problem.mortar import quad_map, quad_N
    xy, faces = _grid(6, jitter=0.2, seed=3)
    D, M = dual_mortar(xy, faces, (0.0, 0.0), (1 / 7, 1 / 7), (7, 7))
    g = np.array([-np.sqrt(0.6), 0, np.sqrt(0.6)]); w = np.array([5, 8, 5]) / 9
    xi, eta = np.meshgrid(g, g, indexing="ij"); ww = np.outer(w, w).ravel()
    ref = np.zeros(xy.shape[0])
    for f in faces:
        _, J = quad_map(xy[f], xi.ravel(), eta.ravel())
        det = J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
        ref[f] += quad_N(xi.ravel(), eta.ravel()).T @ (ww * det)
    # the integrand psi_j(xi(x)) is not polynomial on a distorted face: degree-5 rule error
    assert np.abs(D - ref).max() <= 1e-5 * ref.max()
    assert np.abs(np.asarray(M.sum(axis=1)).ravel() - D).max() <= 1e-14


def test_uniaxial_contact_patch_is_reproduced():
    """Uniaxial compression through a non-matching, jittered, tilted interface.

    With the exact linear solution prescribed on the outer faces, the discrete saddle
    system must return that field and a constant contact pressure lambda_j = p n
    (Sec. 2.3 system; linear fields are reproduced by hex8 and by dual mortar).
    """
    from oracle.saddle import build_saddle
    p = two_block_problem(master_n=(4, 4, 3), slave_n=(3, 3, 3), tilt_deg=5.0, jitter=0.2, seed=7,
                          E_master=1.0, E_slave=3.0, nu_master=0.3, nu_slave=0.25, keep_full=True)
    e = p.extra
    R = e["R"]
    n = R @ np.array([0.0, 0.0, -1.0])
    c = (np.array([0.5, 0.5, 1.0]))                  # interface centre (rotation centre)
    pres = 0.02

    def strain(E, nu):
        return (-pres / E) * ((1 + nu) * np.outer(n, n) - nu * np.eye(3))
    X = e["full_coords"]
    body = e["body_all"]
    eps = np.where(body[:, None, None] == 0, strain(1.0, 0.3)[None], strain(3.0, 0.25)[None])
    u_ex = np.einsum("nij,nj->ni", eps, X - c)
    # assemble the unreduced saddle system and impose u_ex on the outer faces
    K = _full_K(p)
    presc = e["prescribed"]
    free = np.nonzero(~presc)[0]
    fd = (free[:, None] * 3 + np.arange(3)).ravel()
    pd = (np.nonzero(presc)[0][:, None] * 3 + np.arange(3)).ravel()
    f = -K[fd][:, pd] @ u_ex.ravel()[pd]
    S = build_saddle(p)
    A = S.full().toarray()
    b = np.concatenate([f, p.g])
    x = np.linalg.solve(A, b)
    u = x[:p.n_u].reshape(-1, 3)
    lam = x[p.n_u:].reshape(-1, 3)
    assert np.abs(u - u_ex[free]).max() <= 1e-6 * np.abs(u_ex).max()
    assert np.abs(lam - pres * n[None, :]).max() <= 1e-5 * pres
    # without jitter the reproduction is exact to rounding
    p2 = two_block_problem(master_n=(4, 4, 3), slave_n=(3, 3, 3), tilt_deg=5.0, jitter=0.0,
                           E_master=1.0, E_slave=3.0, nu_master=0.3, nu_slave=0.25, keep_full=True)
    K2 = _full_K(p2)
    X2 = p2.extra["full_coords"]
    u_ex2 = np.einsum("nij,nj->ni", eps, X2 - c)
    f2 = -K2[fd][:, pd] @ u_ex2.ravel()[pd]
    x2 = np.linalg.solve(build_saddle(p2).full().toarray(), np.concatenate([f2, p2.g]))
    assert np.abs(x2[:p2.n_u].reshape(-1, 3) - u_ex2[free]).max() <= 1e-12
    assert np.abs(x2[p2.n_u:].reshape(-1, 3) - pres * n[None, :]).max() <= 1e-11
