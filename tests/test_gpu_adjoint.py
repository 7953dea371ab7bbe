"""GPU adjoint path: transposed hierarchy, transposed solve and gradients (through the C-ABI)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle.amg import Options, setup as oracle_setup  # noqa: E402
from oracle.saddle import build_saddle  # noqa: E402
from paper_1912_09056_gb300 import amgc  # noqa: E402
from paper_1912_09056_gb300.adjoint import ElementTables, contact_gradients, objective_gradient, saddle_solve  # noqa: E402
from paper_1912_09056_gb300.problem import two_block_problem, workload  # noqa: E402

SMALL = dict(master_n=(7, 6, 6), slave_n=(6, 5, 5), E_slave=4.0, tilt_deg=5.0, seed=21, active_fraction=0.6,
             log_E_sigma=0.5)
OPTS = dict(levels_max=3, coarse_max_rows=0, transfer=1)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("opts", [dict(levels_max=3, coarse_max_rows=0, transfer=0),
                                  dict(levels_max=3, coarse_max_rows=0, transfer=1, smoother_sweeps=2),
                                  dict(levels_max=4, coarse_max_rows=200, transfer=1),
                                  dict(levels_max=3, coarse_max_rows=0, transfer=1, jacobi_sweeps=2),
                                  dict(levels_max=3, coarse_max_rows=0, transfer=0, smoother_sweeps=2,
                                       jacobi_sweeps=3)])
def test_transposed_cycle_and_apply(opts):
    prob = two_block_problem(**SMALL)
    h = amgc.setup(prob, **opts)
    rng = np.random.default_rng(0)
    x, y = rng.standard_normal((2, prob.n))
    xd, yd = _cuda(x), _cuda(y)
    Mx, MTy = torch.empty_like(xd), torch.empty_like(yd)
    h.vcycle(xd, Mx)
    h.vcycle_transposed(yd, MTy)
    ATx = torch.empty_like(xd)
    h.apply_transposed(xd, ATx)
    torch.cuda.synchronize()
    lhs = float(Mx.cpu().numpy() @ y)
    rhs = float(x @ MTy.cpu().numpy())
    scale = np.linalg.norm(Mx.cpu().numpy()) * np.linalg.norm(y)
    assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs)
    A = build_saddle(prob).full()
    assert np.abs(ATx.cpu().numpy() - A.T @ x).max() <= 1e-13 * np.abs(A.T @ x).max()
    # the transposed solve reaches its tolerance
    c = _cuda(rng.standard_normal(prob.n))
    adj = torch.zeros_like(c)
    it, rr, _ = h.solve_transposed(c, adj, tol=1e-10)
    r = c.cpu().numpy() - A.T @ adj.cpu().numpy()
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(c.cpu().numpy())
    h.close()


def _dense_reference(prob):
    """FP64 dense-LU solution, adjoint and element gradients (independent of the GPU path)."""
    e = prob.extra
    A = build_saddle(prob).full().tocsc()
    lu = spla.splu(A)
    x = lu.solve(prob.rhs)
    n_u = prob.n_u
    c = np.zeros_like(x)
    act = np.nonzero(prob.active)[0]
    c[n_u:].reshape(-1, 3)[act] = prob.triad[act, 0]
    mn = prob.master_node
    c[:n_u].reshape(-1, 3)[mn] = x[:n_u].reshape(-1, 3)[mn]
    adj = spla.splu(A.T.tocsc()).solve(c)
    nf = e["node_free"]
    conn = e["conn"]
    ufull = e["u_D"].copy()
    afull = np.zeros_like(ufull)
    free = nf >= 0
    ufull[free] = x[:n_u].reshape(-1, 3)[nf[free]]
    afull[free] = adj[:n_u].reshape(-1, 3)[nf[free]]
    ue = ufull[conn].reshape(-1, 24)
    ae = afull[conn].reshape(-1, 24)
    Kh = e["Khat"][e["elem_shape"]]
    gE = -np.einsum("ei,eij,ej->e", ae, Kh, ue)
    Ka = np.einsum("eij,ej->ei", Kh, ae).reshape(-1, 8, 3)
    top = e["top_mask"][conn].astype(bool)
    gt = -(e["E_elem"][:, None, None] * Ka * top[:, :, None]).sum(axis=(0, 1))
    J = float(prob.triad[act, 0].ravel() @ x[n_u:].reshape(-1, 3)[act].ravel()) + \
        0.5 * float((x[:n_u].reshape(-1, 3)[mn] ** 2).sum())
    return J, gE, gt


def _gpu_J(prob, tol=1e-12):
    h = amgc.setup(prob, tol=tol, **OPTS)
    b = _cuda(prob.rhs)
    x = torch.zeros_like(b)
    h.solve(b, x)
    J, _ = objective_gradient(prob, x)
    h.close()
    return float(J)


def test_element_gradients_match_dense_reference_and_finite_differences():
    prob = two_block_problem(keep_full=True, **SMALL)
    tables = ElementTables(prob)
    h = amgc.setup(prob, tol=1e-12, **OPTS)
    b = _cuda(prob.rhs)
    x = torch.zeros_like(b)
    h.solve(b, x)
    J, gE, gt, adj, it = contact_gradients(prob, h, x, tables, adj_tol=1e-12)
    gE = gE.cpu().numpy()
    gt = gt.cpu().numpy()
    Jr, gEr, gtr = _dense_reference(prob)
    assert abs(float(J) - Jr) <= 1e-9 * abs(Jr)
    assert np.abs(gE - gEr).max() <= 1e-8 * np.abs(gEr).max()
    assert np.abs(gt - gtr).max() <= 1e-8 * np.abs(gtr).max()
    # central finite differences along 20 seeded directions of the modulus field
    E0 = prob.extra["E_elem"]
    rng = np.random.default_rng(40)
    kw = dict(SMALL)
    kw.pop("log_E_sigma")
    for k in range(20):
        d = rng.standard_normal(E0.size) * E0
        hstep = 1e-4
        Jp = _gpu_J(two_block_problem(E_elem=E0 + hstep * d, **kw))
        Jm = _gpu_J(two_block_problem(E_elem=E0 - hstep * d, **kw))
        fd = (Jp - Jm) / (2 * hstep)
        an = float(gE @ d)
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-12 * abs(Jr)), (k, fd, an)
    # and along the three components of the prescribed top displacement (global frame)
    R = prob.extra["R"]
    t0 = prob.extra["top_disp"]
    for cidx in range(3):
        e_c = np.zeros(3)
        e_c[cidx] = 1.0
        hstep = 1e-5
        Jp = _gpu_J(two_block_problem(E_elem=E0, top_disp=t0 + hstep * (R.T @ e_c), **kw))
        Jm = _gpu_J(two_block_problem(E_elem=E0, top_disp=t0 - hstep * (R.T @ e_c), **kw))
        fd = (Jp - Jm) / (2 * hstep)
        assert abs(fd - gt[cidx]) <= 1e-6 * np.abs(gt).max(), (cidx, fd, gt[cidx])
    h.close()


def test_autograd_function_matches_finite_differences():
    prob = two_block_problem(**SMALL)
    K = _cuda(prob.K_val).requires_grad_(True)
    b = _cuda(prob.rhs).requires_grad_(True)
    opts = amgc.default_options(tol=1e-12, **OPTS)
    x = saddle_solve(K, b, prob, opts, adj_tol=1e-12)
    J, _ = objective_gradient(prob, x)
    J.backward()
    rng = np.random.default_rng(7)
    # symmetric perturbation of the stored K values (same pattern), and of the right-hand side
    D = rng.standard_normal(prob.K_val.shape) * np.abs(prob.K_val).max() * 1e-2
    db = rng.standard_normal(prob.n) * np.abs(prob.rhs).max()
    hstep = 1e-5

    def Jof(Kv, bv):
        with torch.no_grad():
            xx = saddle_solve(_cuda(Kv), _cuda(bv), prob, opts)
            return float(objective_gradient(prob, xx)[0])
    fdK = (Jof(prob.K_val + hstep * D, prob.rhs) - Jof(prob.K_val - hstep * D, prob.rhs)) / (2 * hstep)
    anK = float((K.grad.cpu().numpy() * D).sum())
    assert abs(fdK - anK) <= 1e-6 * abs(anK), (fdK, anK)
    fdb = (Jof(prob.K_val, prob.rhs + hstep * db) - Jof(prob.K_val, prob.rhs - hstep * db)) / (2 * hstep)
    anb = float(b.grad.cpu().numpy() @ db)
    assert abs(fdb - anb) <= 1e-6 * abs(anb), (fdb, anb)


def test_transposed_cycle_refuses_other_smoothers_and_preconditioners():
    prob = workload(0)
    h = amgc.setup(prob, levels_max=3, coarse_max_rows=0)
    r = _cuda(np.ones(prob.n))
    z = torch.empty_like(r)
    h.set_smoother("uzawa")
    with pytest.raises(amgc.AmgcError) as e:
        h.vcycle_transposed(r, z)
    assert e.value.code == amgc.AMGC_EINVAL
    h.set_smoother("cheap_simple")
    h.vcycle_transposed(r, z)
    h.close()
