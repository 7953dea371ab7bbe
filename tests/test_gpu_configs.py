"""Full-size cases of the large, batched and adjoint workloads (3.5 M rows; 64 instances x 4
right-hand sides; 1.0 M rows): properties that hold at any size, and outputs sampled where
their definition can be evaluated one by one on the host."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1912_09056_gb300 import amgc  # noqa: E402
from paper_1912_09056_gb300.adjoint import ElementTables, contact_gradients  # noqa: E402
from paper_1912_09056_gb300.problem import batched_workload, workload  # noqa: E402


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _true_relres(h, b, x, transposed=False):
    y = torch.empty_like(b)
    (h.apply_transposed if transposed else h.apply)(x, y)
    return (torch.linalg.norm(b - y) / torch.linalg.norm(b)).item()


def _check_aggregates(h, prob):
    """Level 0: every node in exactly one non-empty aggregate, no aggregate across bodies, and
    multiplier aggregates aligned with the slave-side displacement aggregates (Algorithm 1)."""
    st = h.stats()
    agg = h.export(0, "agg").astype(np.int64)
    n_agg = st["disp_nodes"][1]
    assert agg.size == prob.n_nodes and agg.min() >= 0 and agg.max() == n_agg - 1
    assert np.unique(agg).size == n_agg
    body = np.asarray(prob.body_id)
    lo = np.full(n_agg, np.iinfo(np.int64).max)
    hi = np.full(n_agg, -1)
    np.minimum.at(lo, agg, body)
    np.maximum.at(hi, agg, body)
    assert np.array_equal(lo, hi), "an aggregate spans two bodies"
    lagg = h.export(0, "lagg").astype(np.int64)
    n_lagg = st["lm_nodes"][1]
    assert lagg.size == prob.n_s and lagg.min() >= 0 and lagg.max() == n_lagg - 1
    dagg = agg[np.asarray(prob.slave_node)]
    first = np.full(n_lagg, -1)
    first[lagg] = dagg
    assert np.array_equal(first[lagg], dagg), "a multiplier aggregate mixes displacement aggregates"
    assert np.unique(first).size == n_lagg, "two multiplier aggregates share a displacement aggregate"


def test_large_fp32_and_fp64_cycles_reach_the_tolerance_and_agree(large_problem):
    prob = large_problem
    opts = dict(levels_max=4, coarse_max_rows=0, transfer=1, smoother_sweeps=3)
    b = _cuda(prob.rhs)
    xs, its = {}, {}
    for precision in (64, 32):
        h = amgc.setup(prob, precision=precision, **opts)
        assert h.stats()["n_levels"] == 4
        if precision == 64:
            _check_aggregates(h, prob)
        x = torch.zeros_like(b)
        it, rr, _ = h.solve(b, x)
        assert rr <= 1e-8 and _true_relres(h, b, x) <= 1e-8
        xs[precision], its[precision] = x, it
        h.close()
    assert its[32] <= its[64] + 3, its
    d = (torch.linalg.norm(xs[32] - xs[64]) / torch.linalg.norm(xs[64])).item()
    assert d <= 1e-6, d


def test_batched_set_converges_and_sampled_instances_match_their_own_solves():
    cat, npt, lpt, rhs, probs, _ = batched_workload(64, seed=3)
    opts = dict(precision=32, levels_max=4, coarse_max_rows=400, transfer=1, schur_damping=1, smoother_sweeps=3,
                autotune=1)
    hb = amgc.setup(cat, node_ptr=npt, lm_ptr=lpt, **opts)
    R = _cuda(rhs)
    X = torch.zeros_like(R)
    nrhs = rhs.shape[0]
    it, rr, _ = hb.solve_batched(R, X, n_sys=len(probs) * nrhs)
    assert np.all(rr <= 1e-8), rr.max()
    Xn = X.cpu().numpy()
    n_u = cat.n_u
    for q in (0, 4, 28, 63):                     # includes slave meshes 3x finer than the master
        h = amgc.setup(probs[q], **opts)
        for k in (0, nrhs - 1):
            bq = np.concatenate([rhs[k, 3 * npt[q]:3 * npt[q + 1]], rhs[k, n_u + 3 * lpt[q]:n_u + 3 * lpt[q + 1]]])
            xq = torch.zeros(bq.size, dtype=torch.float64, device="cuda")
            iq, rq, _ = h.solve(_cuda(bq), xq)
            xb = np.concatenate([Xn[k, 3 * npt[q]:3 * npt[q + 1]], Xn[k, n_u + 3 * lpt[q]:n_u + 3 * lpt[q + 1]]])
            ref = xq.cpu().numpy()
            assert np.linalg.norm(xb - ref) <= 1e-5 * np.linalg.norm(ref), (q, k)
        h.close()
    hb.close()


def test_adjoint_at_full_size_sampled_element_gradients():
    prob = workload(4, keep_full=True)
    e = prob.extra
    tab = ElementTables(prob)
    h = amgc.setup(prob, levels_max=10, coarse_max_rows=5000, transfer=1)
    b = _cuda(prob.rhs)
    x = torch.zeros_like(b)
    h.solve(b, x)
    J, gE, gt, adj, it = contact_gradients(prob, h, x, tab, adj_tol=1e-10)
    # the transposed system is solved to its tolerance
    n_u = prob.n_u
    c = torch.zeros_like(x)
    act = np.nonzero(prob.active)[0]
    cn = c.cpu().numpy()
    cn[n_u:].reshape(-1, 3)[act] = prob.triad[act, 0]
    xn = x.cpu().numpy()
    cn[:n_u].reshape(-1, 3)[prob.master_node] = xn[:n_u].reshape(-1, 3)[prob.master_node]
    assert _true_relres(h, _cuda(cn), adj, transposed=True) <= 1e-10
    # dJ/dE_e = -adj_e^T Khat_e x_e on 300 sampled elements, evaluated on the host
    an = adj.cpu().numpy()
    nf = e["node_free"]
    free = nf >= 0
    uf = e["u_D"].copy()
    af = np.zeros_like(uf)
    uf[free] = xn[:n_u].reshape(-1, 3)[nf[free]]
    af[free] = an[:n_u].reshape(-1, 3)[nf[free]]
    rng = np.random.default_rng(4)
    sample = rng.choice(tab.ne, size=300, replace=False)
    conn = e["conn"][sample]
    Kh = e["Khat"][e["elem_shape"][sample]]
    ref = -np.einsum("ei,eij,ej->e", af[conn].reshape(-1, 24), Kh, uf[conn].reshape(-1, 24))
    got = gE.cpu().numpy()[sample]
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    h.close()
