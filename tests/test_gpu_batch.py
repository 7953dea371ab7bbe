"""Batched hierarchy: a block-diagonal batch of uneven instances equals the instances solved alone."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1912_09056_gb300 import amgc  # noqa: E402
from paper_1912_09056_gb300.problem import batched_workload  # noqa: E402

OPTS = dict(levels_max=3, coarse_max_rows=0, transfer=1)


def _split(v, npt, lpt, n_u):
    """Per-instance [u; lambda] pieces of a concatenated vector."""
    return [np.concatenate([v[3 * npt[q]:3 * npt[q + 1]], v[n_u + 3 * lpt[q]:n_u + 3 * lpt[q + 1]]])
            for q in range(len(npt) - 1)]


@pytest.mark.parametrize("precision, schur_damping", [(64, 0), (32, 0), (64, 1), (32, 1)])
def test_batch_equals_instances(precision, schur_damping):
    cat, npt, lpt, rhs, probs, _ = batched_workload(5, seed=9, lo=5, hi=9)
    hb = amgc.setup(cat, node_ptr=npt, lm_ptr=lpt, precision=precision, schur_damping=schur_damping, **OPTS)
    hs = [amgc.setup(p, precision=precision, schur_damping=schur_damping, **OPTS) for p in probs]
    if schur_damping:
        # per-instance Schur radii equal the instances' own, level by level
        for l in range(hb.stats()["n_levels"] - 1):
            rb = hb.export(l, "schur_rho")
            ri = np.array([h.export(l, "schur_rho")[0] for h in hs])
            assert rb.size == len(probs) and np.allclose(rb, ri, rtol=1e-10, atol=0.0), (l, rb, ri)
    # aggregates and multiplier aggregates: identical per instance (bit for bit, up to the offset)
    agg_b, lagg_b = hb.export(0, "agg"), hb.export(0, "lagg")
    for q, h in enumerate(hs):
        a = agg_b[npt[q]:npt[q + 1]]
        la = lagg_b[lpt[q]:lpt[q + 1]]
        assert np.array_equal(a - a.min(), h.export(0, "agg"))
        assert np.array_equal(la - la.min(), h.export(0, "lagg"))
    # one batched V-cycle equals the instances' V-cycles
    rng = np.random.default_rng(1)
    r = rng.standard_normal(cat.n)
    zb = torch.empty(cat.n, dtype=torch.float64, device="cuda")
    hb.vcycle(torch.from_numpy(r).cuda(), zb)
    zparts = _split(zb.cpu().numpy(), npt, lpt, cat.n_u)
    rparts = _split(r, npt, lpt, cat.n_u)
    for q, h in enumerate(hs):
        zq = torch.empty(rparts[q].size, dtype=torch.float64, device="cuda")
        h.vcycle(torch.from_numpy(rparts[q]).cuda(), zq)
        ref = zq.cpu().numpy()
        tol = 1e-12 if precision == 64 else 1e-5
        assert np.linalg.norm(zparts[q] - ref) <= tol * np.linalg.norm(ref), q
    # batched solve of 5 instances x 4 right-hand sides
    R = torch.from_numpy(np.ascontiguousarray(rhs)).cuda()
    X = torch.zeros_like(R)
    it, rr, _ = hb.solve_batched(R, X, n_sys=len(probs) * rhs.shape[0])
    assert np.all(rr <= 1e-8)
    Xn = X.cpu().numpy()
    for q, h in enumerate(hs):
        for k in range(rhs.shape[0]):
            bq = _split(rhs[k], npt, lpt, cat.n_u)[q]
            xq = torch.zeros(bq.size, dtype=torch.float64, device="cuda")
            iq, rq, _ = h.solve(torch.from_numpy(bq).cuda(), xq)
            xb = _split(Xn[k], npt, lpt, cat.n_u)[q]
            assert abs(int(it[q * rhs.shape[0] + k]) - iq) <= 1, (q, k, it[q * rhs.shape[0] + k], iq)
            ref = xq.cpu().numpy()
            assert np.linalg.norm(xb - ref) <= 1e-6 * np.linalg.norm(ref)
    for h in hs:
        h.close()
    hb.close()


def test_batched_stop_rule_and_transposed_guard():
    cat, npt, lpt, rhs, probs, _ = batched_workload(3, seed=4, lo=4, hi=8)
    hb = amgc.setup(cat, node_ptr=npt, lm_ptr=lpt, levels_max=6, coarse_max_rows=300, transfer=1)
    st = hb.stats()
    assert st["n_levels"] >= 2
    r = torch.ones(cat.n, dtype=torch.float64, device="cuda")
    with pytest.raises(amgc.AmgcError):
        hb.vcycle_transposed(r, torch.empty_like(r))
    hb.close()
