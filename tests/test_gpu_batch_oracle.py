"""The batched path against the FP64 oracle directly: every instance of a block-diagonal batch of
uneven instances gets, inside the one batched hierarchy, the aggregates, multiplier aggregates and
prolongators the oracle builds for it alone (bit for bit / 1e-10, on every level), one batched FP64
V-cycle equals the oracle's V-cycle of each instance within 1e-10, and the batched lockstep FGMRES
meets the oracle's solutions (iterations within +-2)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle.amg import Options, setup as oracle_setup  # noqa: E402
from oracle.krylov import fgmres  # noqa: E402
from paper_1912_09056_gb300 import amgc  # noqa: E402
from paper_1912_09056_gb300.problem import batched_workload  # noqa: E402


def _split(v, npt, lpt, n_u):
    return [np.concatenate([v[3 * npt[q]:3 * npt[q + 1]], v[n_u + 3 * lpt[q]:n_u + 3 * lpt[q + 1]]])
            for q in range(len(npt) - 1)]


def _sub_bsr(h, level, prefix, r0, r1, c0):
    """Rows [r0, r1) of an exported BSR with the block columns shifted by -c0."""
    rp = h.export(level, f"{prefix}_rowptr").astype(np.int64)
    col = h.export(level, f"{prefix}_col").astype(np.int64)
    val = h.export(level, f"{prefix}_val")
    a, b = rp[r0], rp[r1]
    nb = val.size // max(col.size, 1)
    return (rp[r0:r1 + 1] - a).astype(np.int32), (col[a:b] - c0).astype(np.int32), val[a * nb:b * nb]


@pytest.mark.parametrize("schur_damping", [0, 1])
def test_batched_instances_match_the_oracle(schur_damping):
    opts = dict(levels_max=3, coarse_max_rows=0, transfer=1, schur_damping=schur_damping)
    cat, npt, lpt, rhs, probs, _ = batched_workload(5, seed=9, lo=5, hi=9)
    hb = amgc.setup(cat, node_ptr=npt, lm_ptr=lpt, **opts)
    refs = [oracle_setup(p, Options(**opts)) for p in probs]
    nlev = hb.stats()["n_levels"]
    assert all(r.n_levels == nlev for r in refs)
    nq = len(probs)
    node_ptr = np.asarray(npt, dtype=np.int64)
    lm_ptr = np.asarray(lpt, dtype=np.int64)
    for l in range(nlev - 1):
        agg, lagg = hb.export(l, "agg"), hb.export(l, "lagg")
        next_node = np.zeros(nq + 1, dtype=np.int64)
        next_lm = np.zeros(nq + 1, dtype=np.int64)
        for q, ref in enumerate(refs):
            L = ref.levels[l]
            a = agg[node_ptr[q]:node_ptr[q + 1]].astype(np.int64)
            la = lagg[lm_ptr[q]:lm_ptr[q + 1]].astype(np.int64)
            assert np.array_equal(a - a.min(), L.agg), (l, q)
            assert np.array_equal(la - la.min(), L.lagg), (l, q)
            next_node[q + 1] = next_node[q] + L.n_agg
            next_lm[q + 1] = next_lm[q] + L.n_lagg
            assert a.min() == next_node[q] and la.min() == next_lm[q]
            # the instance's prolongator rows: pattern bit for bit, values within 1e-10
            rp, col, val = _sub_bsr(hb, l, "p", int(node_ptr[q]), int(node_ptr[q + 1]), int(next_node[q]))
            P = L.P.pat.tocsr()
            P.sort_indices()
            assert np.array_equal(rp, P.indptr.astype(np.int32)) and np.array_equal(col, P.indices.astype(np.int32))
            blocks = L.P.blocks()
            assert np.abs(val.reshape(blocks.shape) - blocks).max() <= 1e-10 * np.abs(blocks).max()
        node_ptr, lm_ptr = next_node, next_lm
    # one batched FP64 V-cycle against each instance's oracle V-cycle
    r = np.random.default_rng(1).standard_normal(cat.n)
    zb = torch.empty(cat.n, dtype=torch.float64, device="cuda")
    hb.vcycle(torch.from_numpy(r).cuda(), zb)
    zparts = _split(zb.cpu().numpy(), npt, lpt, cat.n_u)
    rparts = _split(r, npt, lpt, cat.n_u)
    for q, ref in enumerate(refs):
        zr = ref.vcycle(rparts[q])
        assert np.abs(zparts[q] - zr).max() <= 1e-10 * np.abs(zr).max(), q
    # the batched solve against the oracle's FGMRES, two right-hand sides per instance
    R = torch.from_numpy(np.ascontiguousarray(rhs)).cuda()
    X = torch.zeros_like(R)
    it, rr, _ = hb.solve_batched(R, X, n_sys=nq * rhs.shape[0])
    assert np.all(rr <= 1e-8)
    Xn = X.cpu().numpy()
    for q, ref in enumerate(refs):
        A = ref.A0()
        for k in (0, rhs.shape[0] - 1):
            bq = _split(rhs[k], npt, lpt, cat.n_u)[q]
            xr, ir, _ = fgmres(A, bq, ref.vcycle, tol=1e-8)
            xb = _split(Xn[k], npt, lpt, cat.n_u)[q]
            assert np.linalg.norm(bq - A @ xb) <= 1e-8 * np.linalg.norm(bq)
            assert abs(int(it[q * rhs.shape[0] + k]) - ir) <= 2, (q, k, it[q * rhs.shape[0] + k], ir)
            assert np.linalg.norm(xb - xr) <= 1e-6 * np.linalg.norm(xr)
    hb.close()
