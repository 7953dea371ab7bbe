"""Active-set changes on the GPU against the oracle: the setup reuse of amgc_update_active_set
equals the oracle's setup(..., reuse=) (patterns bit for bit, values and one V-cycle within 1e-10)
and a fresh GPU setup with the new set; the primal-dual active set strategy of amgc_pdass visits
the oracle's active sets, stops on the same final set and meets the discrete contact conditions
(Sec. 2.2; Eqs. ch4_discretenormalcontact, ch4_discretefrictionless)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle.amg import Options, setup as oracle_setup  # noqa: E402
from oracle.pdass import pdass, with_active_set  # noqa: E402
from paper_1912_09056_gb300 import amgc  # noqa: E402
from paper_1912_09056_gb300.problem import two_block_problem, workload  # noqa: E402
from test_gpu_parity import RTOL, compare_hierarchy, vcycle_and_apply  # noqa: E402
from test_oracle_pdass import _curved_gap, _kkt  # noqa: E402


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


CASES = {
    "tiny_SA_3lvl": (lambda: workload(0), dict(levels_max=3, coarse_max_rows=0, transfer=1), 0.04),
    "small_tilted_SA_4lvl": (
        lambda: two_block_problem(master_n=(13, 12, 11), slave_n=(10, 11, 9), E_slave=10.0, tilt_deg=5.0, seed=11),
        dict(levels_max=4, coarse_max_rows=200, transfer=1), 0.04),
}


@pytest.mark.parametrize("case", list(CASES))
def test_update_active_set_equals_the_oracles_setup_reuse(case):
    make, opts, kappa = CASES[case]
    prob = make()
    g0 = _curved_gap(prob, kappa)
    _, _, hist = pdass(prob, g0)
    a1, a2 = hist[0], hist[-1]
    assert not np.array_equal(a1, a2)
    p1, p2 = with_active_set(prob, g0, a1), with_active_set(prob, g0, a2)
    o = Options(**opts)
    ref = oracle_setup(p2, o, reuse=oracle_setup(p1, o))
    h = amgc.setup(p1, **opts)
    h.update_active_set(a2.astype(np.uint8))
    compare_hierarchy(h, ref)
    ez, ey = vcycle_and_apply(h, ref, prob.n, seed=7)
    assert ey <= 1e-13 and ez <= RTOL, (ey, ez)
    # the same as a fresh setup with the new set (aggregation does not see the active set)
    hf = amgc.setup(p2, **opts)
    r = _cuda(np.random.default_rng(8).standard_normal(prob.n))
    z, zf = torch.empty_like(r), torch.empty_like(r)
    h.vcycle(r, z)
    hf.vcycle(r, zf)
    assert (torch.linalg.norm(z - zf) / torch.linalg.norm(zf)).item() <= 1e-12
    # and back to the first set: the first hierarchy's cycle again
    h0 = amgc.setup(p1, **opts)
    h.update_active_set(a1.astype(np.uint8))
    h0.vcycle(r, zf)
    h.vcycle(r, z)
    assert (torch.linalg.norm(z - zf) / torch.linalg.norm(zf)).item() <= 1e-12
    for hh in (h, hf, h0):
        hh.close()


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("precision", [64, 32])
def test_pdass_visits_the_oracles_active_sets(case, precision):
    make, opts, kappa = CASES[case]
    prob = make()
    g0 = _curved_gap(prob, kappa)
    _, x_ref, hist = pdass(prob, g0)
    assert len(hist) >= 3 and 0 < hist[-1].sum() < prob.n_s
    start = with_active_set(prob, g0, np.ones(prob.n_s, bool))
    h = amgc.setup(start, precision=precision, tol=1e-10, **opts)
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    act, steps, its, code = h.pdass(_cuda(prob.f), _cuda(g0), x, c=1.0, max_steps=20)
    assert code == amgc.AMGC_OK
    assert steps == len(hist), (steps, len(hist))
    assert np.array_equal(act.astype(bool), hist[-1])
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - x_ref) <= 1e-7 * np.linalg.norm(x_ref)
    _kkt(prob, g0, xg, 1e-7)
    h.close()


def test_pdass_rejects_bad_arguments_and_reports_an_unsettled_set():
    prob = workload(0)
    g0 = _curved_gap(prob, 0.04)
    h = amgc.setup(with_active_set(prob, g0, np.ones(prob.n_s, bool)), levels_max=3, coarse_max_rows=0, tol=1e-10)
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    f, g = _cuda(prob.f), _cuda(g0)
    for kw in (dict(c=0.0), dict(c=-1.0), dict(max_steps=0)):
        args = dict(c=1.0, max_steps=5)
        args.update(kw)
        with pytest.raises(amgc.AmgcError) as ei:
            h.pdass(f, g, x, **args)
        assert ei.value.code == amgc.AMGC_EINVAL
    # one solve is not enough for this gap: the set changes, so the call reports it
    act, steps, its, code = h.pdass(f, g, x, c=1.0, max_steps=1, check=False)
    assert code == amgc.AMGC_NOT_CONVERGED and steps == 1
    h.close()
