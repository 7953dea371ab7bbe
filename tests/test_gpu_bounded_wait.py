"""The bounded waits of the staged FP32 apply: a wait that runs out of polls is reported as
AMGC_TIMEOUT, and the hierarchy stays usable.  The waits are made to run out by setting their
poll limit to zero tests of the barrier (amgc_set_wait_limit), so that every wait gives up, on the
tiny workload with the staged kernel forced on the fine level (amgc_set_row_mapping).  (With one
test most waits already see their copy landed on this L2-resident case, so one test is not a
reliable way to run them out.)"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle.amg import Options, setup as oracle_setup  # noqa: E402
from paper_1912_09056_gb300 import amgc  # noqa: E402
from paper_1912_09056_gb300.problem import workload  # noqa: E402

OPTS = dict(levels_max=3, coarse_max_rows=0, transfer=1)


def _cycle(h, r):
    z = torch.empty_like(r)
    h.vcycle(r, z)
    torch.cuda.synchronize()
    return z.cpu().numpy()


def test_wait_limit_gives_timeout_then_normal_cycles():
    prob = workload(0)
    ref = oracle_setup(prob, Options(**OPTS))
    r = np.random.default_rng(21).standard_normal(prob.n)
    z_ref = ref.vcycle(r)
    rd = torch.from_numpy(r).cuda()
    h = amgc.setup(prob, precision=32, **OPTS)
    z_default = _cycle(h, rd)
    h.set_row_mapping(0, "K", 32, 3)              # the staged kernel for the fine K apply
    z_staged = _cycle(h, rd)
    e = np.linalg.norm(z_staged - z_ref) / np.linalg.norm(z_ref)
    assert e <= 1e-4, e
    assert np.abs(z_staged - z_default).max() <= 1e-5 * np.abs(z_default).max()
    h.set_wait_limit(0)                            # every wait gives up without a test
    with pytest.raises(amgc.AmgcError) as ei:
        _cycle(h, rd)
    assert ei.value.code == amgc.AMGC_TIMEOUT
    assert "bounded wait" in str(ei.value)
    b = torch.from_numpy(prob.rhs).cuda()
    x = torch.zeros_like(b)
    it, rr, code = h.solve(b, x, check=False)
    assert code == amgc.AMGC_TIMEOUT
    h.set_wait_limit(-1)                           # the default limit again
    z_again = _cycle(h, rd)
    assert np.array_equal(z_again, z_staged)       # same launches, same order: same bits
    it, rr, code = h.solve(b, x)
    assert code == amgc.AMGC_OK and rr <= 1e-8
    h.close()


def test_row_mapping_override_rejects_bad_requests():
    prob = workload(0)
    h = amgc.setup(prob, precision=64, **OPTS)
    for args in [(0, "K", 32, 1), (0, "P", 64, 3), (9, "K", 64, 0), (2, "P", 64, 0), (0, "K", 64, 7)]:
        with pytest.raises(amgc.AmgcError) as ei:
            h.set_row_mapping(*args)
        assert ei.value.code == amgc.AMGC_EINVAL
    # every mapping of the FP64 fine K gives the same cycle to rounding
    r = torch.from_numpy(np.random.default_rng(2).standard_normal(prob.n)).cuda()
    zs = []
    for m in (-1, 0, 1, 2):
        h.set_row_mapping(0, "K", 64, m)
        zs.append(_cycle(h, r))
    for z in zs[1:]:
        assert np.abs(z - zs[0]).max() <= 1e-13 * np.abs(zs[0]).max()
    h.close()
