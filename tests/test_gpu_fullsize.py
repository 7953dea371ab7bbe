"""Full-size parity on the medium workload (48^3 + 41^3, 568 008 rows) in the bench's configuration."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle.amg import Options, setup as oracle_setup  # noqa: E402
from oracle.krylov import fgmres  # noqa: E402
from paper_1912_09056_gb300 import amgc  # noqa: E402
from paper_1912_09056_gb300.problem import workload  # noqa: E402
from test_gpu_parity import compare_hierarchy, vcycle_and_apply  # noqa: E402

OPTS = dict(levels_max=10, coarse_max_rows=5000, transfer=1)   # the bench's hierarchy options


@pytest.fixture(scope="module")
def medium():
    prob = workload(1)
    return prob, oracle_setup(prob, Options(**OPTS))


def test_medium_hierarchy_is_bit_exact_and_values_match(medium):
    prob, ref = medium
    h = amgc.setup(prob, **OPTS)
    compare_hierarchy(h, ref)
    ez, ey = vcycle_and_apply(h, ref, prob.n, seed=11)
    assert ey <= 1e-13 and ez <= 1e-10, (ey, ez)
    h.close()


def test_medium_solves_fp64_and_fp32_cycle(medium):
    prob, ref = medium
    b = torch.from_numpy(prob.rhs).cuda()
    xr, it_ref, _ = fgmres(ref.A0(), prob.rhs, ref.vcycle, tol=1e-8)
    A = ref.A0()
    for precision in (64, 32):
        h = amgc.setup(prob, precision=precision, **OPTS)
        x = torch.zeros_like(b)
        it, rr, _ = h.solve(b, x)
        xg = x.cpu().numpy()
        assert np.linalg.norm(prob.rhs - A @ xg) <= 1e-8 * np.linalg.norm(prob.rhs)
        assert abs(it - it_ref) <= 2, (precision, it, it_ref)
        assert np.linalg.norm(xg - xr) <= 1e-6 * np.linalg.norm(xr)
        h.close()
