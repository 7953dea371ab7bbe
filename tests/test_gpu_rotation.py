"""The CUDA path keeps the method's indifference to the model's orientation (the paper's rotated
two-body study, Sec. 6.1): rotating the tiny model about x leaves the FGMRES count within 10 %,
and each count within 2 of the oracle's."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle.amg import Options, setup as oracle_setup  # noqa: E402
from oracle.krylov import fgmres  # noqa: E402
from paper_1912_09056_gb300 import amgc  # noqa: E402
from paper_1912_09056_gb300.problem import workload  # noqa: E402


def test_iteration_count_is_rotation_invariant():
    opts = dict(levels_max=3, coarse_max_rows=0, transfer=0)
    counts = []
    for ang in (0.0, 30.0, 60.0, 90.0):
        prob = workload(0, tilt_deg=ang)
        h = amgc.setup(prob, **opts)
        b = torch.from_numpy(prob.rhs).cuda()
        x = torch.zeros_like(b)
        it, rr, _ = h.solve(b, x)
        h.close()
        ref = oracle_setup(prob, Options(**opts))
        _, it_ref, _ = fgmres(ref.A0(), prob.rhs, ref.vcycle, tol=1e-8)
        A = ref.A0()
        assert np.linalg.norm(prob.rhs - A @ x.cpu().numpy()) <= 1e-8 * np.linalg.norm(prob.rhs)
        assert abs(it - it_ref) <= 2, (ang, it, it_ref)
        counts.append(it)
    assert max(counts) <= 1.1 * min(counts) + 1, counts
