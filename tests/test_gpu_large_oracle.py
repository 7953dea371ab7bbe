"""The large workload (3.47 M rows, 4 smoothed-aggregation levels, three CheapSIMPLE sweeps: the
bench's configuration) against the FP64 oracle:
aggregates, multiplier aggregates and every sparsity pattern bit for bit on all levels, transfers,
coarse operators and smoother data within 1e-10, one FP64 V-cycle within 1e-10, and the solutions
of the FP64-cycle and FP32-cycle solves against the oracle's FGMRES solution (all three meet the
1e-8 relative residual; their differences are bounded by the conditioning, about 1e-7 here)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle.amg import Options, setup as oracle_setup  # noqa: E402
from oracle.krylov import fgmres  # noqa: E402
from paper_1912_09056_gb300 import amgc  # noqa: E402
from test_gpu_parity import RTOL, compare_hierarchy, vcycle_and_apply  # noqa: E402

OPTS = dict(levels_max=4, coarse_max_rows=0, transfer=1, smoother_sweeps=3)   # the bench configuration


def test_large_workload_matches_the_oracle(large_problem):
    prob = large_problem
    h = amgc.setup(prob, **OPTS)
    ref = oracle_setup(prob, Options(**OPTS))
    assert ref.n_levels == 4
    compare_hierarchy(h, ref)
    ez, ey = vcycle_and_apply(h, ref, prob.n, seed=5)
    assert ey <= 1e-13, ey
    assert ez <= RTOL, ez
    A = ref.A0()
    xr, it_ref, _ = fgmres(A, prob.rhs, ref.vcycle, tol=1e-8)
    b = torch.from_numpy(prob.rhs).cuda()
    nu = prob.n_u
    for precision, bound in ((64, 1e-6), (32, 1e-6)):
        hh = h if precision == 64 else amgc.setup(prob, precision=precision, **OPTS)
        x = torch.zeros_like(b)
        it, rr, _ = hh.solve(b, x)
        xg = x.cpu().numpy()
        assert np.linalg.norm(prob.rhs - A @ xg) <= 1e-8 * np.linalg.norm(prob.rhs)
        if precision == 64:
            assert abs(it - it_ref) <= 2, (it, it_ref)
        eu = np.linalg.norm(xg[:nu] - xr[:nu]) / np.linalg.norm(xr[:nu])
        el = np.linalg.norm(xg[nu:] - xr[nu:]) / np.linalg.norm(xr[nu:])
        print(f"large workload, FP{precision} cycle: {it} iterations (oracle {it_ref}), "
              f"error against the oracle u {eu:.2e} lambda {el:.2e}")
        assert eu <= bound and el <= 10 * bound, (precision, eu, el)
        if hh is not h:
            hh.close()
    h.close()
