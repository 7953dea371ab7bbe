"""Nested multigrid (Sec. 3.2, Fig. mgmphmodelsA) on the GPU against the oracle's
NestedPreconditioner: outer SIMPLE sweeps on the finest level with a single-field AMG V-cycle on K
as predictor and the exact Schur complement.  One application within 1e-10, FGMRES within +-2
iterations of the oracle and 1e-6 of its solution."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle.krylov import fgmres  # noqa: E402
from oracle.nested import NestedPreconditioner  # noqa: E402
from paper_1912_09056_gb300 import amgc  # noqa: E402
from paper_1912_09056_gb300.problem import two_block_problem, workload  # noqa: E402

CASES = {
    "tiny_3lvl_1sweep": (lambda: workload(0), dict(levels_max=3, coarse_max_rows=0, transfer=1), 1, 0.8),
    "tiny_2lvl_3sweeps_PA": (lambda: workload(0), dict(levels_max=2, coarse_max_rows=0, transfer=0), 3, 0.8),
    "small_tilted_partial_4lvl_2sweeps": (
        lambda: two_block_problem(master_n=(13, 12, 11), slave_n=(10, 11, 9), E_slave=10.0, tilt_deg=5.0, seed=11,
                                  active_fraction=0.6),
        dict(levels_max=4, coarse_max_rows=0, transfer=1), 2, 0.7),
}


@pytest.mark.parametrize("case", list(CASES))
def test_nested_preconditioner_matches_the_oracle(case):
    make, opts, sweeps, omega = CASES[case]
    prob = make()
    ref = NestedPreconditioner(prob, outer_sweeps=sweeps, omega=omega, **opts)
    h = amgc.setup(prob, **opts)
    assert h.stats()["n_levels"] == len(ref.kh.levels)
    h.set_preconditioner(1, outer_sweeps=sweeps, omega=omega)
    rng = np.random.default_rng(3)
    for _ in range(2):
        r = rng.standard_normal(prob.n)
        z = torch.empty(prob.n, dtype=torch.float64, device="cuda")
        h.vcycle(torch.from_numpy(r).cuda(), z)
        zr = ref.apply(r)
        assert np.abs(z.cpu().numpy() - zr).max() <= 1e-10 * np.abs(zr).max()
    A = ref.A()
    b = torch.from_numpy(prob.rhs).cuda()
    x = torch.zeros_like(b)
    it, rr, _ = h.solve(b, x)
    xr, it_ref, _ = fgmres(A, prob.rhs, ref.apply, tol=1e-8)
    xg = x.cpu().numpy()
    assert np.linalg.norm(prob.rhs - A @ xg) <= 1e-8 * np.linalg.norm(prob.rhs)
    assert abs(it - it_ref) <= 2, (it, it_ref)
    assert np.linalg.norm(xg - xr) <= 1e-6 * np.linalg.norm(xr)
    # back to the coupled V-cycle
    h.set_preconditioner(0)
    it0, rr0, _ = h.solve(b, x)
    assert rr0 <= 1e-8
    h.close()


def test_nested_preconditioner_refusals():
    prob = workload(0)
    h32 = amgc.setup(prob, precision=32, levels_max=3, coarse_max_rows=0)
    with pytest.raises(amgc.AmgcError) as ei:
        h32.set_preconditioner(1)
    assert ei.value.code == amgc.AMGC_EINVAL
    h32.close()
    h = amgc.setup(prob, levels_max=3, coarse_max_rows=0)
    for args in [(1, 0, 0.8), (1, 1, 0.0), (2, 1, 0.8)]:
        with pytest.raises(amgc.AmgcError):
            h.set_preconditioner(*args)
    h.set_preconditioner(1)
    r = torch.ones(prob.n, dtype=torch.float64, device="cuda")
    with pytest.raises(amgc.AmgcError) as ei:
        h.vcycle_transposed(r, torch.empty_like(r))
    assert ei.value.code == amgc.AMGC_EINVAL
    h.close()
