"""Edge cases through the C-ABI: no contact interface, all slave nodes inactive, one level, tiny
ragged meshes, a coarsest level beyond the dense limit, zero right-hand side, restart length one."""
import copy

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle.amg import Options, setup as oracle_setup  # noqa: E402
from oracle.krylov import fgmres  # noqa: E402
from paper_1912_09056_gb300 import amgc  # noqa: E402
from paper_1912_09056_gb300.problem import two_block_problem, workload  # noqa: E402


def _solve(h, rhs):
    b = torch.from_numpy(np.ascontiguousarray(rhs)).cuda()
    x = torch.zeros_like(b)
    it, rr, code = h.solve(b, x, check=False)
    return x.cpu().numpy(), it, rr, code


def test_no_contact_interface_is_refused():
    """Without slave nodes the system has no multiplier block: the setup refuses it cleanly."""
    p = copy.copy(workload(0))
    p.D = np.zeros(0); p.M_rowptr = np.zeros(1, np.int32); p.M_col = np.zeros(0, np.int32)
    p.M_val = np.zeros(0); p.slave_node = np.zeros(0, np.int32); p.master_node = np.zeros(0, np.int32)
    p.triad = np.zeros((0, 3, 3)); p.active = np.zeros(0, np.uint8); p.g = np.zeros(0)
    with pytest.raises(amgc.AmgcError) as e:
        amgc.setup(p, levels_max=3, coarse_max_rows=0)
    assert e.value.code == amgc.AMGC_EINVAL
    assert "no slave interface nodes" in str(e.value)


def test_all_slave_nodes_inactive():
    p = two_block_problem(master_n=(6, 6, 6), slave_n=(5, 5, 5), seed=2)
    p.active = np.zeros_like(p.active)
    h = amgc.setup(p, levels_max=3, coarse_max_rows=0, transfer=0)
    x, it, rr, code = _solve(h, p.rhs)
    assert code == amgc.AMGC_OK and rr <= 1e-8
    assert np.abs(x[p.n_u:]).max() <= 1e-12 * np.abs(x[:p.n_u]).max()   # inactive rows force lambda = 0
    ref = oracle_setup(p, Options(levels_max=3, coarse_max_rows=0, transfer=0))
    assert np.array_equal(h.export(0, "agg"), ref.levels[0].agg.astype(np.int32))
    h.close()


def test_single_level_is_a_direct_solve():
    p = workload(0)
    h = amgc.setup(p, levels_max=1, coarse_max_rows=0)
    assert h.stats()["n_levels"] == 1
    x, it, rr, code = _solve(h, p.rhs)
    assert code == amgc.AMGC_OK and it == 1 and rr <= 1e-10
    h.close()


def test_coarsest_too_large_is_refused():
    p = two_block_problem(master_n=(15, 15, 15), slave_n=(13, 13, 13), seed=1)
    assert p.n > 16384
    with pytest.raises(amgc.AmgcError) as e:
        amgc.setup(p, levels_max=1, coarse_max_rows=0)
    assert e.value.code == amgc.AMGC_EINVAL


def test_tiny_ragged_meshes_match_oracle():
    for mn, sn in (((3, 2, 2), (1, 1, 1)), ((2, 3, 1), (2, 1, 2))):
        p = two_block_problem(master_n=mn, slave_n=sn, seed=5, tilt_deg=3.0)
        h = amgc.setup(p, levels_max=2, coarse_max_rows=0, transfer=1)
        ref = oracle_setup(p, Options(levels_max=2, coarse_max_rows=0, transfer=1))
        assert np.array_equal(h.export(0, "agg"), ref.levels[0].agg.astype(np.int32))
        x, it, rr, code = _solve(h, p.rhs)
        assert code == amgc.AMGC_OK and rr <= 1e-8
        h.close()


def test_zero_rhs_and_restart_one():
    p = workload(0)
    h = amgc.setup(p, levels_max=3, coarse_max_rows=0)
    x, it, rr, code = _solve(h, np.zeros(p.n))
    assert code == amgc.AMGC_OK and it == 0 and not np.any(x)
    h.close()
    # FGMRES(1): one-step minimal residual with the V-cycle, restarted every iteration
    h = amgc.setup(p, levels_max=3, coarse_max_rows=0, transfer=0, fgmres_restart=1, fgmres_maxit=3000)
    x, it, rr, code = _solve(h, p.rhs)
    ref = oracle_setup(p, Options(levels_max=3, coarse_max_rows=0, transfer=0))
    _, it_ref, _ = fgmres(ref.A0(), p.rhs, ref.vcycle, tol=1e-8, restart=1, maxit=3000)
    assert code == amgc.AMGC_OK and rr <= 1e-8
    assert abs(it - it_ref) <= 3, (it, it_ref)
    h.close()
