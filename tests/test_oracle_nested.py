"""Pins of the nested multigrid comparison preconditioner (oracle, CPU): the single-field K
hierarchy's V-cycle is a symmetric operator; with a one-level K hierarchy (a direct K solve) one
outer sweep is the SIMPLE preconditioner of Eq. ch6_ASIMPLE; FGMRES converges with it."""
import numpy as np

from oracle.krylov import fgmres
from oracle.nested import NestedPreconditioner
from paper_1912_09056_gb300.problem import two_block_problem, workload


def test_k_vcycle_is_symmetric():
    prob = workload(0)
    N = NestedPreconditioner(prob, levels_max=3, coarse_max_rows=0, transfer=1)
    assert len(N.kh.levels) == 3
    rng = np.random.default_rng(0)
    x, y = rng.standard_normal(N.nu), rng.standard_normal(N.nu)
    a, b = y @ N.kh.vcycle(x), x @ N.kh.vcycle(y)
    assert abs(a - b) <= 1e-11 * (abs(a) + abs(b))
    # and it is a contraction on K's error: ||I - V K||_K < 1 on a random vector
    K = N.K
    e = rng.standard_normal(N.nu)
    e1 = e - N.kh.vcycle(K @ e)
    assert np.sqrt(e1 @ (K @ e1)) < 0.9 * np.sqrt(e @ (K @ e))


def test_one_level_nested_sweep_is_eq_simple():
    p = two_block_problem(master_n=(3, 3, 2), slave_n=(2, 2, 2), tilt_deg=5.0, seed=11, active_fraction=0.6)
    omega = 0.8
    N = NestedPreconditioner(p, outer_sweeps=1, omega=omega, levels_max=1)
    n = p.n
    Minv = np.column_stack([N.apply(e) for e in np.eye(n)])
    K, B1, B2 = N.K.toarray(), N.B1.toarray(), N.B2.toarray()
    AtB1 = np.diag(N.at_inv) @ B1
    Sh = N.Zf.toarray() + B2 @ AtB1
    M = np.block([[K, K @ AtB1], [B2, B2 @ AtB1 - Sh / omega]])
    assert np.abs(np.linalg.inv(Minv) - M).max() <= 1e-9 * np.abs(M).max()


def test_nested_preconditioner_solves_the_tiny_workload():
    prob = workload(0)
    N = NestedPreconditioner(prob, outer_sweeps=1, omega=0.8, levels_max=3, coarse_max_rows=0, transfer=0)
    x, it, _ = fgmres(N.A(), prob.rhs, N.apply, tol=1e-8, maxit=200)
    assert np.linalg.norm(prob.rhs - N.A() @ x) <= 1e-8 * np.linalg.norm(prob.rhs)
    assert it <= 40, it
