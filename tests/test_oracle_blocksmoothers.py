"""Pins of the Uzawa, Braess-Sarazin and SIMPLE block smoothers and of the inner solvers of their
cheap variants (oracle, CPU).

Each smoother, run as the predictor-corrector step list of Algorithms 2-4, must be the
stationary iteration x <- x + M^{-1}(b - A x) with the closed-form block matrix M the paper
gives for it (Eqs. ch6_Uzawa, ch6_ABraessSarazin, ch6_ASIMPLE).  M is recovered from the sweep
itself (one sweep from a zero guess maps b to M^{-1} b), so a dropped term, a wrong sign or a
misplaced damping factor in a step shows up as a mismatch with the formula.  The error-matrix
special cases (Eqs. ch6_errormatUzawa_special, ch6_errormatBraessSarazin) and the inner
solvers' defining properties are pinned as well.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle.blocksmoothers import (braess_sarazin_sweep, ilu0_matrices, ilu0_solver, schur_approx, sgs,
                                   simple_sweep, uzawa_sweep)
from oracle.saddle import block_diag3, build_saddle
from oracle.smoother import atilde_diag
from paper_1912_09056_gb300.problem import two_block_problem


@pytest.fixture(scope="module")
def saddle():
    """A small tilted contact problem with a partial active set (about 200 unknowns)."""
    p = two_block_problem(master_n=(3, 3, 2), slave_n=(2, 2, 2), tilt_deg=5.0, jitter=0.2, seed=11,
                          active_fraction=0.6, E_slave=5.0)
    S = build_saddle(p)
    K = sp.csr_matrix(S.K.val)
    B1 = sp.csr_matrix(S.B1.val)
    B2 = sp.csr_matrix(S.B2.val)
    Zf = sp.csr_matrix(block_diag3(S.Z))
    A = sp.bmat([[K, B1], [B2, -Zf]], format="csr")
    return K, B1, B2, Zf, A


def _sweep_matrix_inverse(sweep, nu, n):
    """Columns of M^{-1}: one sweep from a zero guess applied to the unit right-hand sides."""
    Minv = np.zeros((n, n))
    for i in range(n):
        b = np.zeros(n)
        b[i] = 1.0
        u, lam = sweep(np.zeros(nu), np.zeros(n - nu), b[:nu], b[nu:])
        Minv[:, i] = np.concatenate([u, lam])
    return Minv


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# ------------------------------------------------------------------ inner solvers
def test_sgs_exact_on_a_diagonal_matrix_and_converges():
    rng = np.random.default_rng(0)
    d = rng.uniform(1.0, 3.0, 40)
    b = rng.standard_normal(40)
    x = sgs(sp.diags(d), b, rng.standard_normal(40), sweeps=1, omega=1.0)
    assert np.allclose(x, b / d, rtol=1e-14, atol=0.0)
    # SPD matrix: Gauss-Seidel converges to the solution
    T = sp.diags([-np.ones(39), 2.5 * np.ones(40), -np.ones(39)], [-1, 0, 1], format="csr")
    x = sgs(T, b, np.zeros(40), sweeps=200, omega=1.0)
    assert np.linalg.norm(x - spla.spsolve(T.tocsc(), b)) <= 1e-10 * np.linalg.norm(b)


def test_sgs_is_a_symmetric_operator_for_symmetric_k(saddle):
    """One damped SGS sweep from zero is b -> (symmetric SSOR matrix)^{-1} b for symmetric K."""
    K = saddle[0]
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal(K.shape[0]), rng.standard_normal(K.shape[0])
    z0 = np.zeros(K.shape[0])
    for omega in (1.0, 0.7):
        a = y @ sgs(K, x, z0, 1, omega)
        b = x @ sgs(K, y, z0, 1, omega)
        assert abs(a - b) <= 1e-12 * (abs(a) + abs(b))
    # one sweep from zero is the textbook SSOR preconditioner:
    # M = (1 / (omega (2 - omega))) (D + omega L) D^{-1} (D + omega U)
    Ks = K[:60, :60].toarray()
    D = np.diag(np.diag(Ks))
    Lo, Up = np.tril(Ks, -1), np.triu(Ks, 1)
    for omega in (0.7, 1.3):
        M = (D + omega * Lo) @ np.linalg.inv(D) @ (D + omega * Up) / (omega * (2.0 - omega))
        Minv = np.column_stack([sgs(sp.csr_matrix(Ks), e, np.zeros(60), 1, omega) for e in np.eye(60)])
        assert _rel(Minv, np.linalg.inv(M)) <= 1e-10
    # and it differs from one forward pass (it is not plain Gauss-Seidel)
    one = sgs(K, x, z0, 1, 1.0)
    fwd = spla.spsolve_triangular(sp.tril(K, format="csr"), x, lower=True)
    assert np.linalg.norm(one - fwd) > 1e-6 * np.linalg.norm(fwd)


def test_ilu0_is_exact_without_fill_and_matches_s_on_its_pattern():
    rng = np.random.default_rng(2)
    n = 30
    T = sp.diags([rng.uniform(-1, 0, n - 1), rng.uniform(3, 4, n), rng.uniform(-1, 0, n - 1)], [-1, 0, 1], format="csr")
    b = rng.standard_normal(n)
    assert np.allclose(ilu0_solver(T)(b), np.linalg.solve(T.toarray(), b), rtol=1e-12, atol=1e-14)
    # block tridiagonal with 3 x 3 blocks (no fill on the block pattern): exact
    nb = 8
    D = [rng.standard_normal((3, 3)) + 6 * np.eye(3) for _ in range(nb)]
    O = [rng.standard_normal((3, 3)) for _ in range(nb - 1)]
    Bt = sp.bmat([[D[i] if i == j else (O[min(i, j)] if abs(i - j) == 1 else None) for j in range(nb)]
                  for i in range(nb)], format="csr")
    b = rng.standard_normal(3 * nb)
    assert np.allclose(ilu0_solver(Bt, 3)(b), np.linalg.solve(Bt.toarray(), b), rtol=1e-11, atol=1e-13)
    # a 2D five-point matrix has fill: L U equals S on S's pattern only
    m = 6
    I = sp.identity(m)
    L1 = sp.diags([-np.ones(m - 1), 4 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1])
    S = (sp.kron(I, L1) + sp.kron(sp.diags([-np.ones(m - 1), -np.ones(m - 1)], [-1, 1]), I)).tocsr()
    L, U = ilu0_matrices(S)
    LU = (L @ U).toarray()
    Sd = S.toarray()
    pat = Sd != 0
    assert np.allclose(LU[pat], Sd[pat], rtol=1e-13, atol=1e-13)
    assert np.abs(LU[~pat]).max() > 1e-3          # the dropped fill
    assert set(zip(*L.nonzero())) | set(zip(*U.nonzero())) <= set(zip(*S.nonzero())) | set(zip(range(m * m), range(m * m)))
    assert sp.triu(L, k=1).nnz == 0 and sp.tril(U, k=-1).nnz == 0 and np.all(L.diagonal() == 1.0)


# ------------------------------------------------------------------ block smoothers
def test_uzawa_sweep_is_eq_uzawa(saddle):
    K, B1, B2, Zf, A = saddle
    nu, n = K.shape[0], A.shape[0]
    at_inv = 1.0 / atilde_diag(K, False)
    Sh = schur_approx(B1, B2, Zf, at_inv)
    Kd, Shd = K.toarray(), Sh.toarray()
    k_solve = lambda r: np.linalg.solve(Kd, r)   # noqa: E731
    s_solve = lambda r: np.linalg.solve(Shd, r)  # noqa: E731
    for omega in (0.7, 1.0):
        Minv = _sweep_matrix_inverse(
            lambda u, l, f, g: uzawa_sweep(K, B1, B2, Zf, u, l, f, g, omega, k_solve, s_solve), nu, n)
        M = np.block([[Kd, np.zeros((nu, n - nu))], [B2.toarray(), -Shd]]) / omega
        assert _rel(np.linalg.inv(Minv), M) <= 1e-9
        if omega == 1.0:
            # Eq. ch6_errormatUzawa_special: A - M = [0 B1; 0 B2 A~^{-1} B1]
            E = A.toarray() - np.linalg.inv(Minv)
            Eref = np.block([[np.zeros((nu, nu)), B1.toarray()],
                             [np.zeros((n - nu, nu)), (B2 @ sp.diags(at_inv) @ B1).toarray()]])
            assert _rel(E, Eref) <= 1e-9


def test_braess_sarazin_sweep_is_eq_bs_and_meets_the_constraints(saddle):
    K, B1, B2, Zf, A = saddle
    nu, n = K.shape[0], A.shape[0]
    at_inv = 1.0 / atilde_diag(K, False)
    omega = 1.9
    Sbs = schur_approx(B1, B2, Zf, at_inv, 1.0 / omega).toarray()
    s_solve = lambda r: np.linalg.solve(Sbs, r)  # noqa: E731
    sweep = lambda u, l, f, g: braess_sarazin_sweep(K, B1, B2, Zf, u, l, f, g, omega, at_inv, s_solve)  # noqa: E731
    Minv = _sweep_matrix_inverse(sweep, nu, n)
    M = np.block([[omega * np.diag(1.0 / at_inv), B1.toarray()], [B2.toarray(), -Zf.toarray()]])
    assert _rel(np.linalg.inv(Minv), M) <= 1e-9
    # Eq. ch6_errormatBraessSarazin: the second block row of A - M vanishes, so one sweep from
    # any iterate satisfies the constraint rows B2 u - Z lam = g
    rng = np.random.default_rng(3)
    f, g = rng.standard_normal(nu), rng.standard_normal(n - nu)
    u, lam = sweep(rng.standard_normal(nu), rng.standard_normal(n - nu), f, g)
    rc = g - B2 @ u + Zf @ lam
    assert np.linalg.norm(rc) <= 1e-11 * np.linalg.norm(g)


def test_simple_sweep_is_eq_simple(saddle):
    K, B1, B2, Zf, A = saddle
    nu, n = K.shape[0], A.shape[0]
    for simplec in (False, True):
        at_inv = 1.0 / atilde_diag(K, simplec)
        Shd = schur_approx(B1, B2, Zf, at_inv).toarray()
        Kd = K.toarray()
        omega = 0.8
        sweep = lambda u, l, f, g: simple_sweep(K, B1, B2, Zf, u, l, f, g, omega,  # noqa: E731
                                                lambda r, x0: np.linalg.solve(Kd, r), at_inv,
                                                lambda r: np.linalg.solve(Shd, r))
        Minv = _sweep_matrix_inverse(sweep, nu, n)
        AtB1 = (sp.diags(at_inv) @ B1).toarray()
        # Eq. ch6_ASIMPLE: [K 0; B2 -S_hat] [I A~^{-1} B1; 0 (1/omega) I]
        M = np.block([[Kd, Kd @ AtB1], [B2.toarray(), B2.toarray() @ AtB1 - Shd / omega]])
        assert _rel(np.linalg.inv(Minv), M) <= 1e-9


def test_cheap_variants_reduce_the_error(saddle):
    """With one SGS sweep for K and nodal-block ILU(0) for the Schur approximation, repeated
    sweeps of each smoother reduce the error of A x = b on this small problem.  (SIMPLE with
    A~ = diag(K); with SIMPLEC's row sums the stand-alone iteration diverges here, spectral radius
    about 1.9 at omega = 0.7, which a smoother inside a multigrid cycle may do.)"""
    K, B1, B2, Zf, A = saddle
    nu, n = K.shape[0], A.shape[0]
    rng = np.random.default_rng(4)
    x_true = rng.standard_normal(n)
    b = A @ x_true
    f, g = b[:nu], b[nu:]
    at_inv = 1.0 / atilde_diag(K, False)
    s_simple = ilu0_solver(schur_approx(B1, B2, Zf, at_inv), 3)
    at_d = 1.0 / atilde_diag(K, False)
    s_uz = ilu0_solver(schur_approx(B1, B2, Zf, at_d), 3)
    s_bs = ilu0_solver(schur_approx(B1, B2, Zf, at_d, 1.0 / 1.9), 3)
    smoothers = {
        "uzawa": lambda u, l: uzawa_sweep(K, B1, B2, Zf, u, l, f, g, 0.7,
                                          lambda r: sgs(K, r, np.zeros(nu), 1, 0.7), s_uz),
        "braess_sarazin": lambda u, l: braess_sarazin_sweep(K, B1, B2, Zf, u, l, f, g, 1.9, at_d, s_bs),
        "simple": lambda u, l: simple_sweep(K, B1, B2, Zf, u, l, f, g, 0.7,
                                             lambda r, x0: sgs(K, r, x0, 1, 0.7), at_inv, s_simple),
    }
    for name, sweep in smoothers.items():
        u, lam = np.zeros(nu), np.zeros(n - nu)
        e0 = np.linalg.norm(x_true)
        for _ in range(50):
            u, lam = sweep(u, lam)
        e = np.linalg.norm(np.concatenate([u, lam]) - x_true)
        assert np.isfinite(e) and e < 0.9 * e0, (name, e / e0)


@pytest.mark.parametrize("smoother, omega, sgs_kind", [("uzawa", 0.7, "point"), ("braess_sarazin", 1.9, "point"),
                                                       ("simple_sgs", 0.7, "point"), ("uzawa", 0.7, "colored_block"),
                                                       ("simple_sgs", 0.7, "colored_block")])
def test_block_smoothers_precondition_fgmres_on_the_tiny_workload(smoother, omega, sgs_kind):
    """The 3-level AMG of the tiny workload with three sweeps of each cheap block smoother (the
    paper's settings of Sec. 6.1: Uzawa(0.7) and SIMPLE(0.7) with one SGS(0.7) sweep, Braess-Sarazin
    (1.9), nodal-block ILU(0) for the Schur approximation) makes FGMRES reach 1e-8; the counts
    seen are 16, 18 and 12 against 30 for one CheapSIMPLE sweep; with the data-parallel nodal-block
    SGS in colour order, 15 and 12 for Uzawa and SIMPLE."""
    from oracle.amg import Options, setup
    from oracle.krylov import fgmres
    from paper_1912_09056_gb300.problem import workload
    prob = workload(0)
    H = setup(prob, Options(levels_max=3, coarse_max_rows=0, transfer=0, smoother=smoother, block_omega=omega,
                            smoother_sweeps=3, sgs_kind=sgs_kind))
    x, it, _ = fgmres(H.A0(), prob.rhs, H.vcycle, tol=1e-8, maxit=100)
    assert np.linalg.norm(prob.rhs - H.A0() @ x) <= 1e-8 * np.linalg.norm(prob.rhs)
    assert it <= 30, it


def test_jones_plassmann_colouring_is_proper_and_deterministic(saddle):
    from oracle.aggregate import aggregation_graph
    from oracle.blocksmoothers import jp_coloring
    K = saddle[0]
    nb = K.shape[0] // 3
    pat = sp.csr_matrix((np.ones(K.nnz), (K.tocoo().row // 3, K.tocoo().col // 3)), shape=(nb, nb))
    G = aggregation_graph(pat.tocsr(), np.zeros(nb, dtype=np.int64))
    col = jp_coloring(G)
    assert np.array_equal(col, jp_coloring(G))
    r, c = G.nonzero()
    assert np.all(col[r] != col[c])
    assert col.min() == 0 and col.max() < 27                  # at most max degree + 1 colours


def test_coloured_block_sgs_is_block_gauss_seidel_in_colour_order(saddle):
    """With omega = 1 one sweep is block Gauss-Seidel forward and backward in the node order
    sorted by colour: (D + L_p) x' = b - U_p x, then (D + U_p) x'' = b - L_p x' in that order
    (D the nodal diagonal blocks, L_p / U_p the strictly lower / upper block parts after the
    permutation); the sweep is a symmetric operator and repeated sweeps converge to K^{-1} b."""
    from oracle.aggregate import aggregation_graph
    from oracle.blocksmoothers import block_sgs_colored, jp_coloring
    K = saddle[0]
    n = K.shape[0]
    nb = n // 3
    coo = K.tocoo()
    pat = sp.csr_matrix((np.ones(K.nnz), (coo.row // 3, coo.col // 3)), shape=(nb, nb)).tocsr()
    col = jp_coloring(aggregation_graph(pat, np.zeros(nb, dtype=np.int64)))
    # permutation: nodes sorted by (colour, index); DOF-level permutation keeps the 3 DOFs together
    order = np.lexsort((np.arange(nb), col))
    perm = (order[:, None] * 3 + np.arange(3)[None, :]).ravel()
    Kp = K.toarray()[np.ix_(perm, perm)]
    D = np.zeros_like(Kp)
    for I in range(nb):
        D[3 * I:3 * I + 3, 3 * I:3 * I + 3] = Kp[3 * I:3 * I + 3, 3 * I:3 * I + 3]
    lo = np.zeros_like(Kp)                                  # strictly lower block part
    for I in range(nb):
        lo[3 * I:3 * I + 3, :3 * I] = Kp[3 * I:3 * I + 3, :3 * I]
    up = Kp - D - lo                                        # strictly upper block part
    rng = np.random.default_rng(6)
    b, x0 = rng.standard_normal(n), rng.standard_normal(n)
    xf = np.linalg.solve(D + lo, b[perm] - up @ x0[perm])   # colours ascending
    xb = np.linalg.solve(D + up, b[perm] - lo @ xf)         # colours descending
    got = block_sgs_colored(K, b, x0, col, 3, 1, 1.0)
    assert np.abs(got[perm] - xb).max() <= 1e-10 * np.abs(xb).max()
    # symmetric for symmetric K, any omega in (0, 2)
    x, y = rng.standard_normal(n), rng.standard_normal(n)
    z = np.zeros(n)
    for omega in (1.0, 0.8):
        a1 = y @ block_sgs_colored(K, x, z, col, 3, 1, omega)
        a2 = x @ block_sgs_colored(K, y, z, col, 3, 1, omega)
        assert abs(a1 - a2) <= 1e-10 * (abs(a1) + abs(a2))
    xs = block_sgs_colored(K, b, np.zeros(n), col, 3, 300, 1.0)
    assert np.linalg.norm(K @ xs - b) <= 1e-8 * np.linalg.norm(b)
