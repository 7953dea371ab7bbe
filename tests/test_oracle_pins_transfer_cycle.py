"""Pins of three oracle parts against definitions computed another way, each with planted
mistakes that the pin must catch (the mistakes live in copies made here, on the CPU):

* the tentative multiplier prolongator P-hat^lambda (Sec. 4.1, Eq. ch6_segregatedtransfers): the
  thin QR of one nullspace column per aggregate and component, so its columns are orthonormal and
  it reproduces the multiplier nullspace from the coarse one;
* the nodal Schur blocks (Eq. ch6_simplecapprox): S_hat = Z + B2 A~^-1 B1 is minus the Schur
  complement of [A~ B1; B2 -Z], whose inverse is the multiplier block of the inverse of that
  matrix (block-inverse identity), for A~ = diag(K) and for SIMPLEC's absolute row sums;
* the V-cycle with smoothing on (Fig. mgalgorithm, Algorithm 4): a two-level cycle with an exact
  coarse solve equals the dense composition pre-smooth, coarse correction P A_c^-1 P^T, post-smooth,
  with the CheapSIMPLE sweep written as the product of its step matrices.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.amg import Options, setup
from oracle.saddle import block_diag3, build_saddle
from oracle.smoother import atilde_diag, schur_blocks
from oracle.transfer import tentative_lagmult


# ----------------------------------------------------------------------------- P-hat^lambda
def _lagmult_defects(make, lagg, n_lagg, Bl):
    """max |Pl^T Pl - I|, max |Pl Bc - B| (B: the 3-column multiplier nullspace) and the smallest
    coarse nullspace entry, for a builder with the signature of tentative_lagmult."""
    Pl, norm = make(lagg, n_lagg, Bl)
    V = Pl.val.toarray()
    orth = np.abs(V.T @ V - np.eye(3 * n_lagg)).max()
    B = np.zeros((3 * lagg.size, 3))
    Bc = np.zeros((3 * n_lagg, 3))
    for c in range(3):
        B[c::3, c] = Bl
        Bc[c::3, c] = norm
    repro = np.abs(V @ Bc - B).max()
    return orth, repro, float(np.min(norm))


def _uneven_lm_aggregates(seed):
    """A multiplier aggregate map with aggregate sizes 1, 2, 3, 5 and 7 in shuffled order, and a
    positive non-uniform nullspace entry per node (as on coarse levels, where it is a norm)."""
    rng = np.random.default_rng(seed)
    sizes = [1, 2, 3, 5, 7]
    lagg = np.concatenate([np.full(s, a) for a, s in enumerate(sizes)])
    lagg = lagg[rng.permutation(lagg.size)].astype(np.int64)
    Bl = rng.uniform(0.3, 2.5, size=lagg.size)
    return lagg, len(sizes), Bl


@pytest.mark.parametrize("seed", [0, 1])
def test_tentative_lagmult_is_orthonormal_and_reproduces_the_nullspace(seed):
    lagg, n_lagg, Bl = _uneven_lm_aggregates(seed)
    orth, repro, nmin = _lagmult_defects(tentative_lagmult, lagg, n_lagg, Bl)
    assert orth <= 1e-14 and repro <= 1e-14 and nmin > 0
    # the fine level's constant nullspace (every b_l = 1) gives weights 1/sqrt(|A_l|)
    ones = np.ones(lagg.size)
    Pl, norm = tentative_lagmult(lagg, n_lagg, ones)
    sizes = np.bincount(lagg, minlength=n_lagg)
    assert np.allclose(norm, np.sqrt(sizes), rtol=0, atol=1e-15)
    w = np.asarray(Pl.val.sum(axis=1)).ravel()[0::3]
    assert np.allclose(w, 1.0 / np.sqrt(sizes[lagg]), rtol=0, atol=1e-15)


def test_tentative_lagmult_on_the_tiny_hierarchy(cfg0):
    """Levels 0 and 1 of the 3-level hierarchy: orthonormal columns, nullspace reproduced."""
    h = setup(cfg0, Options(levels_max=3, coarse_max_rows=0, transfer=1))
    for L in h.levels[:-1]:
        orth, repro, nmin = _lagmult_defects(tentative_lagmult, L.lagg, L.n_lagg, L.Bl)
        assert orth <= 1e-13 and repro <= 1e-13 and nmin > 0
        assert np.array_equal(L.Pl.val.toarray(), tentative_lagmult(L.lagg, L.n_lagg, L.Bl)[0].val.toarray())


def _lagmult_size_weights(lagg, n_lagg, Bl):      # planted: b_l / |A_l| instead of b_l / ||b_L||
    Pl, norm = tentative_lagmult(lagg, n_lagg, Bl)
    cnt = np.bincount(lagg, minlength=n_lagg).astype(float)
    V = Pl.val.tocsr(copy=True)
    rows = np.repeat(np.arange(V.shape[0]), np.diff(V.indptr))
    V.data = Bl[rows // 3] / cnt[lagg[rows // 3]]
    Pl.val = V
    return Pl, cnt


def _lagmult_no_sqrt(lagg, n_lagg, Bl):           # planted: ||b_L||^2 in place of ||b_L||
    norm2 = np.bincount(lagg, weights=Bl * Bl, minlength=n_lagg)
    Pl, _ = tentative_lagmult(lagg, n_lagg, Bl)
    V = Pl.val.tocsr(copy=True)
    rows = np.repeat(np.arange(V.shape[0]), np.diff(V.indptr))
    V.data = Bl[rows // 3] / norm2[lagg[rows // 3]]
    Pl.val = V
    return Pl, norm2


@pytest.mark.parametrize("mutant", [_lagmult_size_weights, _lagmult_no_sqrt])
def test_planted_lagmult_mistakes_fail_the_pin(mutant):
    lagg, n_lagg, Bl = _uneven_lm_aggregates(0)
    orth, repro, _ = _lagmult_defects(mutant, lagg, n_lagg, Bl)
    assert orth > 1e-3 or repro > 1e-3


# ----------------------------------------------------------------------------- Schur blocks
def _schur_blocks_by_block_inverse(K, B1, B2, C, at):
    """Nodal 3x3 blocks of S_hat from the inverse of M = [diag(at) B1; B2 C], C = -Z the
    multiplier block of the saddle matrix: (M^-1)_{lambda lambda} = (C - B2 diag(at)^-1 B1)^-1,
    and S_hat = -(C - B2 diag(at)^-1 B1)."""
    nu = K.shape[0]
    M = np.block([[np.diag(at), B1], [B2, C]])
    Mi_ll = np.linalg.inv(M)[nu:, nu:]
    S = -np.linalg.inv(Mi_ll)
    nl = C.shape[0] // 3
    return np.stack([S[3 * l:3 * l + 3, 3 * l:3 * l + 3] for l in range(nl)])


def _small_contact():
    """A small tilted, partially active two-block contact with a finer slave mesh (dense-sized)."""
    from paper_1912_09056_gb300.problem import two_block_problem
    return two_block_problem(master_n=(3, 3, 2), slave_n=(4, 4, 2), E_slave=10.0, tilt_deg=5.0, seed=7,
                             active_fraction=0.7)


@pytest.mark.parametrize("simplec", [False, True])
def test_schur_blocks_equal_the_block_inverse_route(simplec):
    prob = _small_contact()
    S = build_saddle(prob)
    A = sp.bmat([[S.K.val, S.B1.val], [S.B2.val, -block_diag3(S.Z)]], format="csr").toarray()
    nu = S.K.val.shape[0]
    Kd, B1, B2, C = A[:nu, :nu], A[:nu, nu:], A[nu:, :nu], A[nu:, nu:]
    # A~ from its definition on the dense K: the diagonal, or the absolute row sums (SIMPLEC)
    at = np.array([np.abs(Kd[i]).sum() for i in range(nu)]) if simplec else np.array([Kd[i, i] for i in range(nu)])
    assert np.allclose(atilde_diag(S.K.val, simplec), at, rtol=1e-15, atol=0)
    ref = _schur_blocks_by_block_inverse(Kd, B1, B2, C, at)
    got = schur_blocks(S.B1.val, S.B2.val, S.Z, 1.0 / at)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-10 * scale
    # inactive nodes have B2 rows 0 and -Z = I, so their block is -I exactly
    inactive = np.nonzero(prob.active == 0)[0]
    assert inactive.size > 0
    assert np.abs(got[inactive] + np.eye(3)).max() <= 1e-14


def _schur_neg_z(B1, B2, Z, at_inv):                 # planted: sign of Z
    return schur_blocks(B1, B2, -Z, at_inv)


def _schur_transposed(B1, B2, Z, at_inv):           # planted: B1^T A~^-1 B2^T in place of B2 A~^-1 B1
    return schur_blocks(B2.T.tocsr(), B1.T.tocsr(), Z, at_inv)


def _schur_wrong_atilde(B1, B2, Z, at_inv):         # planted: A~^-2
    return schur_blocks(B1, B2, Z, at_inv * at_inv)


@pytest.mark.parametrize("mutant", [_schur_neg_z, _schur_transposed, _schur_wrong_atilde])
def test_planted_schur_mistakes_fail_the_pin(mutant):
    prob = _small_contact()
    S = build_saddle(prob)
    A = sp.bmat([[S.K.val, S.B1.val], [S.B2.val, -block_diag3(S.Z)]], format="csr").toarray()
    nu = S.K.val.shape[0]
    at = np.diag(A[:nu, :nu]).copy()
    ref = _schur_blocks_by_block_inverse(A[:nu, :nu], A[:nu, nu:], A[nu:, :nu], A[nu:, nu:], at)
    got = mutant(S.B1.val, S.B2.val, S.Z, 1.0 / at)
    assert np.abs(got - ref).max() > 1e-6 * np.abs(ref).max()


# ----------------------------------------------------------------------------- smoothed V-cycle
def _sweep_matrix(A, nu, omega, jacobi_sweeps, alpha):
    """Q of one CheapSIMPLE sweep in residual form, x <- x + Q (b - A x), built densely from the
    step matrices of Algorithm 4 in its cheap form:
        predictor   J = sum_{i<nJ} (I - omega D^-1 K)^i omega D^-1   (nJ damped Jacobi sweeps)
        corrector   dlam = -S_bd^-1 (r_lambda - B2 du),  S_bd = nodal blocks of Z + B2 A~^-1 B1
        update      lambda += alpha dlam,  u = u + du - alpha A~^-1 B1 dlam
    with D = A~ = diag(K), all read off the dense saddle matrix."""
    n = A.shape[0]
    K, B1, B2 = A[:nu, :nu], A[:nu, nu:], A[nu:, :nu]
    Z = -A[nu:, nu:]
    d = np.diag(K).copy()
    Dw = np.diag(omega / d)
    J = np.zeros((nu, nu))
    E = np.eye(nu)
    for _ in range(jacobi_sweeps):
        J += E @ Dw
        E = E @ (np.eye(nu) - Dw @ K)
    Sh = Z + B2 @ np.diag(1.0 / d) @ B1
    nl = n - nu
    Sbd_inv = np.zeros((nl, nl))
    for l in range(nl // 3):
        s = slice(3 * l, 3 * l + 3)
        Sbd_inv[s, s] = np.linalg.inv(Sh[s, s])
    I_u, I_l = np.eye(nu), np.eye(nl)
    F_pred = np.block([[J, np.zeros((nu, nl))], [np.zeros((nl, nu)), I_l]])
    F_elim = np.block([[I_u, np.zeros((nu, nl))], [-B2, I_l]])
    F_corr = np.block([[I_u, np.zeros((nu, nl))], [np.zeros((nl, nu)), -Sbd_inv]])
    F_upd = np.block([[I_u, -alpha * np.diag(1.0 / d) @ B1], [np.zeros((nl, nu)), alpha * I_l]])
    return F_upd @ F_corr @ F_elim @ F_pred


def _two_level_dense(h):
    """Dense A, P = diag(P^u, P^lambda), R = P^T, A_c = R A P and the fine sweep matrix Q."""
    L0 = h.levels[0]
    A = L0.A().toarray()
    P = np.block([[L0.P.val.toarray(), np.zeros((L0.nu_dofs, L0.Pl.val.shape[1]))],
                  [np.zeros((3 * L0.nl, L0.P.val.shape[1])), L0.Pl.val.toarray()]])
    R = P.T
    Ac = R @ A @ P
    Q = _sweep_matrix(A, L0.nu_dofs, L0.omega_j, h.opts.jacobi_sweeps, L0.alpha)
    return A, P, R, Ac, Q


def _compose(A, P, R, Ac, Q, b, sweeps, post=True, stale=False):
    x = np.zeros_like(b)
    for _ in range(sweeps):
        x = x + Q @ (b - A @ x)
    r = b if stale else b - A @ x
    x = x + P @ np.linalg.solve(Ac, R @ r)
    if post:
        for _ in range(sweeps):
            x = x + Q @ (b - A @ x)
    return x


@pytest.mark.parametrize("transfer, jacobi_sweeps, sweeps", [(1, 1, 1), (0, 2, 1), (1, 1, 2)])
def test_two_level_smoothed_vcycle_equals_the_dense_composition(cfg0, transfer, jacobi_sweeps, sweeps):
    h = setup(cfg0, Options(levels_max=2, coarse_max_rows=0, transfer=transfer, jacobi_sweeps=jacobi_sweeps,
                            smoother_sweeps=sweeps))
    assert h.n_levels == 2
    A, P, R, Ac, Q = _two_level_dense(h)
    rng = np.random.default_rng(11)
    for _ in range(3):
        b = rng.standard_normal(cfg0.n)
        ref = _compose(A, P, R, Ac, Q, b, sweeps)
        got = h.vcycle(b)
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


def _mutant_vcycle(h, b, kind):
    """The oracle's two-level cycle with one planted mistake."""
    L = h.levels[0]
    nu = L.nu_dofs
    f, g = b[:nu], b[nu:]
    u, lam = h.smooth(L, np.zeros(nu), np.zeros(b.size - nu), f, g)
    if kind == "stale_residual":
        ru, rl = f, g
    else:
        ru, rl = h.residual(L, u, lam, f, g)
    c = h.vcycle(np.concatenate([L.R.val @ ru, L.Rl.val @ rl]), 1)
    nuc = h.levels[1].nu_dofs
    u = u + L.P.val @ c[:nuc]
    lam = lam + L.Pl.val @ c[nuc:]
    if kind != "no_post":
        u, lam = h.smooth(L, u, lam, f, g)
    if kind == "wrong_alpha":
        L.alpha, a0 = 1.0, L.alpha
        try:
            u, lam = h.smooth(L, u, lam, f, g)
        finally:
            L.alpha = a0
    return np.concatenate([u, lam])


@pytest.mark.parametrize("kind", ["no_post", "stale_residual", "wrong_alpha"])
def test_planted_cycle_mistakes_fail_the_pin(cfg0, kind):
    h = setup(cfg0, Options(levels_max=2, coarse_max_rows=0, transfer=1))
    A, P, R, Ac, Q = _two_level_dense(h)
    b = np.random.default_rng(12).standard_normal(cfg0.n)
    ref = _compose(A, P, R, Ac, Q, b, 1)
    assert np.abs(h.vcycle(b) - ref).max() <= 1e-10 * np.abs(ref).max()
    bad = _mutant_vcycle(h, b, kind)
    assert np.abs(bad - ref).max() > 1e-6 * np.abs(ref).max()
