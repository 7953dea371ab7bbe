"""GPU parity: the CUDA library (through the C-ABI) against the FP64 oracle.

Integer outputs (aggregates, multiplier aggregates, sparsity patterns) must agree bit for
bit; FP64 values within 1e-10 relative; solves must reach the 1e-8 relative residual.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle.amg import Options, setup as oracle_setup  # noqa: E402
from oracle.krylov import fgmres  # noqa: E402
from paper_1912_09056_gb300 import amgc  # noqa: E402
from paper_1912_09056_gb300.problem import two_block_problem, workload  # noqa: E402

RTOL = 1e-10


def rel(a, b):
    d = np.abs(np.asarray(a) - np.asarray(b)).max() if np.size(a) else 0.0
    s = np.abs(np.asarray(b)).max() if np.size(b) else 1.0
    return d / (s if s > 0 else 1.0)


def _pattern(M):
    P = M.pat.tocsr()
    P.sort_indices()
    return P.indptr.astype(np.int32), P.indices.astype(np.int32)


def _check_block(h, level, prefix, M, what):
    rp, col = _pattern(M)
    g_rp = h.export(level, f"{prefix}_rowptr")
    g_col = h.export(level, f"{prefix}_col")
    assert np.array_equal(g_rp, rp), f"{what}: row pointers differ on level {level}"
    assert np.array_equal(g_col, col), f"{what}: block columns differ on level {level}"
    blocks = M.blocks()
    if blocks.size:
        g_val = h.export(level, f"{prefix}_val").reshape(blocks.shape)
        assert rel(g_val, blocks) <= RTOL, f"{what}: values differ on level {level}: {rel(g_val, blocks):.2e}"


def compare_hierarchy(h, ref):
    st = h.stats()
    assert st["n_levels"] == ref.n_levels
    for l, L in enumerate(ref.levels):
        assert st["rows"][l] == L.rows and st["disp_nodes"][l] == L.nn and st["lm_nodes"][l] == L.nl
        _check_block(h, l, "k", L.K, "K")
        _check_block(h, l, "b1", L.B1, "B1")
        _check_block(h, l, "b2", L.B2, "B2")
        assert rel(h.export(l, "z").reshape(-1, 3, 3), L.Z) <= RTOL
        if l < ref.n_levels - 1:
            assert np.array_equal(h.export(l, "agg"), L.agg.astype(np.int32)), f"aggregates differ on level {l}"
            assert np.array_equal(h.export(l, "lagg"), L.lagg.astype(np.int32)), f"LM aggregates differ on level {l}"
            _check_block(h, l, "p", L.P, "P")
            lam_max, omega = h.export(l, "omega")
            assert abs(lam_max - L.lam_max) <= 1e-12 * L.lam_max
            assert abs(omega - L.omega_j) <= 1e-12 * L.omega_j
            assert rel(h.export(l, "atinv"), L.at_inv) <= RTOL
            # with the Schur-step damping the library folds alpha_l / alpha into the inverted blocks
            a = ref.opts.simple_alpha
            fac = L.alpha / a if a > 0 else 1.0
            assert rel(h.export(l, "sinv").reshape(-1, 3, 3), L.S_inv * fac) <= RTOL
            if ref.opts.schur_damping and L.nl > 0:
                rho = h.export(l, "schur_rho")
                assert rho.size == 1 and abs(rho[0] - L.schur_rho) <= 1e-10 * L.schur_rho
            else:
                assert h.export(l, "schur_rho").size == 0
            w = np.asarray(L.Pl.val.sum(axis=1)).ravel()[0::3]
            assert rel(h.export(l, "pl_w"), w) <= RTOL
            Bn = h.export(l + 1, "nullspace").reshape(-1, 6)
            assert rel(Bn, ref.levels[l + 1].B) <= RTOL
        else:
            Ad = L.A().toarray()
            inv = h.export(l, "coarse_inv").reshape(Ad.shape)
            ref_inv = np.linalg.inv(Ad)
            # explicit inverse: agreement limited by cond(A_c) * eps
            assert rel(inv, ref_inv) <= 1e-16 * np.linalg.cond(Ad) * 100


def vcycle_and_apply(h, ref, n, seed=0):
    rng = np.random.default_rng(seed)
    r = rng.standard_normal(n)
    rd = torch.from_numpy(r).cuda()
    zd = torch.empty_like(rd)
    h.vcycle(rd, zd)
    yd = torch.empty_like(rd)
    h.apply(rd, yd)
    torch.cuda.synchronize()
    z_ref = ref.vcycle(r)
    y_ref = ref.A0() @ r
    # element by element: the largest difference against the largest reference entry
    ez = rel(zd.cpu().numpy(), z_ref)
    ey = rel(yd.cpu().numpy(), y_ref)
    return ez, ey


CASES = {
    "tiny_PA_3lvl": (lambda: workload(0), dict(levels_max=3, coarse_max_rows=0, transfer=0)),
    "tiny_SA_3lvl": (lambda: workload(0), dict(levels_max=3, coarse_max_rows=0, transfer=1)),
    "small_tilted_partial_SA": (
        lambda: two_block_problem(master_n=(13, 12, 11), slave_n=(10, 11, 9), E_slave=10.0, tilt_deg=5.0, seed=11,
                                  active_fraction=0.6),
        dict(levels_max=4, coarse_max_rows=200, transfer=1)),
    "small_simplec_2sweeps": (
        lambda: two_block_problem(master_n=(9, 9, 9), slave_n=(8, 8, 8), seed=5, active_fraction=0.5),
        dict(levels_max=3, coarse_max_rows=0, transfer=1, simplec=1, smoother_sweeps=2, jacobi_sweeps=2)),
    # slave mesh 2.3x finer than the master: rho(S_bd^-1 S_hat) ~ 10, Schur-step damping on
    "slave_finer_schur_damped": (
        lambda: two_block_problem(master_n=(6, 6, 4), slave_n=(14, 14, 6), E_slave=40.0, tilt_deg=6.0, seed=13,
                                  active_fraction=0.8),
        dict(levels_max=3, coarse_max_rows=0, transfer=1, schur_damping=1)),
}


@pytest.mark.parametrize("case", list(CASES))
def test_hierarchy_vcycle_and_solve_match_oracle(case):
    make, opts = CASES[case]
    prob = make()
    h = amgc.setup(prob, **opts)
    ref = oracle_setup(prob, Options(**opts))
    compare_hierarchy(h, ref)
    ez, ey = vcycle_and_apply(h, ref, prob.n)
    assert ey <= 1e-13, f"saddle apply differs: {ey:.2e}"
    assert ez <= RTOL, f"V-cycle differs: {ez:.2e}"
    b = torch.from_numpy(prob.rhs).cuda()
    x = torch.zeros_like(b)
    it, relres, _ = h.solve(b, x)
    xr, it_ref, _ = fgmres(ref.A0(), prob.rhs, ref.vcycle, tol=1e-8)
    A = ref.A0()
    xg = x.cpu().numpy()
    assert np.linalg.norm(prob.rhs - A @ xg) <= 1e-8 * np.linalg.norm(prob.rhs)
    assert abs(it - it_ref) <= 2, (it, it_ref)
    assert np.linalg.norm(xg - xr) <= 1e-6 * np.linalg.norm(xr)
    # host-buffer entry point gives the same solution
    xh, it_h, rr_h, _ = h.solve_host(prob.rhs)
    assert it_h == it and np.array_equal(xh, xg)
    xp = torch.empty(prob.n, dtype=torch.float64).pin_memory()   # caller-owned page-locked output
    _, it_p, _, _ = h.solve_host(prob.rhs, x=xp.numpy())
    assert it_p == it and np.array_equal(xp.numpy(), xg)
    # and so does the split form (u on the device, lambda on the host)
    u = torch.empty(prob.n_u, dtype=torch.float64, device="cuda")
    lam = np.empty(prob.n - prob.n_u)
    it_s, _, _ = h.solve_split(b, u, lam)
    assert it_s == it and np.array_equal(u.cpu().numpy(), xg[:prob.n_u]) and np.array_equal(lam, xg[prob.n_u:])
    h.close()


def test_setup_is_deterministic():
    prob = two_block_problem(master_n=(10, 10, 10), slave_n=(9, 9, 9), seed=2, tilt_deg=3.0, active_fraction=0.7)
    opts = dict(levels_max=3, coarse_max_rows=0, transfer=1)
    h1 = amgc.setup(prob, **opts)
    h2 = amgc.setup(prob, **opts)
    for what in ("agg", "lagg", "p_col", "p_val", "sinv"):
        assert np.array_equal(h1.export(0, what), h2.export(0, what)), what
    for what in ("k_col", "k_val", "b1_val", "b2_val"):
        assert np.array_equal(h1.export(1, what), h2.export(1, what)), what
    h1.close()
    h2.close()


def test_rejects_bad_input():
    prob = workload(0)
    bad = workload(0)
    bad.K_col = bad.K_col.copy()
    bad.K_col[5] = prob.n_nodes + 7          # column out of range
    with pytest.raises(amgc.AmgcError) as e:
        amgc.setup(bad, levels_max=3, coarse_max_rows=0)
    assert e.value.code == amgc.AMGC_EINVAL
    bad = workload(0)
    bad.slave_node = bad.slave_node.copy()
    bad.slave_node[0] = bad.slave_node[1]    # duplicate slave node
    with pytest.raises(amgc.AmgcError):
        amgc.setup(bad, levels_max=3, coarse_max_rows=0)
    # non-finite right-hand side -> breakdown, not a hang
    h = amgc.setup(prob, levels_max=3, coarse_max_rows=0)
    b = torch.from_numpy(prob.rhs).cuda()
    b[3] = float("nan")
    x = torch.zeros_like(b)
    _, _, code = h.solve(b, x, check=False)
    assert code == amgc.AMGC_BREAKDOWN
    # iteration limit -> not converged
    h2 = amgc.setup(prob, levels_max=3, coarse_max_rows=0, fgmres_maxit=2)
    it, rr, code = h2.solve(torch.from_numpy(prob.rhs).cuda(), x, check=False)
    assert code == amgc.AMGC_NOT_CONVERGED and it == 2 and rr > 1e-8
    h.close()
    h2.close()


# FP32 cycle: FP32 storage, arithmetic and accumulation inside the V-cycle, FP64 Schur-block
# inverses, coarsest inverse and FGMRES.  One cycle's relative deviation from the FP64 oracle
# is bounded by a few thousand FP32 roundings (2^-24 ~ 6e-8) through at most ~330-term sums
# on three levels: 1e-4 leaves an order of magnitude of margin.  The solve itself is FP64 and
# must reach the same 1e-8 relative residual.
FP32_CYCLE_RTOL = 1e-4


@pytest.mark.parametrize("case", ["tiny_SA_3lvl", "small_tilted_partial_SA", "small_simplec_2sweeps",
                                  "slave_finer_schur_damped"])
def test_fp32_cycle_matches_oracle_and_solves(case):
    make, opts = CASES[case]
    prob = make()
    h64 = amgc.setup(prob, **opts)
    h32 = amgc.setup(prob, precision=32, **opts)
    ref = oracle_setup(prob, Options(**opts))
    ez, ey = vcycle_and_apply(h32, ref, prob.n, seed=3)
    assert ey <= 1e-13, "the operator apply stays FP64"
    assert ez <= FP32_CYCLE_RTOL, f"FP32 V-cycle differs: {ez:.2e}"
    assert ez > 1e-12, "FP32 cycle unexpectedly bit-identical to FP64"
    b = torch.from_numpy(prob.rhs).cuda()
    x64 = torch.zeros_like(b)
    x32 = torch.zeros_like(b)
    it64, rr64, _ = h64.solve(b, x64)
    it32, rr32, _ = h32.solve(b, x32)
    A = ref.A0()
    assert np.linalg.norm(prob.rhs - A @ x32.cpu().numpy()) <= 1e-8 * np.linalg.norm(prob.rhs)
    assert it32 <= it64 + 3, (it32, it64)
    h64.close()
    h32.close()


def test_autotuned_mappings_and_graph_replay_give_the_same_cycle():
    """Row-mapping choices and CUDA-graph replay change scheduling, not arithmetic results beyond rounding."""
    make, opts = CASES["small_tilted_partial_SA"]
    prob = make()
    h0 = amgc.setup(prob, **opts)
    h1 = amgc.setup(prob, autotune=1, **opts)
    rng = np.random.default_rng(5)
    r = torch.from_numpy(rng.standard_normal(prob.n)).cuda()
    z0, z1, z2 = torch.empty_like(r), torch.empty_like(r), torch.empty_like(r)
    h0.vcycle(r, z0)            # graph replay
    h0.profile(1)               # timing mode runs the kernels directly
    h0.vcycle(r, z2)
    h0.profile(0)
    h1.vcycle(r, z1)
    torch.cuda.synchronize()
    assert torch.equal(z0, z2)
    assert (torch.linalg.norm(z0 - z1) / torch.linalg.norm(z0)).item() <= 1e-13
    h0.close()
    h1.close()


def test_fp32_autotuned_mappings_give_the_same_cycle():
    """The FP32 row-mapping candidates (warp, SELL with one or two threads, the shared-memory
    staged kernel) differ only in FP32 rounding of the same sums."""
    make, opts = CASES["small_tilted_partial_SA"]
    prob = make()
    h0 = amgc.setup(prob, precision=32, **opts)
    h1 = amgc.setup(prob, precision=32, autotune=1, **opts)
    rng = np.random.default_rng(6)
    r = torch.from_numpy(rng.standard_normal(prob.n)).cuda()
    z0, z1 = torch.empty_like(r), torch.empty_like(r)
    h0.vcycle(r, z0)
    h1.vcycle(r, z1)
    torch.cuda.synchronize()
    assert (torch.linalg.norm(z0 - z1) / torch.linalg.norm(z0)).item() <= 1e-5
    h0.close()
    h1.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_smoother_forms_give_the_same_cycle(precision):
    """The sweep's corrector + B1 update as two launches (form 0), fused into one single-CTA launch
    (form 1, the same arithmetic: the same bits) and split onto a second stream beside the Jacobi
    step (form 2, the interface rows' K products summed in another order): the oracle's cycle in
    every form, and with the default and the autotuned forms."""
    prob = two_block_problem(master_n=(13, 12, 11), slave_n=(10, 11, 9), E_slave=10.0, tilt_deg=5.0, seed=11,
                             active_fraction=0.6)
    opts = dict(levels_max=4, coarse_max_rows=200, transfer=1, smoother_sweeps=2)
    h = amgc.setup(prob, precision=precision, **opts)
    r = torch.from_numpy(np.random.default_rng(9).standard_normal(prob.n)).cuda()
    nlev = h.stats()["n_levels"]
    z = {}
    for form in (-1, 0, 1, 2):
        for l in range(nlev - 1):
            h.set_row_mapping(l, "fuse", precision, form)
        z[form] = torch.empty_like(r)
        h.vcycle(r, z[form])
    assert torch.equal(z[0], z[1])
    tight = 1e-13 if precision == 64 else 1e-5
    for form in (2, -1):
        assert (torch.linalg.norm(z[form] - z[0]) / torch.linalg.norm(z[0])).item() <= tight, form
    assert not torch.equal(z[2], z[0]), "the split sweep ran (level 0 sums its interface rows in another order)"
    ref = oracle_setup(prob, Options(**opts))
    zr = ref.vcycle(r.cpu().numpy())
    for form in (0, 2, -1):
        assert rel(z[form].cpu().numpy(), zr) <= (RTOL if precision == 64 else 1e-4), form
    h.close()
    # the autotuned hierarchy (row mappings and forms chosen by timing) gives the oracle's cycle too
    ht = amgc.setup(prob, precision=precision, autotune=1, **opts)
    z1 = torch.empty_like(r)
    ht.vcycle(r, z1)
    assert rel(z1.cpu().numpy(), zr) <= (1e-12 if precision == 64 else 1e-4)
    ht.close()
