"""Block smoothers of Sec. 5.1 in the cheap forms of Sec. 5.2 on the GPU against the oracle:
Uzawa (Algorithm 2), Braess-Sarazin (Algorithm 3) and SIMPLE / SIMPLEC (Algorithm 4) with damped
symmetric block Gauss-Seidel in Jones-Plassmann colour order for K and block ILU(0) of the Schur
approximation.  The colouring bit for bit on every smoothed level, one V-cycle within 1e-10,
FGMRES within +-2 iterations of the oracle and 1e-6 of its solution (the paper's settings of its
rotated two-body study, Sec. 6.1: three sweeps, one SGS(0.7) sweep inside)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle.aggregate import aggregation_graph  # noqa: E402
from oracle.amg import Options, setup as oracle_setup  # noqa: E402
from oracle.blocksmoothers import jp_coloring  # noqa: E402
from oracle.krylov import fgmres  # noqa: E402
from paper_1912_09056_gb300 import amgc  # noqa: E402
from paper_1912_09056_gb300.problem import two_block_problem, workload  # noqa: E402

PROBLEMS = {
    "tiny_PA_3lvl": (lambda: workload(0), dict(levels_max=3, coarse_max_rows=0, transfer=0)),
    "small_tilted_partial_SA_3lvl": (
        lambda: two_block_problem(master_n=(9, 9, 7), slave_n=(8, 7, 6), E_slave=10.0, tilt_deg=5.0, seed=11,
                                  active_fraction=0.6),
        dict(levels_max=3, coarse_max_rows=0, transfer=1)),
}
SMOOTHERS = {   # name: (oracle smoother, omega, simplec)
    "uzawa": ("uzawa", 0.7, 0),
    "braess_sarazin": ("braess_sarazin", 1.9, 0),
    "simple_sgs": ("simple_sgs", 0.7, 0),
    "simplec_sgs": ("simple_sgs", 0.7, 1),
}


@pytest.mark.parametrize("problem", list(PROBLEMS))
@pytest.mark.parametrize("smoother", list(SMOOTHERS))
def test_block_smoother_matches_the_oracle(problem, smoother):
    make, opts = PROBLEMS[problem]
    kind, omega, simplec = SMOOTHERS[smoother]
    prob = make()
    o = dict(opts, smoother_sweeps=3, simplec=simplec)
    ref = oracle_setup(prob, Options(smoother=kind, block_omega=omega, sgs_kind="colored_block", sgs_sweeps=1,
                                     sgs_omega=0.7, **o))
    h = amgc.setup(prob, **o)
    h.set_smoother(kind, omega=omega, sgs_sweeps=1, sgs_omega=0.7)
    if kind != "braess_sarazin":
        for l, L in enumerate(ref.levels[:-1]):
            col = jp_coloring(aggregation_graph(L.K.pat, np.zeros(L.nn, dtype=np.int64)), ref.opts.seed)
            assert np.array_equal(h.export(l, "color"), col.astype(np.int32)), l
    rng = np.random.default_rng(4)
    r = rng.standard_normal(prob.n)
    z = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    h.vcycle(torch.from_numpy(r).cuda(), z)
    zr = ref.vcycle(r)
    assert np.abs(z.cpu().numpy() - zr).max() <= 1e-10 * np.abs(zr).max()
    A = ref.A0()
    b = torch.from_numpy(prob.rhs).cuda()
    x = torch.zeros_like(b)
    it, rr, _ = h.solve(b, x)
    xr, it_ref, _ = fgmres(A, prob.rhs, ref.vcycle, tol=1e-8, maxit=600)
    xg = x.cpu().numpy()
    assert np.linalg.norm(prob.rhs - A @ xg) <= 1e-8 * np.linalg.norm(prob.rhs)
    assert abs(it - it_ref) <= 2, (it, it_ref)
    assert np.linalg.norm(xg - xr) <= 1e-6 * np.linalg.norm(xr)
    h.close()


def test_block_smoothers_rank_as_in_the_paper_and_refuse_fp32():
    """On the tiny workload three SIMPLE(SGS) sweeps need fewer FGMRES iterations than three
    Uzawa sweeps, and both fewer than one CheapSIMPLE sweep (the ordering of the paper's rotated
    two-body study, Sec. 6.1); FP32 and batched hierarchies refuse the block smoothers."""
    prob = workload(0)
    b = torch.from_numpy(prob.rhs).cuda()
    its = {}
    for kind in ("cheap_simple", "uzawa", "simple_sgs"):
        h = amgc.setup(prob, levels_max=3, coarse_max_rows=0, transfer=0,
                       smoother_sweeps=1 if kind == "cheap_simple" else 3)
        if kind != "cheap_simple":
            h.set_smoother(kind, omega=0.7)
        x = torch.zeros_like(b)
        its[kind], rr, _ = h.solve(b, x)
        assert rr <= 1e-8
        h.close()
    assert its["simple_sgs"] < its["uzawa"] < its["cheap_simple"], its
    h32 = amgc.setup(prob, precision=32, levels_max=3, coarse_max_rows=0)
    with pytest.raises(amgc.AmgcError) as ei:
        h32.set_smoother("uzawa")
    assert ei.value.code == amgc.AMGC_EINVAL
    h32.close()
