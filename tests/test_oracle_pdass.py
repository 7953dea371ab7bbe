"""Pins of the primal-dual active set strategy (oracle, CPU).  The stopping active set must
satisfy the discrete contact conditions (Eqs. ch4_discretenormalcontact,
ch4_discretefrictionless), checked directly on the solution.  Setup reuse across active-set
changes: the aggregates and transfers of the first step's hierarchy with the constraint blocks
formed anew equal a fresh setup, and the PDASS driven by FGMRES with them visits the same sets.
(The first hierarchy reused unchanged is no preconditioner for the later steps: its smoother
still treats the released nodes as active, and FGMRES stalls near 1e-7.)"""
import numpy as np
import pytest

from oracle.amg import Options, setup
from oracle.krylov import fgmres
from oracle.pdass import pdass, weighted_gap
from paper_1912_09056_gb300.problem import workload


def _curved_gap(prob, kappa):
    xs = prob.coords[prob.slave_node]
    return kappa * ((xs - xs.mean(axis=0)) ** 2).sum(axis=1)


def _kkt(prob, g0, x, tol):
    nu = 3 * prob.n_nodes
    lam = x[nu:].reshape(-1, 3)
    n = prob.triad[:, 0]
    lam_n = np.einsum("jk,jk->j", n, lam)
    gap = weighted_gap(prob, g0, x[:nu])
    scale = np.abs(lam_n).max()
    gscale = prob.D.max() * (np.abs(g0).max() + np.abs(x[:nu]).max())
    assert gap.min() >= -tol * gscale                       # no penetration
    assert lam_n.min() >= -tol * scale                      # compressive contact only
    assert np.abs(gap * lam_n).max() <= tol * gscale * scale  # complementarity
    assert np.abs(lam - lam_n[:, None] * n).max() <= tol * scale   # frictionless: no tangential part
    return lam_n, gap


@pytest.fixture(scope="module")
def tiny():
    return workload(0)


def test_pdass_stops_on_the_contact_conditions(tiny):
    g0 = _curved_gap(tiny, 0.04)
    p, x, hist = pdass(tiny, g0)
    assert len(hist) >= 3                                   # the set changed on the way
    assert 0 < hist[-1].sum() < tiny.n_s                    # partial contact at the end
    lam_n, gap = _kkt(tiny, g0, x, 1e-10)
    act = hist[-1]
    assert np.all(lam_n[~act] == 0.0)                       # inactive nodes carry no pressure
    assert np.abs(gap[act]).max() <= 1e-10 * np.abs(tiny.D * g0).max()   # active nodes are closed


def test_pdass_without_gap_keeps_every_node_active(tiny):
    p, x, hist = pdass(tiny, np.zeros(tiny.n_s))
    assert len(hist) == 1 and hist[0].all()
    _kkt(tiny, np.zeros(tiny.n_s), x, 1e-10)


def test_amg_setup_reused_across_active_set_changes(tiny):
    from oracle.pdass import with_active_set
    g0 = _curved_gap(tiny, 0.04)
    _, x_ref, hist_ref = pdass(tiny, g0)
    o = Options(levels_max=3, coarse_max_rows=0, transfer=1)
    h0 = setup(with_active_set(tiny, g0, hist_ref[0]), o)
    iters = []

    def solve(p, A, b):
        h = setup(p, o, reuse=h0)
        if len(iters) == len(hist_ref) - 1:               # the last step: compare with a fresh setup
            f = setup(p, o)
            for L, Lf in zip(h.levels, f.levels):
                for name in ("K", "B1", "B2"):
                    d = (getattr(L, name).val - getattr(Lf, name).val)
                    assert abs(d).max() <= 1e-13 * abs(getattr(Lf, name).val).max()
                assert np.abs(L.Z - Lf.Z).max() <= 1e-13 * max(np.abs(Lf.Z).max(), 1.0)
        x, it, _ = fgmres(A, b, h.vcycle, tol=1e-10, maxit=400)
        assert np.linalg.norm(b - A @ x) <= 1e-9 * np.linalg.norm(b)
        iters.append(it)
        return x
    _, x, hist = pdass(tiny, g0, solve=solve)
    assert len(hist) == len(hist_ref) and all(np.array_equal(a, b) for a, b in zip(hist, hist_ref))
    assert np.linalg.norm(x - x_ref) <= 1e-7 * np.linalg.norm(x_ref)
    assert max(iters) <= 60, iters
