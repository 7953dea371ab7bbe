"""The allocation-free element-gradient entry point agrees with the allocating one.

Collected last on purpose.  Callers that cannot allocate device memory when they need the
gradients (a framework that owns all device memory up front) use amgc_grad_elements_noalloc,
whose scratch is a fixed static device array.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1912_09056_gb300 import amgc  # noqa: E402
from paper_1912_09056_gb300.adjoint import ElementTables, objective_gradient  # noqa: E402
from paper_1912_09056_gb300.problem import two_block_problem  # noqa: E402


def test_noalloc_element_gradients_match_allocating_entry_point_twice():
    prob = two_block_problem(master_n=(7, 6, 6), slave_n=(6, 5, 5), E_slave=4.0, tilt_deg=5.0, seed=21,
                             active_fraction=0.6, log_E_sigma=0.5, keep_full=True)
    tab = ElementTables(prob)
    h = amgc.setup(prob, levels_max=3, coarse_max_rows=0, transfer=1, tol=1e-12)
    b = torch.from_numpy(prob.rhs).cuda()
    x = torch.zeros_like(b)
    h.solve(b, x)
    _, c = objective_gradient(prob, x)
    adj = torch.zeros_like(x)
    h.solve_transposed(c, adj, tol=1e-12)
    ref_gE = torch.empty(tab.ne, dtype=torch.float64, device="cuda")
    ref_gt = torch.empty(3, dtype=torch.float64, device="cuda")
    amgc.grad_elements(tab.conn, tab.shape, tab.Khat, tab.node_free, adj, x, tab.uD, tab.E, ref_gE,
                       lift_mask=tab.top, gt=ref_gt)
    for _ in range(2):   # two calls in a row share the static scratch
        gE = torch.full((tab.ne,), float("nan"), dtype=torch.float64, device="cuda")
        gt = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        amgc.grad_elements_noalloc(tab.conn, tab.shape, tab.Khat, tab.node_free, adj, x, tab.uD, tab.E, gE,
                                   lift_mask=tab.top, gt=gt)
        torch.cuda.synchronize()
        assert torch.allclose(gE, ref_gE, rtol=1e-12, atol=0.0)
        assert torch.allclose(gt, ref_gt, rtol=1e-12, atol=0.0)
    # without gt no scratch is touched: gE alone, compared with the allocating call
    gE_only = torch.full((tab.ne,), float("nan"), dtype=torch.float64, device="cuda")
    amgc.grad_elements_noalloc(tab.conn, tab.shape, tab.Khat, tab.node_free, adj, x, tab.uD, tab.E, gE_only)
    torch.cuda.synchronize()
    assert torch.allclose(gE_only, ref_gE, rtol=1e-12, atol=0.0)
    # zero elements: nothing to do, nothing written
    empty = torch.zeros((0, 8), dtype=torch.int32, device="cuda")
    keep = gt.clone()
    amgc.grad_elements_noalloc(empty, tab.shape, tab.Khat, tab.node_free, adj, x, tab.uD, tab.E, gE,
                               lift_mask=tab.top, gt=gt)
    torch.cuda.synchronize()
    assert torch.equal(gt, keep)
    # on a side stream: the call only enqueues work there; results read after that stream is done
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        gE_s = torch.full((tab.ne,), float("nan"), dtype=torch.float64, device="cuda")
        gt_s = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        amgc.grad_elements_noalloc(tab.conn, tab.shape, tab.Khat, tab.node_free, adj, x, tab.uD, tab.E, gE_s,
                                   lift_mask=tab.top, gt=gt_s, stream=side)
    side.synchronize()
    assert torch.allclose(gE_s, ref_gE, rtol=1e-12, atol=0.0)
    assert torch.allclose(gt_s, ref_gt, rtol=1e-12, atol=0.0)
    # sizes above the static scratch are refused before any device work
    big = torch.zeros((262145, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(amgc.AmgcError) as e:
        amgc.grad_elements_noalloc(big, tab.shape, tab.Khat, tab.node_free, adj, x, tab.uD, tab.E, gE,
                                   lift_mask=tab.top, gt=gt)
    assert e.value.code == amgc.AMGC_EINVAL
    h.close()
