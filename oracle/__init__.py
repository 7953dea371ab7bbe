"""Plain FP64 CPU oracle of the block-AMG contact preconditioner (test infrastructure only).

This package is the slow, obviously-correct statement of what the CUDA library computes,
written from the paper (arXiv 1912.09056, Wiesner, Mayr, Popp, Gee, Wall) and used only by
the tests, by ``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``.  The
product path never imports it, and it imports nothing from the product package except the
seeded input generator's data class (which holds no multigrid arithmetic).

Modules:
  saddle    -- the 2x2 block saddle-point operator [K B1; B2 -Z] (Sec. 2.3)
  aggregate -- MIS-2 displacement aggregation and Lagrange-multiplier aggregation (Algorithm 1)
  transfer  -- tentative/smoothed transfers and Galerkin products (Sec. 3.1.2, Sec. 4.1)
  smoother  -- the CheapSIMPLE block smoother (Algorithm 4, Eq. ch6_simplecapprox, Sec. 5.2)
  amg       -- hierarchy setup and the V-cycle (Fig. mgalgorithm)
  krylov    -- right-preconditioned flexible GMRES (Sec. 3, stopping rule Eq. 7 of Sec. 6.1)

Parity status: every function here is pinned by a ``-m "not gpu"`` test in tests/.
"""
