"""Plain float64 CPU oracle for the space-time PDHG method of Liu, Osher, Li and
Shu, "A primal-dual approach for solving conservation laws with implicit in
time approximations" (arXiv 2207.07234).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference arm of ``bench.py`` use it.  It shares no code with the
CUDA library under ``paper_2207_07234_gb300/``; the only module both sides use
is ``pdhg_workloads`` (seeded problem descriptions, no method arithmetic).

Modules (each function cites the passage of the paper it follows):

* ``spatial``   -- spatial operators D(v), their Jacobian-vector products and
                   transposes (Sec. 3.2; DG P2 reading of Sec. 3.2.2-3.2.3).
* ``spacetime`` -- the all-slices residual R(u) (Sec. 3.1), J(u)v and J(u)^T phi
                   (summation by parts, Sec. 3.1).
* ``precond``   -- K_d^{-1} (Eq. 2.8 and 2.10 discretised; Sec. 3.3) by FFT in x and a
                   tridiagonal solve in t; a dense K_d for small grids.
* ``pdhg``      -- Algorithm 1 and the residual Res(u, phi) (Eq. 2.12, Sec. 3.3).
* ``newton``    -- the definition of the discrete solution: the implicit scheme
                   solved time step by time step with Newton's method.
* ``dg_exact``  -- exact-rational DG assembly (Sec. 3.2.2, 3.2.3, Appendix A).
* ``variants``  -- Algorithm 2 (refinement of the time mesh, Sec. 3.4) and
                   Algorithm 3 (one time step at a time, Sec. 3.5).
* ``adjoint``   -- gradients of a terminal objective through the scheme: the
                   sequential discrete adjoint and Algorithm 1 on the problem
                   linearised at the solution.

Pins (the tests that tie this oracle to something other than itself) live in
``tests/test_oracle_*.py``: printed matrices (Eq. 3.5, A.1), Table 1, Table 2's
errors, the iteration counts of Sec. 4.3 and Table 3 (within 10%, 15% and 5%: counts
depend on step-size readings, so these pins are approximate), closed forms, the
proposition of Sec. 2.3, dense solves, finite differences of Newton solves.
"""
