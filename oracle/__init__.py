"""Oracle: a plain, slow FP64 CPU restatement of the method of Chen, Cao and Serra-Capizzano,
"Fast algebraic multigrid for block-structured dense and Toeplitz-like-plus-Cross systems
arising from nonlocal diffusion problems" (arXiv:2202.11288).

THIS PACKAGE IS TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import or call it. The solver library
(``paper_2202_11288_gb300``) never imports it and shares no code with it.

Contents
--------
``model``  -- the collocation matrices of section 2.2 assembled densely from the printed
             coefficients (section 2.2.1 nonsymmetric system, section 2.2.2 eq. (2.10)),
             and independently from exact quadrature of the piecewise-quadratic basis
             (section 2); the manufactured right-hand side for u = x^2 (1 - x)^2.
``amg``    -- section 3.1: restriction / prolongation, Galerkin coarse operators (dense
             R A P, eq. (3.6)), damped Jacobi (eq. (3.3)), the block V-cycle of
             Algorithm 2 with a dense LU at the coarsest level, the outer iteration and the
             stopping rule of section 5; the Cross splitting of eq. (3.7) read off a
             dense level matrix; the two-grid factor of Theorem 4.1. Also, as an option
             that is not the paper's, the geometric transfer (the same restriction rows on
             the unknowns listed by position), pinned by tests/test_oracle_geometric.py.
``timestep`` -- section 5: the time-dependent problem advanced by the BDF4 scheme of eq.
             (5.1) with the shifted system (sigma I + A) U^k = ..., for the exact solution
             u = e^t (1 + x)^6 of Tables 2 and 3.
``weakly``  -- section 2.1: the weakly singular nonlocal model of eq. (2.3) (diagonal minus
             the 2x2 Toeplitz block matrix), assembled from exact element integrals, and its
             BDF4 time stepping for Table 1.
``fractional`` -- a fractional kernel |s|^{-(1+2a)} with a horizon (not in the paper): exact
             element integrals of the same collocation, Hadamard finite parts for a >= 1/2.
             PARITY UNPINNED by the paper (pinned only by mathematics: a = -1/2 is the printed
             matrix, exactness on quadratics, Hadamard's definition by quadrature).
``krylov`` -- an outer iteration that is not the paper's: restarted, right-preconditioned
             flexible GMRES with one V-cycle as the preconditioner (Saad's FGMRES, classical
             Gram-Schmidt done twice, Givens rotations), pinned by tests/test_oracle_krylov.py to
             the minimal-residual property on an explicit Krylov basis and to exact solves.
``large``  -- the same finest-level operator for sizes where a dense matrix does not fit:
             selected dense rows, and the product computed with numpy's FFT as the
             convolution step (section 3.2, eq. (3.4)).

Parity status: every function here is pinned by ``tests/test_oracle_*.py`` (printed
coefficients vs quadrature, Example 3.1, Toeplitz closure, SPD and the two-grid bound of
Theorem 4.1, LU agreement, order of accuracy, the sixteen BDF4 errors of Tables 2 and 3, the
printed coefficient formulas of section 2.1 and the twelve BDF4 errors of Table 1).
``fractional`` is the one part whose parity the paper cannot pin.
"""
