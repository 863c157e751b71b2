"""Pins of the flexible GMRES oracle (oracle/krylov.py) to the defining properties of GMRES."""
import numpy as np
import pytest

from oracle import amg, fractional, krylov, model


def _system(n, seed):
    rng = np.random.default_rng(seed)
    A = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / np.sqrt(n)
    M = np.eye(n) + 0.2 * rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    return A, M, b


@pytest.mark.parametrize("j", [1, 2, 3, 5, 7])
def test_residual_is_the_minimum_over_the_preconditioned_krylov_space(j):
    """With a fixed linear preconditioner M the j-step iterate minimises ||b - A x|| over
    x in M K_j(A M, b): compared with least squares on an explicit basis of that space."""
    A, M, b = _system(24, 7 + j)
    u, est, _ = krylov.restart_cycle(A, b, np.zeros_like(b), lambda v: M @ v, j)
    K = np.empty((b.size, j))
    K[:, 0] = b
    for i in range(1, j):
        K[:, i] = A @ (M @ K[:, i - 1])
    Q, _ = np.linalg.qr(K)
    y, *_ = np.linalg.lstsq(A @ M @ Q, b, rcond=None)
    best = np.linalg.norm(b - A @ M @ Q @ y)
    got = np.linalg.norm(b - A @ u)
    assert abs(got - best) <= 1e-10 * np.linalg.norm(b)
    assert abs(est - got) <= 1e-10 * np.linalg.norm(b)   # the Givens estimate is the residual
    assert np.linalg.norm(u - M @ Q @ y) <= 1e-8 * np.linalg.norm(u)  # the minimiser is unique


def test_n_steps_solve_exactly():
    A, M, b = _system(12, 3)
    u, est, _ = krylov.restart_cycle(A, b, np.zeros_like(b), lambda v: M @ v, 12)
    assert np.linalg.norm(b - A @ u) <= 1e-10 * np.linalg.norm(b)


def test_exact_inverse_as_preconditioner_solves_in_one_step():
    A, _, b = _system(16, 5)
    Ainv = np.linalg.inv(A)
    u, est, _ = krylov.restart_cycle(A, b, np.zeros_like(b), lambda v: Ainv @ v, 1)
    assert np.linalg.norm(b - A @ u) <= 1e-12 * np.linalg.norm(b) and est <= 1e-12


def test_breakdown_gives_the_exact_solution_and_no_nan():
    """A = I, b = e_1: the first step already spans the solution (h_{1,0} = 0); further steps
    meet zero pivots, which contribute nothing."""
    n = 6
    A = np.eye(n)
    b = np.zeros(n)
    b[0] = 2.0
    u, est, _ = krylov.restart_cycle(A, b, np.zeros(n), lambda v: v, 3)
    assert np.all(np.isfinite(u)) and np.allclose(u, b, atol=1e-15) and est == 0.0


def test_restarts_reach_tol_from_a_starting_guess():
    A, M, b = _system(30, 11)
    x0 = np.ones(30)
    u, its, rel, iterates = krylov.solve(A, b, lambda v: M @ v, steps=4, tol=1e-10, x0=x0)
    assert rel < 1e-10 and len(iterates) == its
    assert np.linalg.norm(b - A @ u) <= 1e-10 * np.linalg.norm(b - A @ x0)
    res = [np.linalg.norm(b - A @ x) for x in iterates]
    assert all(r1 <= r0 * (1 + 1e-12) for r0, r1 in zip(res, res[1:]))  # never increases


@pytest.mark.parametrize("variant", [0, 1])
def test_vcycle_preconditioned_solve_matches_the_direct_solution(variant):
    """On the paper's system (K = 7, constant kernel) the V-cycle-preconditioned FGMRES reaches
    the LU solution, in fewer V-cycles than the stationary iteration of section 5."""
    N = 2 ** 7
    A = model.assemble(variant, N, 8)
    H = amg.Hierarchy(A, kc=3)
    b = np.random.default_rng(2).uniform(-1, 1, A.shape[0])
    u, its, rel, _ = krylov.solve(A, b, lambda v: amg.vcycle(H, H.K, v), steps=4, tol=1e-10)
    x = np.linalg.solve(A, b)
    assert rel < 1e-10
    assert np.linalg.norm(u - x) <= 1e-9 * np.linalg.norm(x)
    _, its_stat, _, _ = amg.solve(H, b, tol=1e-10)
    assert 4 * its <= its_stat + 4  # no more V-cycles, up to those of one restart cycle


def test_fractional_nonsymmetric_case_where_the_stationary_iteration_diverges():
    """Fractional kernel a = 0.45, nonsymmetric system, geometric transfer (K = 7): the
    stationary V-cycle iteration diverges, the V-cycle-preconditioned FGMRES converges to the
    direct solution."""
    N = 2 ** 7
    A = fractional.assemble(1, N, 25, 0.45)
    H = amg.Hierarchy(A, kc=3, transfer="geometric")
    b = np.random.default_rng(4).uniform(-1, 1, A.shape[0])
    _, _, rel_stat, _ = amg.solve(H, b, tol=1e-10, max_iters=60)
    assert not rel_stat < 1e-3
    u, its, rel, _ = krylov.solve(A, b, lambda v: amg.vcycle(H, H.K, v), steps=8, tol=1e-10)
    x = np.linalg.solve(A, b)
    assert rel < 1e-10 and np.linalg.norm(u - x) <= 1e-8 * np.linalg.norm(x)
