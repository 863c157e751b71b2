"""Oracle of the geometric transfer (an option of this build, not the paper's transfer): full
weighting on the unknowns listed by position. Pinned by what it must be: exact on linear
functions at the interior points (where the paper's concatenated-vector transfer is not, on the
midpoint part), Toeplitz coarse matrices in position order, V-cycle limit = LU solution."""
import numpy as np
import pytest
import sympy as sp

from oracle import amg, fractional, model
from oracle.model import NONSYM, SPD


def _positions(N):
    """Positions (units of h) of the concatenated unknowns [v; w] of a level with N nodes."""
    return np.concatenate([np.arange(1, N + 1), np.arange(1, N + 2) - 0.5])


@pytest.mark.parametrize("N", [7, 15, 63])
def test_restriction_is_exact_on_linear_functions(N):
    n = 2 * N + 1
    Nc = (N - 1) // 2
    xf, xc = _positions(N), 2.0 * _positions(Nc)  # coarse mesh size 2h
    f = lambda x: 3.0 * x - 1.25
    R = amg.restriction_geometric(n)
    assert np.allclose(R @ f(xf), f(xc), rtol=0, atol=1e-12)
    # the paper's transfer is shifted by h/2 on the midpoint part
    Rp = amg.restriction(n)
    err = np.abs(Rp @ f(xf) - f(xc))
    assert err[:Nc].max() < 1e-12 and err[Nc + 1:].min() > 1.0


@pytest.mark.parametrize("N", [7, 31])
def test_prolongation_interpolates_linear_functions_inside(N):
    n = 2 * N + 1
    Nc = (N - 1) // 2
    xf, xc = _positions(N), 2.0 * _positions(Nc)
    f = lambda x: 0.5 * x + 2.0
    P = 2.0 * amg.restriction_geometric(n).T
    u = P @ f(xc)
    inside = (xf > 1.0) & (xf < N)  # every fine point with coarse neighbours on both sides
    assert np.allclose(u[inside], f(xf[inside]), rtol=0, atol=1e-12)


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("a", [sp.Rational(-1, 2), sp.Rational(1, 4)])
def test_coarse_matrices_are_toeplitz_in_position_order(variant, a):
    N, r = 64, 6
    H = amg.Hierarchy(fractional.assemble(variant, N, r, a), kc=3, transfer="geometric")
    for k in range(H.K - 1, H.kc - 1, -1):
        Ak = H.A[k]
        p = amg.position_order(Ak.shape[0])
        As = Ak[np.ix_(p, p)]
        assert np.max(np.abs(As[1:, 1:] - As[:-1, :-1])) <= 1e-12 * np.abs(As).max(), k


@pytest.mark.parametrize("variant", [SPD, NONSYM])
def test_vcycle_limit_is_the_lu_solution(variant):
    N, r = 32, 4
    A = model.assemble(variant, N, r)
    H = amg.Hierarchy(A, kc=3, transfer="geometric")
    b = np.random.default_rng(5).uniform(-1, 1, 2 * N - 1)
    u, it, rel, _ = amg.solve(H, b, tol=1e-14, max_iters=60)
    assert rel < 1e-14
    x = np.linalg.solve(A, b)
    assert np.linalg.norm(u - x) <= 1e-12 * np.linalg.norm(x)


@pytest.mark.parametrize("variant", [SPD, NONSYM])
def test_fractional_kernel_converges_fast(variant):
    """a = 1/4, N = 2^9, delta = 0.05: the paper's transfer needs 127 / 72 cycles to 1e-10,
    the geometric one at most 15 (the constant kernel takes 11 with either)."""
    N, r = 512, 25
    b = np.random.default_rng(0).uniform(-1, 1, 2 * N - 1)
    A = fractional.assemble(variant, N, r, sp.Rational(1, 4))
    it = amg.solve(amg.Hierarchy(A, kc=3, transfer="geometric"), b, tol=1e-10,
                   max_iters=100)[1]
    assert it <= 15


@pytest.mark.parametrize("a", [sp.Rational(-1, 2), sp.Integer(0), sp.Rational(1, 4)])
def test_two_grid_factor_below_one(a):
    """SPD system, N = 64, r = 6, omega = 2/3: ||S T||_A < 1 with the geometric transfer; for the
    fractional kernels it is far below the paper transfer's factor (the cause of the slow
    V-cycle), for the constant kernel both are below Theorem 4.1's sqrt(47/48)."""
    A = fractional.assemble(SPD, 64, 6, a)
    fg = amg.two_grid_factor(A, 2.0 / 3.0, "geometric")
    fp = amg.two_grid_factor(A, 2.0 / 3.0)
    assert 0.0 < fg < 1.0
    if a == sp.Rational(-1, 2):
        assert fg <= np.sqrt(47.0 / 48.0) and fp <= np.sqrt(47.0 / 48.0)
    else:
        assert fg < fp
