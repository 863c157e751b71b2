"""Pins of the 2-D oracle (oracle/twod.py): the paper defines no 2-D system, so its parity is pinned
by mathematics only.

* a brute-force 2-D integration of entries over the square horizon (no factorisation used);
* exactness of the full stencil (with its exterior couplings) on the polynomials the
  tensor-product quadratic interpolant reproduces, against the closed-form square average;
* the relation to the printed 1-D matrix: A2 = A1 (x) I + I (x) A1 - A1 (x) A1 / (12 r);
* SPD (Cholesky) for the shifted-symmetric variant;
* Galerkin coarse operators equal the tensor formula with the 1-D Galerkin levels;
* the V-cycle converges and its limit is the LU solution; the large-size product equals the
  dense one.
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import amg, model, twod
from oracle.model import NONSYM, SPD
from synth import uniform_pm1


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("N,r", [(8, 2), (16, 3), (4, 6)])
def test_relation_to_the_printed_1d_matrix(variant, N, r):
    A2 = twod.assemble(variant, N, r)
    A1 = model.assemble(variant, N, r)
    d = 12.0 * r
    I = np.eye(A1.shape[0])
    ref = np.kron(A1, I) + np.kron(I, A1) - np.kron(A1, A1) / d
    assert np.max(np.abs(A2 - ref)) <= 1e-12 * np.max(np.abs(ref))


def _phi(xq, is_node_type):
    """The quadratic basis function centred at xq (units of h) as a plain function."""
    def f(y):
        if is_node_type:
            t = y - (xq - 1)
            if xq - 1 <= y <= xq:
                return t * (2 * t - 1)
            s = (xq + 1) - y
            if xq < y <= xq + 1:
                return s * (2 * s - 1)
            return 0.0
        if xq - 0.5 <= y <= xq + 0.5:
            return 4 * (y - (xq - 0.5)) * ((xq + 0.5) - y)
        return 0.0
    return f


@pytest.mark.parametrize("variant", [SPD, NONSYM])
def test_entries_by_brute_force_2d_integration(variant):
    N, r = 6, 2
    A2 = twod.assemble(variant, N, r)
    pts = twod.points(N)
    n = len(pts)
    rng = np.random.default_rng(3)
    picks = [(0, 0, 0, 0), (2, 7, 2, 7), (3, 8, 4, 9)] + [tuple(rng.integers(n, size=4))
                                                         for _ in range(9)]
    for i, j, p, q in picks:
        xi, ni = pts[i]
        yj, nj = pts[j]
        xp, np_ = pts[p]
        yq, nq_ = pts[q]
        fx = _phi(float(xp), twod._basis_type(variant, ni, np_))
        fy = _phi(float(yq), twod._basis_type(variant, nj, nq_))
        # breakpoints of the integrand at half steps: integrate cell by cell over the square
        brk = np.arange(-r, r + 0.25, 0.5)
        total = 0.0
        for a0, a1 in zip(brk[:-1], brk[1:]):
            for b0, b1 in zip(brk[:-1], brk[1:]):
                v, _ = integrate.dblquad(lambda s2, s1: fx(float(xi) + s1) * fy(float(yj) + s2),
                                         a0, a1, b0, b1, epsabs=1e-13, epsrel=1e-13)
                total += v
        ident = 1.0 if (i, j) == (p, q) else 0.0
        want = 12.0 * r * (ident - total / (2.0 * r) ** 2)
        assert abs(A2[i * n + j, p * n + q] - want) <= 1e-9 * 12 * r, (i, j, p, q)


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("a,b", [(0, 0), (1, 0), (0, 1), (1, 1), (2, 0), (0, 2), (2, 1), (1, 2),
                                 (2, 2)])
def test_full_stencil_exact_on_tensor_quadratics(variant, a, b):
    """d [f - average of f over the square]: the square average of x^a y^b is the product of
    the 1-D averages, and the 1-D average of x^2 over [x - r, x + r] is x^2 + r^2 / 3."""
    N, r = 8, 3
    f = lambda x, y: float(x) ** a * float(y) ** b  # noqa: E731
    avg = {0: lambda x: 1.0, 1: lambda x: x, 2: lambda x: x * x + r * r / 3.0}
    got = twod.full_stencil_apply(variant, N, r, f)
    pts = [float(x) for x, _ in twod.points(N)]
    want = np.array([[12.0 * r * (f(x, y) - avg[a](x) * avg[b](y)) for y in pts] for x in pts])
    assert np.max(np.abs(got - want)) <= 1e-9 * max(1.0, np.max(np.abs(want)))


def test_spd_variant_is_symmetric_positive_definite():
    A2 = twod.assemble(SPD, 16, 3)
    assert np.array_equal(A2, A2.T)
    np.linalg.cholesky(A2)


@pytest.mark.parametrize("variant", [SPD, NONSYM])
def test_galerkin_levels_are_the_tensor_formula(variant):
    """R2 A2 P2 = A_c (x) Q_c + Q_c (x) A_c - A_c (x) A_c / d at every level, with A_c the 1-D
    Galerkin levels and Q_c the 1-D Galerkin levels of the identity."""
    N, r = 16, 3
    K = 4
    H = twod.Hierarchy(twod.assemble(variant, N, r), kc=2)
    d = 12.0 * r
    A = model.assemble(variant, N, r)
    Q = np.eye(A.shape[0])
    for k in range(K, 1, -1):
        ref = np.kron(A, Q) + np.kron(Q, A) - np.kron(A, A) / d
        assert np.max(np.abs(H.A[k] - ref)) <= 1e-11 * np.max(np.abs(ref)), k
        A, Q = amg.galerkin(A), amg.galerkin(Q)


@pytest.mark.parametrize("variant", [SPD, NONSYM])
def test_vcycle_limit_is_the_lu_solution(variant):
    N, r = 16, 3
    A2 = twod.assemble(variant, N, r)
    H = twod.Hierarchy(A2, kc=2)
    b = uniform_pm1(A2.shape[0], 17)
    u, it, rel, _ = twod.solve(H, b, tol=1e-13, max_iters=200)
    assert rel < 1e-13 and it < 60
    x = np.linalg.solve(A2, b)
    assert np.linalg.norm(u - x) <= 1e-10 * np.linalg.norm(x)


@pytest.mark.parametrize("variant", [SPD, NONSYM])
def test_large_size_product_equals_dense(variant):
    N, r = 16, 3
    A2 = twod.assemble(variant, N, r)
    u = uniform_pm1(A2.shape[0], 2)
    y = twod.matvec_large(variant, N, r, u)
    assert np.linalg.norm(y - A2 @ u) <= 1e-13 * np.abs(A2).sum(0).max() * np.linalg.norm(u)
