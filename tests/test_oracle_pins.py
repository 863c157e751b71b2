"""Pins of the oracle against what the paper and the mathematics fix (no GPU)."""
import os

import numpy as np
import pytest

from oracle import amg, model
from oracle.model import NONSYM, SPD
from synth import uniform_pm1

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- coefficients (section 2.2) ---------------------------------------------------------

@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("N,r", [(8, 1), (8, 2), (8, 3), (16, 5), (8, 7), (8, 9)])
def test_printed_coefficients_equal_exact_quadrature(variant, N, r):
    """The printed integers of section 2.2 equal the exact collocation integrals of the
    quadratic basis (section 2), entry by entry, including truncated bands (r >= N-1)."""
    printed = model.assemble(variant, N, r)
    quad = model.assemble_quadrature(variant, N, r)
    assert np.array_equal(printed, quad)


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("row_is_node", [True, False])
@pytest.mark.parametrize("r", [1, 2, 5, 16])
def test_stencil_row_sum_and_quadratic_exactness(variant, row_is_node, r):
    """Full stencil: annihilates constants and x (row-sum identity of Lemma 4.3 / 4.6),
    and reproduces -L_delta x^2 = -2 gamma delta^3 / 3 scaled by eta_h, i.e. sum of
    entry * dist^2 = -4 r^3 in units of h."""
    d2 = np.arange(-(2 * r + 1), 2 * r + 2)
    w = np.array([model.stencil_entry(variant, row_is_node, k, r) for k in d2])
    x = d2 / 2.0
    assert np.sum(w) == 0.0
    assert np.sum(w * x) == 0.0
    assert np.sum(w * x * x) == pytest.approx(-4.0 * r ** 3, rel=0, abs=1e-9)


def test_spd_row_sum_identity_lemma43():
    for r in (1, 3, 10):
        cf = model.coefficients(r)
        assert cf["a_int"][0] + 2 * cf["a_int"][1:].sum() + 2 * cf["a_half"].sum() == 0.0


# --- transfers and Galerkin (section 3) -------------------------------------------------

def test_example_3_1_printed_coarse_matrix():
    """Example 3.1: A = I_7, D = I_8, B and C all ones; the printed 7x7 coarse matrix (x 8)
    is reproduced by full weighting on the concatenated vector and P = 2 R^T."""
    M = np.block([[np.eye(7), np.ones((7, 8))], [np.ones((8, 7)), np.eye(8)]])
    coarse = amg.galerkin(M) * 8.0
    expected = np.loadtxt(os.path.join(GOLDEN, "example31.txt"))
    assert np.array_equal(coarse, expected)


def test_example_3_1_fails_for_per_block_restriction():
    """Planted alternative reading: restricting v and w separately does not reproduce it."""
    M = np.block([[np.eye(7), np.ones((7, 8))], [np.ones((8, 7)), np.eye(8)]])
    Rv = amg.restriction(7)              # 3 x 7
    Rw = np.zeros((4, 8))
    for I in range(4):                   # a per-block variant of the same stencil
        Rw[I, 2 * I] = 0.25
        Rw[I, 2 * I + 1] = 0.5
        if 2 * I + 2 < 8:
            Rw[I, 2 * I + 2] = 0.25
    R = np.block([[Rv, np.zeros((3, 8))], [np.zeros((4, 7)), Rw]])
    coarse = R @ M @ (2 * R.T) * 8.0
    expected = np.loadtxt(os.path.join(GOLDEN, "example31.txt"))
    assert not np.array_equal(coarse, expected)


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("K,r", [(6, 4), (6, 7), (7, 16)])
def test_toeplitz_plus_cross_closure_and_lemma31(variant, K, r):
    """At every level the four blocks of eq. (3.7) are Toeplitz, and the Toeplitz part of
    Lemma 3.1 (8 a'_i = a_{2i-2} + 4 a_{2i-1} + 6 a_{2i} + 4 a_{2i+1} + a_{2i+2}) holds."""
    N = 1 << K
    H = amg.Hierarchy(model.assemble(variant, N, r), kc=2)
    for k in range(K, H.kc, -1):
        fine = amg.split_cross(H.A[k])
        coarse = amg.split_cross(H.A[k - 1])
        scale = np.max(np.abs(H.A[k]))
        for blk in "ABCD":
            assert amg.is_toeplitz(coarse["blocks"][blk], tol=1e-13 * scale)
            t = fine[blk]
            Nf, Nc = fine["N"], coarse["N"]
            for dlt in range(-(Nc - 1), Nc):
                idx = [2 * dlt + s + Nf - 1 for s in (-2, -1, 0, 1, 2)]
                val = (t[idx[0]] + 4 * t[idx[1]] + 6 * t[idx[2]] + 4 * t[idx[3]] + t[idx[4]]) / 8
                assert abs(val - coarse[blk][dlt + Nc - 1]) <= 1e-13 * scale


# --- theory of section 4 ----------------------------------------------------------------

@pytest.mark.parametrize("K,r", [(5, 4), (6, 8), (7, 16)])
def test_spd_hierarchy_and_jacobi_bound(K, r):
    """Lemma 4.5: the SPD system is symmetric positive definite (and so are its Galerkin
    coarse matrices); Lemma 4.7: lambda_max(D^{-1} A) lies in [1, 2]."""
    N = 1 << K
    H = amg.Hierarchy(model.assemble(SPD, N, r), kc=2)
    for k in range(K, H.kc - 1, -1):
        A = H.A[k]
        assert np.allclose(A, A.T, rtol=0, atol=1e-12 * np.abs(A).max())
        np.linalg.cholesky(A)
    A = H.A[K]
    d = np.diag(A)
    lam = np.linalg.eigvalsh(A / np.sqrt(np.outer(d, d))).max()
    assert 1.0 <= lam <= 2.0


@pytest.mark.parametrize("K,r", [(5, 4), (6, 8)])
@pytest.mark.parametrize("omega", [1.0, 2.0 / 3.0, 0.5])
def test_two_grid_factor_theorem41(K, r, omega):
    """Theorem 4.1: ||S_K T_K||_A <= sqrt(47/48) < 1 for 0 < omega <= 1."""
    A = model.assemble(SPD, 1 << K, r)
    f = amg.two_grid_factor(A, omega)
    assert 0.0 < f <= np.sqrt(47.0 / 48.0)


# --- solver -----------------------------------------------------------------------------

@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("K,r,kc", [(4, 2, 3), (5, 4, 3), (6, 8, 3), (6, 8, 1)])
def test_vcycle_converges_to_lu_solution(variant, K, r, kc):
    N = 1 << K
    A = model.assemble(variant, N, r)
    H = amg.Hierarchy(A, kc=kc)
    b = uniform_pm1(A.shape[0], seed=11)
    u, it, rel, _ = amg.solve(H, b, tol=1e-14, max_iters=200)
    assert rel < 1e-14
    x = np.linalg.solve(A, b)
    assert np.linalg.norm(u - x) <= 1e-11 * np.linalg.norm(x)


def test_vcycle_is_exact_when_coarsest_is_finest():
    A = model.assemble(SPD, 16, 2)
    H = amg.Hierarchy(A, kc=4)
    b = uniform_pm1(A.shape[0], seed=2)
    e = amg.vcycle(H, 4, b)
    assert np.allclose(A @ e, b, rtol=0, atol=1e-12 * np.abs(b).max())


@pytest.mark.parametrize("variant", [SPD, NONSYM])
def test_vcycle_iteration_count_small_case(variant):
    """N = 128, delta = 1/8 (r = 16): V(1,1), omega = 2/3, kc = 3 reaches 1e-10 quickly and
    the count does not grow with N (section 5: a few iterations per system)."""
    its = []
    for K in (6, 7, 8):
        N = 1 << K
        A = model.assemble(variant, N, model.horizon_ratio(0.125, 1.0 / N))
        H = amg.Hierarchy(A, kc=3)
        b = uniform_pm1(A.shape[0], seed=0)
        _, it, rel, _ = amg.solve(H, b, tol=1e-10, max_iters=60)
        assert rel < 1e-10
        its.append(it)
    assert max(its) <= 16
    assert max(its) - min(its) <= 3


@pytest.mark.parametrize("variant", [SPD, NONSYM])
def test_manufactured_solution_fourth_order(variant):
    """Fixed delta = 1/8, u = x^2 (1-x)^2: the discrete solution converges with order ~4
    (Tables 2-3 report rates 3.99 at fixed delta)."""
    errs = []
    for K in (5, 6, 7):
        N = 1 << K
        r = model.horizon_ratio(0.125, 1.0 / N)
        A = model.assemble(variant, N, r)
        b, uex = model.manufactured(variant, N, r)
        u = np.linalg.solve(A, b)
        errs.append(np.max(np.abs(u - uex)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 3.8) and np.all(rates < 4.2), (errs, rates)
    assert errs[-1] < 1e-8
