"""Oracle of the weakly singular nonlocal model (section 2.1, eq. (2.3)) against what the
paper prints: the coefficient formulas of M, N, P, Q and D (equal to the exact element
integrals, except p_0 and the boundary weights eta_{i/2}, i >= 2, which are read as garbled),
and the twelve BDF4 errors of Table 1 (tests/golden/bdf4_table1.txt)."""
import math
import os

import numpy as np
import pytest

from oracle import amg, weakly

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "bdf4_table1.txt")


def printed(gamma, K):
    """The printed coefficient formulas of section 2.1 (k >= 1 for m, p; k >= 0 for q)."""
    e3, e2 = 3 - gamma, 2 - gamma
    m = lambda k: 4 * ((k + 1) ** e3 - (k - 1) ** e3) - e3 * ((k + 1) ** e2 + 6 * k ** e2 + (k - 1) ** e2)  # noqa: E731
    q = lambda k: -8 * ((k + 1) ** e3 - k ** e3) + 4 * e3 * ((k + 1) ** e2 + k ** e2)  # noqa: E731
    return {"m0": 2 * (1 + gamma), "n0": (2 - gamma) * 2 ** (gamma + 1),
            "m": [m(k) for k in range(1, K)], "q": [q(k) for k in range(0, K)],
            "p": [m(k + 0.5) for k in range(1, K)], "n": [q(k - 0.5) for k in range(1, K)],
            "p0": 4 * (1.5 ** e3 - 0.5 ** e3) - e3 * (1.5 ** e2 + 3 * 0.5 ** e2),
            "eta_half": (2 - gamma) * (1 - gamma) * 2 ** (gamma - 1)}


@pytest.mark.parametrize("gamma", [0.0, 0.25, 0.5, 0.9])
def test_printed_coefficients_are_the_element_integrals(gamma):
    N, K = 24, 8
    c = lambda p2, q2: weakly.coupling(p2, q2, N, gamma)  # noqa: E731
    pr = printed(gamma, K)
    node, mid = 2 * 8, 2 * 8 - 1  # an interior node and midpoint (twice-coordinates)
    assert math.isclose(c(node, node), pr["m0"], rel_tol=1e-13)
    assert math.isclose(c(mid, mid), pr["n0"], rel_tol=1e-13)
    for k in range(1, K):
        assert math.isclose(c(node, node + 2 * k), pr["m"][k - 1], rel_tol=1e-11)   # M
        assert math.isclose(c(mid, mid + 2 * k), pr["n"][k - 1], rel_tol=1e-11)     # N
        assert math.isclose(c(mid, mid + 1 + 2 * k), pr["p"][k - 1], rel_tol=1e-11)  # P
    for k in range(0, K):
        assert math.isclose(c(node, node + 1 + 2 * k), pr["q"][k], rel_tol=1e-11)  # Q
    # diagonal d_{i/2} and the first boundary weight
    d = weakly.diagonal(N, gamma)
    x2 = weakly.points(N)
    for idx in (0, 5, N - 2, N - 1, 2 * N - 2):
        i = x2[idx]
        assert math.isclose(d[idx], (3 - gamma) * (2 - gamma) * ((i / 2) ** (1 - gamma) + (N - i / 2) ** (1 - gamma)), rel_tol=1e-14)
    assert math.isclose(c(1, 0), pr["eta_half"], rel_tol=1e-13)
    # read as garbled: the printed p_0 is no entry of the matrix (the nearest mid-node one is)
    assert not math.isclose(c(mid, mid + 1), pr["p0"], rel_tol=1e-3)


def table_rows():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                g, N, e = line.split()
                rows.append((float(g), int(N), float(e)))
    return rows


@pytest.mark.parametrize("gamma,N,printed_err", table_rows())
def test_bdf4_matches_table_1(gamma, N, printed_err):
    """N <= 128: within 5 units of the last printed digit. N = 256: the error (about 2e-11 of
    max|u|) is at the level where the closed-form coefficients lose precision to cancellation
    (differences of powers of k ~ 2N in FP64), so only 1 % is required there."""
    err, _ = weakly.bdf4(N, gamma)
    unit = 10.0 ** (math.floor(math.log10(printed_err)) - 4)
    tol = 5 * unit if N <= 128 else 0.01 * printed_err
    assert abs(err - printed_err) <= tol, (err, printed_err)


def test_vcycle_converges_on_the_shifted_system():
    """Algorithm 2 (dense Galerkin, LU at k_c = 3) on the BDF4 matrix sigma I + A_h: a few cycles
    per step, as Table 1 reports (2-4 iterations at tol 1e-15)."""
    N, gamma = 64, 0.5
    A = weakly.assemble(N, gamma)
    sigma = 25.0 * weakly.eta(N, gamma) / 12.0 * N
    H = amg.Hierarchy(A + sigma * np.eye(A.shape[0]), kc=3)
    b = np.random.default_rng(0).uniform(-1, 1, A.shape[0])
    u, iters, rel, _ = amg.solve(H, b, tol=1e-12, omega_pre=1.0, omega_post=0.5)
    assert rel < 1e-12 and iters <= 8
