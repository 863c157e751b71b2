"""The weakly singular nonlocal model of section 2.1 (eq. (2.3)) and its time stepping.

Test infrastructure only (see the package docstring).

Problem: u_t + L u = f on (0, 1), L u(x) = int_0^1 (u(x) - u(y)) |x - y|^{-gamma} dy,
0 <= gamma < 1, u given at x = 0 and x = 1. (Section 2.1 writes u_t - L u with this L; the
sign that gives a well-posed problem, and the one that reproduces Table 1, is u_t + L u.)
Piecewise quadratic collocation at the nodes x_j = j h and midpoints x_{j-1/2} (the unknown
ordering of eq. (2.3): nodes 1..N-1, then midpoints 1/2..N-1/2), scaled by
eta_{h,gamma} = (3-gamma)(2-gamma)(1-gamma) / h^{1-gamma}:

    A_h U = eta_{h,gamma} F + K,    A_h = diag(D_1, D_2) - [M Q; P N],

where the diagonal is eta times int_0^1 |x_p - y|^{-gamma} dy, every entry of [M Q; P N] is
eta times int phi_q(y) |x_p - y|^{-gamma} dy, and K holds the same integrals of the two
boundary basis functions times u(0), u(1). All of them are computed here as exact integrals
of a quadratic times |s|^{-gamma} over each element: closed-form antiderivatives of the powers
of |s| on every element, evaluated in 40-digit arithmetic (no quadrature rule).

Readings of the printed formulas (pinned in tests/test_oracle_weakly.py): the printed d_{i/2},
m_k, n_k, q_k and p_k (k >= 1) equal these integrals; the printed p_0 and eta_{i/2} (i >= 2) do
not (they match no entry of the matrix); and the right-hand side is eta F + K with K unscaled
(the printed eta (F + K) scales K twice). With these readings the BDF4 errors of Table 1 are
reproduced.
"""
from __future__ import annotations

import math
from functools import lru_cache

import mpmath
import numpy as np

_DPS = 40  # decimal digits of the exact antiderivatives' evaluation


def _antideriv(coeffs, gamma, s):
    """Antiderivative at s >= 0 of sum_k coeffs[k] s^{k - gamma} (mpmath numbers; 0 at s = 0,
    every exponent k + 1 - gamma being positive)."""
    if s == 0:
        return mpmath.mpf(0)
    return sum(c * s ** (k + 1 - gamma) / (k + 1 - gamma) for k, c in enumerate(coeffs))


def _element_integral(a, y0, y1, gamma):
    """int_{y0}^{y1} phi(y) |y|^{-gamma} dy for phi = a0 + a1 u + a2 u^2, u = y - y0.

    Exact: phi is rewritten in powers of y, split at y = 0 into powers of |y|, and integrated with
    the closed-form antiderivatives, evaluated in 40-digit arithmetic. Far from the singularity
    the terms (size |y|^{3-gamma}) cancel down to the result (size |y|^{-gamma}); at 40 digits
    that costs at most log10(|y|^3) digits, so the result is exact to double precision at every
    distance, with no quadrature rule involved."""
    with mpmath.workdps(_DPS):
        g = mpmath.mpf(gamma)
        y0m, y1m = mpmath.mpf(y0), mpmath.mpf(y1)
        a0, a1, a2 = (mpmath.mpf(v) for v in a)
        c = (a0 - a1 * y0m + a2 * y0m * y0m, a1 - 2 * a2 * y0m, a2)
        tot = mpmath.mpf(0)
        if y1m > 0:
            tot += _antideriv(c, g, y1m) - _antideriv(c, g, max(y0m, mpmath.mpf(0)))
        if y0m < 0:  # y = -t
            cm = (c[0], -c[1], c[2])
            tot += _antideriv(cm, g, -y0m) - _antideriv(cm, g, -min(y1m, mpmath.mpf(0)))
        return float(tot)


@lru_cache(maxsize=None)
def _coupling_rel(d2: int, q_odd: bool, left: bool, right: bool, gamma: float) -> float:
    """The integral of coupling for a basis function at twice-distance d2 = q2 - p2 from the
    collocation point: it depends only on d2, the basis type and whether the basis function is
    cut at x = 0 (left) or x = 1 (right)."""
    c = d2 / 2.0  # centre of the basis function relative to the collocation point (units of h)
    if q_odd:  # midpoint: 4 u (1 - u) on [c - 1/2, c + 1/2], u = y - (c - 1/2)
        pieces = [(c - 0.5, c + 0.5, (0.0, 4.0, -4.0))]
    else:      # node: 2u^2 - u on [c - 1, c] and (1 - u)(1 - 2u) on [c, c + 1], u = y - lower end
        pieces = []
        if not left:
            pieces.append((c - 1, c, (0.0, -1.0, 2.0)))
        if not right:
            pieces.append((c, c + 1, (1.0, -3.0, 2.0)))
    return sum(_element_integral(a, y0, y1, gamma) for y0, y1, a in pieces)


def coupling(p2: int, q2: int, N: int, gamma: float) -> float:
    """(3-gamma)(2-gamma)(1-gamma) int phi_q(y) |x_p - y|^{-gamma} dy / h^{1-gamma}, i.e.
    eta_{h,gamma} times the integral, at twice-coordinates p2 (collocation point) and q2."""
    tot = _coupling_rel(q2 - p2, q2 % 2 == 1, q2 == 0, q2 == 2 * N, float(gamma))
    return (3 - gamma) * (2 - gamma) * (1 - gamma) * tot


def points(N: int):
    """Twice-coordinates of the unknowns: nodes 2, 4, .., 2N-2, then midpoints 1, 3, .., 2N-1."""
    return [2 * i for i in range(1, N)] + [2 * i - 1 for i in range(1, N + 1)]


def diagonal(N: int, gamma: float) -> np.ndarray:
    """eta_{h,gamma} int_0^1 |x_p - y|^{-gamma} dy = (3-gamma)(2-gamma)((x_p/h)^{1-gamma} +
    ((1-x_p)/h)^{1-gamma}) at the unknowns."""
    x = np.array(points(N)) / 2.0
    return (3 - gamma) * (2 - gamma) * (x ** (1 - gamma) + (N - x) ** (1 - gamma))


def assemble(N: int, gamma: float) -> np.ndarray:
    """Dense A_h = diag(D_1, D_2) - [M Q; P N] of eq. (2.3)."""
    pts = points(N)
    T = np.array([[coupling(p, q, N, gamma) for q in pts] for p in pts])
    return np.diag(diagonal(N, gamma)) - T


def boundary_columns(N: int, gamma: float):
    """K = K0 u(0) + KN u(1): the couplings of the boundary basis functions."""
    pts = points(N)
    return (np.array([coupling(p, 0, N, gamma) for p in pts]),
            np.array([coupling(p, 2 * N, N, gamma) for p in pts]))


def eta(N: int, gamma: float) -> float:
    return (3 - gamma) * (2 - gamma) * (1 - gamma) * N ** (1 - gamma)


def phi(x):
    """Spatial factor (1 + x)^6 of the exact solution of section 5."""
    return (1.0 + x) ** 6


def L_phi(x, gamma):
    """L phi for phi = (1 + x)^6 in closed form: with phi(x) - phi(y) = -sum_k c_k (y - x)^k,
    int_0^1 (y - x)^k |y - x|^{-gamma} dy = ((1-x)^{k+1-gamma} + (-1)^k x^{k+1-gamma})
    / (k+1-gamma)."""
    s = 0.0
    for k in range(1, 7):
        ck = math.comb(6, k) * (1.0 + x) ** (6 - k)
        s -= ck * ((1.0 - x) ** (k + 1 - gamma) + (-1) ** k * x ** (k + 1 - gamma)) / (k + 1 - gamma)
    return s


def bdf4(N: int, gamma: float, T: float = 1.0):
    """Eq. (5.1) with tau = h for u = e^t (1 + x)^6 from the exact U^0..U^3: each step solves
    (sigma I + A_h) U^k = (eta / tau) hist + e^{t_k} (eta (phi + L phi) + K0 phi(0) + KN phi(1)),
    sigma = 25 eta / (12 tau). Returns (max-norm error at T, U_T)."""
    tau = 1.0 / N
    steps = int(round(T / tau))
    e = eta(N, gamma)
    A = assemble(N, gamma)
    M = A + 25.0 * e / (12.0 * tau) * np.eye(A.shape[0])
    K0, KN = boundary_columns(N, gamma)
    x = np.array(points(N)) / (2.0 * N)
    G = e * (phi(x) + L_phi(x, gamma)) + K0 * phi(0.0) + KN * phi(1.0)
    U = [np.exp(j * tau) * phi(x) for j in range(4)]
    for k in range(4, steps + 1):
        hist = 4.0 * U[-1] - 3.0 * U[-2] + (4.0 / 3.0) * U[-3] - 0.25 * U[-4]
        U.append(np.linalg.solve(M, (e / tau) * hist + np.exp(k * tau) * G))
        U.pop(0)
    return float(np.max(np.abs(U[-1] - np.exp(steps * tau) * phi(x)))), U[-1]
