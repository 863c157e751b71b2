"""The weakly singular nonlocal model of section 2.1 (eq. (3system)) and its time stepping.

Test infrastructure only (see the package docstring).

Problem: u_t + L u = f on (0, 1), L u(x) = int_0^1 (u(x) - u(y)) |x - y|^{-gamma} dy,
0 <= gamma < 1, u given at x = 0 and x = 1. (Section 2.1 writes u_t - L u with this L; the
sign that gives a well-posed problem, and the one that reproduces Table 1, is u_t + L u.)
Piecewise quadratic collocation at the nodes x_j = j h and midpoints x_{j-1/2} (the unknown
ordering of eq. (3system): nodes 1..N-1, then midpoints 1/2..N-1/2), scaled by
eta_{h,gamma} = (3-gamma)(2-gamma)(1-gamma) / h^{1-gamma}:

    A_h U = eta_{h,gamma} F + K,    A_h = diag(D_1, D_2) - [M Q; P N],

where the diagonal is eta times int_0^1 |x_p - y|^{-gamma} dy, every entry of [M Q; P N] is
eta times int phi_q(y) |x_p - y|^{-gamma} dy, and K holds the same integrals of the two
boundary basis functions times u(0), u(1). All of them are computed here as exact integrals
of a quadratic times |s|^{-gamma} over each element (closed-form antiderivatives next to the
singularity, 20-point Gauss-Legendre on the smooth far elements).

Readings of the printed formulas (pinned in tests/test_oracle_weakly.py): the printed d_{i/2},
m_k, n_k, q_k and p_k (k >= 1) equal these integrals; the printed p_0 and eta_{i/2} (i >= 2) do
not (they match no entry of the matrix); and the right-hand side is eta F + K with K unscaled
(the printed eta (F + K) scales K twice). With these readings the BDF4 errors of Table 1 are
reproduced.
"""
from __future__ import annotations

import math

import numpy as np


def _antideriv(coeffs, gamma, s):
    """Antiderivative at s >= 0 of sum_k coeffs[k] s^{k - gamma}."""
    return sum(c * s ** (k + 1 - gamma) / (k + 1 - gamma) for k, c in enumerate(coeffs))


_GL_X, _GL_W = np.polynomial.legendre.leggauss(20)


def _int_poly_weight(c, lo, hi, gamma):
    """int_lo^hi (c0 + c1 s + c2 s^2) |s|^{-gamma} ds for lo < hi (units of h).

    Near the singularity (an end within 4 of s = 0) the closed-form antiderivatives are exact
    and well conditioned; farther away they cancel (terms of size |s|^{3-gamma} against a result
    of size |s|^{-gamma}), and the integrand is smooth on the element, so 20-point
    Gauss-Legendre quadrature (exact to rounding for this smooth weight) is used instead."""
    if lo >= 4.0 or hi <= -4.0:
        ys = 0.5 * (hi - lo) * _GL_X + 0.5 * (hi + lo)
        vals = (c[0] + c[1] * ys + c[2] * ys * ys) * np.abs(ys) ** (-gamma)
        return float(0.5 * (hi - lo) * np.dot(_GL_W, vals))
    tot = 0.0
    if hi > 0.0:
        tot += _antideriv(c, gamma, hi) - _antideriv(c, gamma, max(lo, 0.0))
    if lo < 0.0:  # s = -t
        cm = (c[0], -c[1], c[2])
        tot += _antideriv(cm, gamma, -lo) - _antideriv(cm, gamma, -min(hi, 0.0))
    return tot


def _basis_pieces(q2: int, N: int):
    """Pieces of the basis function at twice-coordinate q2 (units of h/2) on [0, N]:
    (y0, y1, A, B, C) with phi(y) = A + B y + C y^2 on [y0, y1] (y in units of h)."""
    c = q2 / 2.0
    if q2 % 2 == 0:  # node: t(2t - 1) with t = y - (c - 1) on the left, t = (c + 1) - y right
        out = []
        if c - 1 >= 0:
            a = -(c - 1)
            out.append((c - 1, c, 2 * a * a - a, 4 * a - 1, 2.0))
        if c + 1 <= N:
            a = c + 1
            out.append((c, c + 1, 2 * a * a - a, -4 * a + 1, 2.0))
        return out
    # midpoint: 4 (y - (c - 1/2)) ((c + 1/2) - y)
    return [(c - 0.5, c + 0.5, -4.0 * (c * c - 0.25), 8.0 * c, -4.0)]


def coupling(p2: int, q2: int, N: int, gamma: float) -> float:
    """(3-gamma)(2-gamma)(1-gamma) int phi_q(y) |x_p - y|^{-gamma} dy / h^{1-gamma}, i.e.
    eta_{h,gamma} times the integral, at twice-coordinates p2 (collocation point) and q2."""
    xp = p2 / 2.0
    tot = 0.0
    for y0, y1, A, B, C in _basis_pieces(q2, N):
        # the piece as a polynomial in s = y - xp, built around the element's own left end
        # (local coordinate u = y - y0 keeps the coefficients small): phi = a0 + a1 u + a2 u^2
        a0 = A + B * y0 + C * y0 * y0
        a1 = B + 2 * C * y0
        a2 = C
        d = xp - y0  # y - y0 = s + d
        c = (a0 + a1 * d + a2 * d * d, a1 + 2 * a2 * d, a2)
        tot += _int_poly_weight(c, y0 - xp, y1 - xp, gamma)
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
    """Dense A_h = diag(D_1, D_2) - [M Q; P N] of eq. (3system)."""
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
    """Eq. (bdf4) with tau = h for u = e^t (1 + x)^6 from the exact U^0..U^3: each step solves
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
