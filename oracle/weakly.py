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


def _element_integral(a, y0, y1, gamma):
    """int_{y0}^{y1} phi(y) |y|^{-gamma} dy for phi = a0 + a1 u + a2 u^2, u = y - y0.

    Near the singularity (an end within 4 of y = 0) the closed-form antiderivatives of the
    polynomial in y are exact and well conditioned; farther away they cancel (terms of size
    |y|^{3-gamma} against a result of size |y|^{-gamma}), while the integrand is smooth on the
    element, so 20-point Gauss-Legendre quadrature is used with phi evaluated in u."""
    if y0 >= 4.0 or y1 <= -4.0:
        u = 0.5 * (y1 - y0) * (_GL_X + 1.0)
        vals = (a[0] + u * (a[1] + u * a[2])) * np.abs(y0 + u) ** (-gamma)
        return float(0.5 * (y1 - y0) * np.dot(_GL_W, vals))
    c = (a[0] - a[1] * y0 + a[2] * y0 * y0, a[1] - 2 * a[2] * y0, a[2])
    tot = 0.0
    if y1 > 0.0:
        tot += _antideriv(c, gamma, y1) - _antideriv(c, gamma, max(y0, 0.0))
    if y0 < 0.0:  # y = -t
        cm = (c[0], -c[1], c[2])
        tot += _antideriv(cm, gamma, -y0) - _antideriv(cm, gamma, -min(y1, 0.0))
    return tot


def _basis_pieces(q2: int, N: int):
    """Pieces of the basis function at twice-coordinate q2 (units of h/2) on [0, N]:
    (y0, y1, (a0, a1, a2)) with phi = a0 + a1 u + a2 u^2, u = y - y0 (y in units of h)."""
    c = q2 / 2.0
    if q2 % 2 == 0:  # node: t (2t - 1), t = distance to the far end of each element
        out = []
        if c - 1 >= 0:
            out.append((c - 1, c, (0.0, -1.0, 2.0)))      # 2u^2 - u
        if c + 1 <= N:
            out.append((c, c + 1, (1.0, -3.0, 2.0)))      # (1 - u)(1 - 2u)
        return out
    return [(c - 0.5, c + 0.5, (0.0, 4.0, -4.0))]         # midpoint: 4 u (1 - u)


def coupling(p2: int, q2: int, N: int, gamma: float) -> float:
    """(3-gamma)(2-gamma)(1-gamma) int phi_q(y) |x_p - y|^{-gamma} dy / h^{1-gamma}, i.e.
    eta_{h,gamma} times the integral, at twice-coordinates p2 (collocation point) and q2."""
    xp = p2 / 2.0
    tot = 0.0
    for y0, y1, a in _basis_pieces(q2, N):
        tot += _element_integral(a, y0 - xp, y1 - xp, gamma)
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
