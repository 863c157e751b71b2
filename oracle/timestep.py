"""Time-dependent problem of section 5: u_t = L_delta u + f on (0, 1) x (0, T], u = g on the
interaction domain, advanced by the BDF4 scheme of eq. (5.1).

Test infrastructure only (see the package docstring).

The collocation system of section 2.2 is A U = eta_h (-L_delta u)(x_p) - (exterior
couplings of g), with eta_h = 6/(gamma h) (the printed integer coefficients are eta_h times
the collocation of -L_delta). With the discrete operator L_delta U = -(A U + B_ext g) / eta_h,
eq. (5.1), (25/12 I - tau L_delta) U^k = 4 U^{k-1} - 3 U^{k-2} + 4/3 U^{k-3} - 1/4 U^{k-4}
+ tau F^k, multiplied by eta_h / tau reads

    (sigma I + A) U^k = (eta_h / tau) (4 U^{k-1} - 3 U^{k-2} + 4/3 U^{k-3} - 1/4 U^{k-4})
                        + eta_h F^k(x_p) - B_ext g^k,      sigma = 25 eta_h / (12 tau).

The test problem of section 5 has the exact solution u = e^t (1 + x)^6, so F = u_t - L_delta u
= e^t (phi - L_delta phi) with phi = (1 + x)^6 and g^k = e^{t_k} phi: the source part of step
k is e^{t_k} G with one vector G. The kernel constant is the paper's gamma = 3 / delta^3 with
delta = r h (the horizon the stencil resolves). The first four levels are the exact solution
(the paper does not say how they were obtained); tau = h as in Tables 2 and 3. Each step is a
dense LU solve (the matrix does not change with k).
"""
from __future__ import annotations

import numpy as np

from . import model


def phi(x):
    """Spatial factor (1 + x)^6 of the exact solution of section 5."""
    return (1.0 + x) ** 6


def phi_antiderivative(x):
    return (1.0 + x) ** 7 / 7.0


def eta_h(N: int, r: int, gamma: float | None = None) -> float:
    """eta_h = 6 / (gamma h), gamma = 3 / delta^3 by default (delta = r h)."""
    h = 1.0 / N
    if gamma is None:
        gamma = 3.0 / (r * h) ** 3
    return 6.0 / (gamma * h)


def source_vector(variant: int, N: int, r: int, gamma: float | None = None) -> np.ndarray:
    """G = eta_h (phi - L_delta phi)(x_p) - B_ext phi: the source part of every step, per unit
    e^{t_k}."""
    b, _ = model.manufactured_rhs(variant, N, r, phi, phi_antiderivative)  # eta_h (-L phi) - B g
    x = model.collocation_points(N)
    return eta_h(N, r, gamma) * phi(x) + b


def bdf4(variant: int, N: int, r: int, T: float = 1.0, gamma: float | None = None):
    """Runs eq. (5.1) with tau = h from the exact starting values U^0..U^3 to t = T.

    Returns (error, U_T): the maximum-norm error at t = T and the final level."""
    h = 1.0 / N
    tau = h
    steps = int(round(T / tau))
    eta = eta_h(N, r, gamma)
    sigma = 25.0 * eta / (12.0 * tau)
    A = model.assemble(variant, N, r)
    M = A + sigma * np.eye(A.shape[0])
    G = source_vector(variant, N, r, gamma)
    x = model.collocation_points(N)
    U = [np.exp(j * tau) * phi(x) for j in range(4)]
    for k in range(4, steps + 1):
        hist = 4.0 * U[-1] - 3.0 * U[-2] + (4.0 / 3.0) * U[-3] - 0.25 * U[-4]
        U.append(np.linalg.solve(M, (eta / tau) * hist + np.exp(k * tau) * G))
        U.pop(0)
    err = float(np.max(np.abs(U[-1] - np.exp(steps * tau) * phi(x))))
    return err, U[-1]
