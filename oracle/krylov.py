"""Flexible GMRES with the V-cycle as its preconditioner: an outer iteration that is not the
paper's.

Test infrastructure only (see the package docstring).

The paper solves A u = b by the stationary iteration u <- u + B (b - A u), B one V-cycle of
Algorithm 2 (section 5). This module states the Krylov alternative the library offers as an
option: right-preconditioned flexible GMRES (Saad, "Iterative methods for sparse linear
systems", 2nd ed., section 9.4.1), restarted after `steps` steps with the true residual formed
again, i.e. per restart cycle from the iterate u:

    r = b - A u,  beta = ||r||,  v_0 = r / beta
    for j = 0 .. steps-1:
        z_j = B v_j                         (one V-cycle, zero initial guess)
        w = A z_j
        h_{:j} = V_j^T w, w -= V_j h_{:j}   (classical Gram-Schmidt, done twice: the second
        h'     = V_j^T w, w -= V_j h'        pass's coefficients are added to the first's)
        h_{j+1,j} = ||w||,  v_{j+1} = w / h_{j+1,j}  (0 if h_{j+1,j} = 0)
    y = argmin || beta e_1 - Hbar y ||  (Givens rotations on the (steps+1) x steps Hessenberg
                                          matrix Hbar; a zero pivot gives y_j = 0)
    u <- u + Z y.

The library runs exactly these steps (its parity tests compare iterates); the pins are the
defining properties of GMRES: with a fixed linear B the residual after j steps is the
smallest over u + span{B v_0, .., B v_{j-1}} = u + B K_j(A B, r) (checked against an
explicit least-squares problem on that space), n steps solve an n x n system exactly, and
B = A^{-1} solves in one step.
"""
from __future__ import annotations

import numpy as np


def _rotation(a: float, b: float):
    """Givens rotation (c, s) with [c s; -s c] [a; b] = [r; 0], r >= 0 (c = 1, s = 0 if a = b = 0)."""
    r = float(np.hypot(a, b))
    if r == 0.0:
        return 1.0, 0.0, 0.0
    return a / r, b / r, r


def restart_cycle(A, b: np.ndarray, u: np.ndarray, prec, steps: int):
    """One restart cycle of FGMRES(steps) from u. Returns (u_new, estimated residual norm
    |g_steps| of the least-squares problem, list of the Hessenberg columns)."""
    r = b - A @ u
    beta = float(np.linalg.norm(r))
    n = b.size
    V = np.zeros((steps + 1, n))
    Z = np.zeros((steps, n))
    Hbar = np.zeros((steps + 1, steps))
    cs, sn = np.zeros(steps), np.zeros(steps)
    g = np.zeros(steps + 1)
    g[0] = beta
    if beta == 0.0:
        return u.copy(), 0.0, Hbar
    V[0] = r / beta
    for j in range(steps):
        Z[j] = prec(V[j])
        w = A @ Z[j]
        h = V[: j + 1] @ w
        w = w - h @ V[: j + 1]
        h2 = V[: j + 1] @ w
        w = w - h2 @ V[: j + 1]
        col = np.zeros(steps + 1)
        col[: j + 1] = h + h2
        col[j + 1] = float(np.linalg.norm(w))
        Hbar[:, j] = col
        V[j + 1] = w / col[j + 1] if col[j + 1] > 0.0 else 0.0
        # the earlier rotations, then a new one that zeroes the subdiagonal entry
        for i in range(j):
            t = cs[i] * col[i] + sn[i] * col[i + 1]
            col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1]
            col[i] = t
        cs[j], sn[j], col[j] = _rotation(col[j], col[j + 1])
        col[j + 1] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        Hbar[:, j] = col  # now the j-th column of the triangular factor R
    # back substitution R y = g[:steps]
    y = np.zeros(steps)
    for i in range(steps - 1, -1, -1):
        s = g[i] - Hbar[i, i + 1:steps] @ y[i + 1:]
        y[i] = s / Hbar[i, i] if Hbar[i, i] != 0.0 else 0.0
    return u + y @ Z, abs(g[steps]), Hbar


def solve(A, b: np.ndarray, prec, steps: int, tol: float = 1e-10, max_restarts: int = 100,
          x0: np.ndarray | None = None):
    """Restarted FGMRES(steps) until ||b - A u|| / ||b - A u_0|| < tol. Returns (u, restarts,
    relres, list of the iterates after each restart)."""
    u = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r0 = float(np.linalg.norm(b - A @ u))
    rel = 1.0 if r0 > 0 else 0.0
    its, iterates = 0, []
    while rel >= tol and its < max_restarts:
        u, _, _ = restart_cycle(A, b, u, prec, steps)
        rel = float(np.linalg.norm(b - A @ u)) / r0
        its += 1
        iterates.append(u.copy())
    return u, its, rel, iterates
