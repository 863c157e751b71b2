"""Block V-cycle AMG of section 3 with dense matrices, FP64.

Test infrastructure only (see the package docstring).

Levels are numbered as in section 3.1: level k has N_k = 2^k - 1 and n_k = 2 N_k + 1
unknowns (the concatenated vector [v; w], eq. before Algorithm 2); the finest level K has
N = 2^K intervals. The coarsest level kc is solved with a dense LU (Algorithm 2 defines
B_1 = A_1^{-1}; the coarsest level is a parameter, default 3).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sps


def restriction(n_fine: int) -> np.ndarray:
    """I_k^{k-1} = 1/4 [1 2 1] stencil rows (section 3.1), dense (n_c x n_f), n_c = (n_f-1)/2.

    Row I (1-based) holds 1/4, 1/2, 1/4 at columns 2I-1, 2I, 2I+1 of the concatenated
    fine vector.
    """
    n_c = (n_fine - 1) // 2
    R = np.zeros((n_c, n_fine))
    for I in range(1, n_c + 1):
        R[I - 1, 2 * I - 2] = 0.25
        R[I - 1, 2 * I - 1] = 0.5
        R[I - 1, 2 * I] = 0.25
    return R


def prolongation(n_fine: int) -> np.ndarray:
    """I_{k-1}^k = 2 (I_k^{k-1})^T (section 3.1)."""
    return 2.0 * restriction(n_fine).T


def position_order(n: int) -> np.ndarray:
    """Concatenated indices [v; w] of a level with n = 2N + 1 unknowns, listed by position:
    node v_i sits at x = i h (i = 1..N), midpoint w_j at x = (j - 1/2) h (j = 1..N+1)."""
    N = (n - 1) // 2
    x = np.concatenate([np.arange(1, N + 1), np.arange(1, N + 2) - 0.5])
    return np.argsort(x, kind="stable")


def restriction_geometric(n_fine: int) -> np.ndarray:
    """Not the paper's transfer: the same 1/4 [1 2 1] rows applied to the unknowns listed by
    position (spacing h/2), the coarse unknowns being the fine nodes x = I h, which are the
    nodes and midpoints of the coarse mesh. Returned in the concatenated orderings of both
    levels: R[pc, pf] with the rows / columns permuted by position_order. PARITY UNPINNED by
    the paper (pinned by mathematics only: tests/test_oracle_geometric.py)."""
    n_c = (n_fine - 1) // 2
    pf, pc = position_order(n_fine), position_order(n_c)
    R = np.zeros((n_c, n_fine))
    R[np.ix_(pc, pf)] = restriction(n_fine)
    return R


TRANSFERS = {"paper": restriction, "geometric": restriction_geometric}


def restriction_sparse(n_fine: int, transfer: str = "paper") -> sps.csr_matrix:
    """The restriction of ``restriction`` (or ``restriction_geometric``) held as a sparse
    matrix: the same three entries 1/4, 1/2, 1/4 per row at the same columns, so that the
    Galerkin product of a dense A_k costs O(n^2) instead of O(n^3)."""
    n_c = (n_fine - 1) // 2
    I = np.arange(n_c)
    rows = np.repeat(I, 3)
    cols = (2 * I[:, None] + np.arange(3)[None, :]).ravel()
    vals = np.tile([0.25, 0.5, 0.25], n_c)
    if transfer == "geometric":
        pf, pc = position_order(n_fine), position_order(n_c)
        rows, cols = pc[rows], pf[cols]
    elif transfer != "paper":
        raise ValueError("transfer")
    return sps.csr_matrix((vals, (rows, cols)), shape=(n_c, n_fine))


def galerkin(A: np.ndarray, transfer: str = "paper") -> np.ndarray:
    """A_{k-1} = I_k^{k-1} A_k I_{k-1}^k (eq. (3.2), eq. (3.6)), I_{k-1}^k = 2 (I_k^{k-1})^T.

    Each coarse entry is the sum of the nine fine entries the restriction rows select,
    (1/8) sum_{a,b} w_a w_b A_k(2I+a, 2J+b); the sparse restriction forms exactly those sums."""
    R = restriction_sparse(A.shape[0], transfer)
    RA = np.asarray(R @ A)                       # n_c x n_f
    return 2.0 * np.ascontiguousarray(np.asarray(R @ RA.T).T)


class Hierarchy:
    """Dense level matrices A_K..A_kc plus the LU factors of the coarsest one."""

    def __init__(self, A_fine: np.ndarray, kc: int = 3, transfer: str = "paper"):
        n = A_fine.shape[0]
        K = int(round(np.log2(n + 1))) - 1
        if (1 << (K + 1)) - 1 != n:
            raise ValueError("finest size must be 2^(K+1) - 1")
        if not (1 <= kc <= K):
            raise ValueError("coarsest level out of range")
        self.K, self.kc = K, kc
        self.transfer = transfer
        self.A = {K: A_fine}
        for k in range(K, kc, -1):
            self.A[k - 1] = galerkin(self.A[k], transfer)
        self.lu = sla.lu_factor(self.A[kc])

    def n(self, k: int) -> int:
        return (1 << (k + 1)) - 1


def vcycle(H: Hierarchy, k: int, b: np.ndarray, m1: int = 1, m2: int = 1,
           omega_pre: float = 2.0 / 3.0, omega_post: float = 2.0 / 3.0) -> np.ndarray:
    """Algorithm 2: returns B_k b with zero initial guess.

    1. pre-smooth m1 times: u <- u + omega_pre D^{-1} (b - A u)  (damped Jacobi, eq. (3.3);
       the update form is the standard one, the smoother being I - omega D^{-1} A);
    2. coarse-grid solution e = B_{k-1} I_k^{k-1} (b - A u);
    3. correction u <- u + I_{k-1}^k e;
    4. post-smooth m2 times with omega_post;
    5. B_k b = u.  At the coarsest level B_kc = A_kc^{-1} (dense LU).
    """
    if k == H.kc:
        return sla.lu_solve(H.lu, b)
    A = H.A[k]
    d = np.diag(A)
    u = np.zeros_like(b)
    for _ in range(m1):
        u = u + omega_pre * (b - A @ u) / d
    r = b - A @ u
    R = TRANSFERS[getattr(H, "transfer", "paper")](A.shape[0])
    e = vcycle(H, k - 1, R @ r, m1, m2, omega_pre, omega_post)
    u = u + 2.0 * R.T @ e
    for _ in range(m2):
        u = u + omega_post * (b - A @ u) / d
    return u


def solve(H: Hierarchy, b: np.ndarray, tol: float = 1e-10, max_iters: int = 100,
          x0: np.ndarray | None = None, **vc):
    """Outer iteration of section 5: u_{i+1} = u_i + B_K (b - A u_i) until
    ||r_i||_2 / ||r_0||_2 < tol, with r_0 = b - A u_0 (u_0 = 0 unless x0 is given).

    Returns (u, iterations, relres, list of iterates u_1, u_2, ...).
    """
    A = H.A[H.K]
    u = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - A @ u
    r0 = np.linalg.norm(r)
    iterates = []
    rel = np.linalg.norm(r) / r0 if r0 > 0 else 0.0
    it = 0
    while rel >= tol and it < max_iters:
        u = u + vcycle(H, H.K, r, **vc)
        r = b - A @ u
        rel = np.linalg.norm(r) / r0
        it += 1
        iterates.append(u.copy())
    return u, it, rel, iterates


# ----------------------------------------------------------------------------------------
# Cross splitting (eq. (3.7)) read off a dense level matrix
# ----------------------------------------------------------------------------------------

def split_cross(M: np.ndarray) -> dict:
    """Split a level matrix (n = 2 N_k + 1) as in eq. (3.7).

    Toeplitz blocks A (rows/cols 1..N), B_bar (rows 1..N, cols N+2..2N+1), C_bar, D_bar,
    returned as generators t[d] = T(i, j) for d = i - j in [-(N-1), N-1], stored at index
    d + N - 1 and read from the first column and first row. The Cross: p = column N+1 over
    rows 1..N, q = row N+1 over cols 1..N, o = entry (N+1, N+1), zeta = row N+1 over cols
    N+2.., xi = column N+1 over rows N+2...
    """
    n = M.shape[0]
    N = (n - 1) // 2

    def gen(T):
        g = np.empty(2 * N - 1)
        g[N - 1:] = T[:, 0]               # d = 0..N-1  -> T[d, 0]
        g[:N - 1] = T[0, 1:][::-1]        # d = -(N-1)..-1 -> T[0, -d]
        return g

    blocks = {"A": M[:N, :N], "B": M[:N, N + 1:], "C": M[N + 1:, :N], "D": M[N + 1:, N + 1:]}
    out = {k: gen(T) for k, T in blocks.items()}
    out["blocks"] = blocks
    out.update(p=M[:N, N].copy(), q=M[N, :N].copy(), o=float(M[N, N]),
               zeta=M[N, N + 1:].copy(), xi=M[N + 1:, N].copy(), N=N)
    return out


def is_toeplitz(T: np.ndarray, tol: float = 0.0) -> bool:
    """True if every diagonal of T is constant (to ``tol`` absolute)."""
    m, n = T.shape
    for d in range(-(n - 1), m):
        diag = np.diagonal(T, offset=-d)
        if diag.size and np.max(np.abs(diag - diag[0])) > tol:
            return False
    return True


# ----------------------------------------------------------------------------------------
# Two-grid factor of Theorem 4.1
# ----------------------------------------------------------------------------------------

def two_grid_factor(A: np.ndarray, omega: float, transfer: str = "paper") -> float:
    """||S_K T_K||_A with T_K = I - P A_c^{-1} R A and S_K = I - omega D^{-1} A (section 3.1).

    The A-norm of a matrix M is ||L^T M L^{-T}||_2 where A = L L^T (A must be SPD).
    """
    n = A.shape[0]
    R = TRANSFERS[transfer](n)
    P = 2.0 * R.T
    Ac = R @ A @ P
    T = np.eye(n) - P @ np.linalg.solve(Ac, R @ A)
    S = np.eye(n) - omega * (A / np.diag(A)[:, None])
    L = np.linalg.cholesky(A)
    M = L.T @ (S @ T) @ np.linalg.inv(L.T)
    return float(np.linalg.norm(M, 2))
