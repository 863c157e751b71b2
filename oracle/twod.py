"""2-D Toeplitz-like-plus-Cross systems (the 2-D configuration; not defined by the paper).

Test infrastructure only (see the package docstring).

The paper builds the 1-D collocation systems of section 2.2 and leaves the 2-D case to cited
companion work. The reading taken here (PARITY UNPINNED by the paper; pinned by mathematics, see
tests/test_oracle_twod.py):

* domain (0, 1)^2, constant kernel on a SQUARE horizon [-delta, delta]^2 (the l-infinity ball),
  -L u(x) = gamma * integral over the square of [u(x) - u(x + s)] ds;
* tensor-product piecewise-quadratic collocation: the unknowns are the products of the 1-D
  unknowns of section 2.2 (nodes then midpoints on each axis), U[i, j] at (x_i, y_j), and the
  vector is U flattened row by row (i slow, j fast);
* the same scaling as 1-D, in units of h: an entry is 6 / (2 delta) times
  [ (2 delta)^2 delta_{(i,j),(p,q)} - integral over the square of phi_p(x_i + s1) phi_q(y_j + s2) ],
  so that the 1-D matrix's largest entries and the 2-D ones have the same size. With the 1-D
  integrals S[i, p] = integral_{-delta}^{delta} phi_p(x_i + s) ds (the square factorises),
  M = S / (2 delta) and d = 12 r (delta = r h):  A2 = d (I (x) I - M (x) M).
  The 1-D matrix is A1 = 6 (2 delta I - S) / h = d (I - M), hence also
  A2 = A1 (x) I + I (x) A1 - (A1 (x) A1) / d;
* SPD variant: both axes use the shifted-symmetric rows of section 2.2.2; nonsymmetric variant:
  both axes use the nonsymmetric collocation of section 2.2.1;
* transfers: the 1-D full weighting on the concatenated vector (section 3.1) on each axis,
  R2 = R (x) R, P2 = P (x) P = 4 R2^T; Galerkin coarse operators R2 A2 P2 (eq. (3.2));
  damped Jacobi with the diagonal of A2 (eq. (3.3)); dense LU at the coarsest level.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sps

from . import amg
from .model import NONSYM, SPD, _basis_pieces, _integral


def points(N: int):
    """The 1-D unknowns in units of h (nodes 1..N-1, then midpoints 1/2..N-1/2), as
    (coordinate, is_node)."""
    return [(Fraction(i), True) for i in range(1, N)] + \
           [(Fraction(2 * i - 1, 2), False) for i in range(1, N + 1)]


def _basis_type(variant: int, row_is_node: bool, col_is_node: bool) -> bool:
    """Node-type basis for column q at row p: the SPD system collocates midpoint rows on the
    mesh shifted by h/2, where midpoints carry the node-type basis (section 2.2.2)."""
    if variant == SPD and not row_is_node:
        return not col_is_node
    return col_is_node


def integral_row(variant: int, xp: Fraction, row_is_node: bool, cols, r: int) -> list:
    """S[p, q] = integral_{-r}^{r} phi_q(x_p + s) ds (units of h, exact) for the columns cols."""
    out = []
    for xq, col_is_node in cols:
        pieces = _basis_pieces(xq, _basis_type(variant, row_is_node, col_is_node))
        out.append(_integral(pieces, xp - r, xp + r))
    return out


def integral_matrix(variant: int, N: int, r: int) -> np.ndarray:
    """S (n x n, n = 2N - 1) over the interior unknowns."""
    pts = points(N)
    return np.array([[float(v) for v in integral_row(variant, xp, isn, pts, r)]
                     for xp, isn in pts])


def assemble(variant: int, N: int, r: int) -> np.ndarray:
    """Dense 2-D matrix d (I (x) I - M (x) M), n^2 x n^2, from the exact 1-D integrals."""
    if variant not in (SPD, NONSYM):
        raise ValueError("variant")
    S = integral_matrix(variant, N, r)
    M = S / (2.0 * r)
    n = S.shape[0]
    return 12.0 * r * (np.eye(n * n) - np.kron(M, M))


def full_stencil_apply(variant: int, N: int, r: int, f) -> np.ndarray:
    """The 2-D collocation operator with its exterior couplings, applied to samples of f(x, y)
    (coordinates in units of h) on every grid point within reach: entry (i, j) is
    d [f(x_i, y_j) - (1 / (2r)^2) sum_{q, q'} S[i, q] S[j, q'] f(x_q, y_q')], q over all nodes and
    midpoints of the extended 1-D grid (the interior and the collar of width r)."""
    pts = points(N)
    ext = [(Fraction(k, 2), k % 2 == 0) for k in range(-2 * r - 2, 2 * N + 2 * r + 3)]
    Sx = np.array([[float(v) for v in integral_row(variant, xp, isn, ext, r)] for xp, isn in pts])
    coords = np.array([float(x) for x, _ in ext])
    F = np.array([[f(a, b) for b in coords] for a in coords])
    own = np.array([[f(float(a), float(b)) for b, _ in pts] for a, _ in pts])
    return 12.0 * r * (own - Sx @ F @ Sx.T / (2.0 * r) ** 2)


def restriction(n_fine: int) -> sps.csr_matrix:
    """R2 = R (x) R with the 1-D restriction of section 3.1 on each axis (sparse)."""
    R = amg.restriction_sparse(n_fine)
    return sps.kron(R, R, format="csr")


def galerkin(A: np.ndarray, n_fine: int) -> np.ndarray:
    """R2 A P2 with P2 = P (x) P = 4 R2^T (eq. (3.2) on each axis)."""
    R2 = restriction(n_fine)
    RA = np.asarray(R2 @ A)
    return 4.0 * np.ascontiguousarray(np.asarray(R2 @ RA.T).T)


class Hierarchy:
    """Dense 2-D level matrices A2_K..A2_kc (level k: n_k^2 unknowns, n_k = 2^(k+1) - 1) and
    the LU factors of the coarsest one."""

    def __init__(self, A_fine: np.ndarray, kc: int = 3):
        nn = A_fine.shape[0]
        n = int(round(np.sqrt(nn)))
        K = int(round(np.log2(n + 1))) - 1
        if n * n != nn or (1 << (K + 1)) - 1 != n or not (1 <= kc <= K):
            raise ValueError("finest size must be (2^(K+1) - 1)^2 and 1 <= kc <= K")
        self.K, self.kc = K, kc
        self.A = {K: A_fine}
        for k in range(K, kc, -1):
            self.A[k - 1] = galerkin(self.A[k], (1 << (k + 1)) - 1)
        self.lu = sla.lu_factor(self.A[kc])


def vcycle(H: Hierarchy, k: int, b: np.ndarray, m1: int = 1, m2: int = 1,
           omega_pre: float = 2.0 / 3.0, omega_post: float = 2.0 / 3.0) -> np.ndarray:
    """Algorithm 2 with the 2-D transfers: m1 damped Jacobi sweeps from 0, the coarse-grid
    correction with R2 and P2 = 4 R2^T, m2 sweeps; LU at the coarsest level."""
    if k == H.kc:
        return sla.lu_solve(H.lu, b)
    A = H.A[k]
    dg = np.diag(A)
    u = np.zeros_like(b)
    for _ in range(m1):
        u = u + omega_pre * (b - A @ u) / dg
    R2 = restriction((1 << (k + 1)) - 1)
    e = vcycle(H, k - 1, R2 @ (b - A @ u), m1, m2, omega_pre, omega_post)
    u = u + 4.0 * (R2.T @ e)
    for _ in range(m2):
        u = u + omega_post * (b - A @ u) / dg
    return u


def solve(H: Hierarchy, b: np.ndarray, tol: float = 1e-10, max_iters: int = 100):
    """Outer iteration u += B (b - A u) from u = 0 until ||r||_2 / ||b||_2 < tol (section 5).
    Returns (u, iterations, relres, iterates)."""
    A = H.A[H.K]
    u = np.zeros_like(b)
    r = b.copy()
    r0 = np.linalg.norm(r)
    rel = 1.0 if r0 > 0 else 0.0
    it, iterates = 0, []
    while rel >= tol and it < max_iters:
        u = u + vcycle(H, H.K, r)
        r = b - A @ u
        rel = np.linalg.norm(r) / r0
        it += 1
        iterates.append(u.copy())
    return u, it, rel, iterates


def matvec_large(variant: int, N: int, r: int, u: np.ndarray) -> np.ndarray:
    """A2 u for sizes where the dense matrix does not fit: d (U - M U M^T) with
    M = I - A1 / d applied by the FFT-convolution product of the printed 1-D blocks."""
    from . import large
    n = 2 * N - 1
    d = 12.0 * r
    U = u.reshape(n, n)

    def m_rows(X):  # X M^T: M applied to every row
        return X - np.stack([large.matvec(variant, N, r, row) for row in X]) / d

    W = m_rows(U)                  # U M^T
    V = m_rows(W.T.copy()).T       # M (U M^T)
    return (d * (U - V)).ravel()
