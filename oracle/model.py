"""Collocation matrices of the 1-D peridynamic model (section 2.2), dense, FP64.

Test infrastructure only (see the package docstring).

Unknown ordering (section 2.2.1, the grid function U_h): nodes u_1..u_{N-1} first, then
midpoints u_{1/2}..u_{N-1/2}; N = 1/h intervals, horizon ratio r = floor(delta/h) (r = 1
when delta <= h), section 2.2.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

SPD = 0      # shifted-symmetric system, section 2.2.2, eq. (2.10)
NONSYM = 1   # nonsymmetric indefinite system, section 2.2.1, eq. (2.9)


def horizon_ratio(delta: float, h: float) -> int:
    """r = floor(delta/h) if delta >= h, else r = 1 (section 2.2)."""
    if delta <= h:
        return 1
    return int(math.floor(delta / h))


# ----------------------------------------------------------------------------------------
# Printed coefficients
# ----------------------------------------------------------------------------------------

def coefficients(r: int) -> dict:
    """The printed stencil coefficients for horizon ratio r.

    a_0 = 12r-2, a_m = -2 (1<=m<=r-1), a_r = -1, a_{m+1/2} = -4 (0<=m<=r-1)   (section 2.2.1
    and eq. (2.11)); c_m = -2 (0<=m<=r-2), c_{r-1} = -9/4, c_r = 1/4;
    d_0 = 12r-4, d_m = -4 (1<=m<=r-1), d_r = -2 (section 2.2.1).

    Returned as arrays: ``a_int[m]`` = a_m (m=0..r), ``a_half[m]`` = a_{m+1/2} (m=0..r-1),
    ``c[m]`` (m=0..r), ``d[m]`` (m=0..r).
    """
    if r < 1:
        raise ValueError("r must be >= 1")
    a_int = np.full(r + 1, -2.0)
    a_int[0] = 12.0 * r - 2.0
    a_int[r] = -1.0
    a_half = np.full(r, -4.0)
    c = np.full(r + 1, -2.0)
    c[r - 1] = -9.0 / 4.0
    c[r] = 1.0 / 4.0
    d = np.full(r + 1, -4.0)
    d[0] = 12.0 * r - 4.0
    d[r] = -2.0
    return {"a_int": a_int, "a_half": a_half, "c": c, "d": d}


def toeplitz(col, row) -> np.ndarray:
    """Matlab-style toeplitz(col, row): T[i, j] = col[i-j] for i >= j, row[j-i] for j > i."""
    col = np.asarray(col, dtype=np.float64)
    row = np.asarray(row, dtype=np.float64)
    m, n = len(col), len(row)
    T = np.empty((m, n))
    for i in range(m):
        for j in range(n):
            T[i, j] = col[i - j] if i >= j else row[j - i]
    return T


def _fit(values, length: int) -> list:
    """Pad with zeros or truncate a coefficient list to ``length`` (the 0_{1 x k} blocks)."""
    v = list(values)[:length]
    return v + [0.0] * (length - len(v))


def assemble(variant: int, N: int, r: int) -> np.ndarray:
    """Dense matrix of eq. (2.9) (variant NONSYM) or eq. (2.10) (variant SPD).

    A = toeplitz(a_0..a_r, 0), (N-1)x(N-1);
    B = toeplitz([a_{1/2}..a_{r-1/2}, 0], [a_{1/2}, a_{1/2}, a_{3/2}..a_{r-1/2}, 0]), (N-1)xN;
    SPD:    C = B^T, D = A_hat = toeplitz(a_0..a_r, 0), NxN;
    NONSYM: C = toeplitz([c_0, c_0, c_1..c_r, 0], [c_0..c_r, 0]), Nx(N-1);
            D = toeplitz(d_0..d_r, 0), NxN.
    """
    cf = coefficients(r)
    a_int, a_half, c, d = cf["a_int"], cf["a_half"], cf["c"], cf["d"]
    colA = _fit(a_int, N - 1)
    A = toeplitz(colA, colA)
    B = toeplitz(_fit(a_half, N - 1), _fit([a_half[0]] + list(a_half), N))
    if variant == SPD:
        C = B.T.copy()
        colD = _fit(a_int, N)
        D = toeplitz(colD, colD)
    elif variant == NONSYM:
        C = toeplitz(_fit([c[0]] + list(c), N), _fit(c, N - 1))
        colD = _fit(d, N)
        D = toeplitz(colD, colD)
    else:
        raise ValueError("variant")
    return np.block([[A, B], [C, D]])


# ----------------------------------------------------------------------------------------
# Stencil by distance (used for rows that reach exterior points, i.e. the right-hand side)
# ----------------------------------------------------------------------------------------

def stencil_entry(variant: int, row_is_node: bool, dist2: int, r: int) -> float:
    """Entry coupling a collocation point to a grid point at distance dist2/2 (units of h).

    Integer rows (and all rows of the SPD system) use a_{dist}: integer distance m gives
    a_m, half-integer distance m+1/2 gives a_{m+1/2}. Midpoint rows of the nonsymmetric
    system couple to nodes (half-integer distance m+1/2) with c_m and to midpoints
    (integer distance m) with d_m. These are exactly the entries of the Toeplitz blocks
    printed in section 2.2, read as functions of the distance between points.
    """
    cf = coefficients(r)
    dist2 = abs(int(dist2))
    m, odd = divmod(dist2, 2)
    if row_is_node or variant == SPD:
        if odd:
            return float(cf["a_half"][m]) if m <= r - 1 else 0.0
        return float(cf["a_int"][m]) if m <= r else 0.0
    if odd:
        return float(cf["c"][m]) if m <= r else 0.0
    return float(cf["d"][m]) if m <= r else 0.0


# ----------------------------------------------------------------------------------------
# Independent assembly by exact quadrature of the quadratic basis (section 2)
# ----------------------------------------------------------------------------------------

def _basis_pieces(center: Fraction, node_type: bool):
    """Polynomial pieces of a basis function in units of h, as (lo, hi, f).

    Node type (phi_m, section 2): on [c-1, c], t = y-(c-1), phi = t(2t-1); on [c, c+1],
    s = (c+1)-y, phi = s(2s-1). Midpoint type (phi_{m-1/2}): 4(y-(c-1/2))((c+1/2)-y) on
    [c-1/2, c+1/2].
    """
    c = center
    if node_type:
        return [(c - 1, c, lambda y: (y - (c - 1)) * (2 * (y - (c - 1)) - 1)),
                (c, c + 1, lambda y: ((c + 1) - y) * (2 * ((c + 1) - y) - 1))]
    half = Fraction(1, 2)
    return [(c - half, c + half, lambda y: 4 * (y - (c - half)) * ((c + half) - y))]


def _integral(pieces, lo: Fraction, hi: Fraction) -> Fraction:
    """Exact integral over [lo, hi] of a piecewise quadratic (Simpson is exact on quadratics)."""
    total = Fraction(0)
    for a, b, f in pieces:
        x0, x1 = max(a, lo), min(b, hi)
        if x1 > x0:
            xm = (x0 + x1) / 2
            total += (x1 - x0) * (f(x0) + 4 * f(xm) + f(x1)) / 6
    return total


def quadrature_entry(variant: int, row_x: Fraction, row_is_node: bool, col_x: Fraction,
                     r: int) -> Fraction:
    """(6/h) * integral over |s| < delta of [phi_q(x_p) - phi_q(x_p + s)] ds, delta = r h.

    This is the collocation of -L_delta u (section 2.2, constant kernel gamma) scaled by
    eta_h = 6/(gamma h): the kernel constant cancels. For the SPD (shifted-symmetric) system
    a midpoint row is collocated on the mesh shifted by h/2, so there midpoints carry the
    node-type basis and nodes the midpoint-type basis (section 2.2.2).
    """
    col_is_node = (col_x.denominator == 1)
    if variant == SPD and not row_is_node:
        node_type = not col_is_node
    else:
        node_type = col_is_node
    pieces = _basis_pieces(col_x, node_type)
    integ = _integral(pieces, row_x - r, row_x + r)
    diag = 2 * r if col_x == row_x else 0
    return 6 * (diag - integ)


def assemble_quadrature(variant: int, N: int, r: int) -> np.ndarray:
    """Dense matrix built entry by entry from :func:`quadrature_entry` (exact rationals)."""
    pts = [(Fraction(i), True) for i in range(1, N)] + \
          [(Fraction(2 * i - 1, 2), False) for i in range(1, N + 1)]
    n = len(pts)
    M = np.empty((n, n))
    for a, (xp, is_node) in enumerate(pts):
        for b, (xq, _) in enumerate(pts):
            M[a, b] = float(quadrature_entry(variant, xp, is_node, xq, r))
    return M


# ----------------------------------------------------------------------------------------
# Right-hand side of the manufactured problem
# ----------------------------------------------------------------------------------------

def grid_points(N: int):
    """Interior unknown coordinates in units of h: nodes 1..N-1 then midpoints 1/2..N-1/2."""
    nodes = np.arange(1, N, dtype=np.float64)
    mids = np.arange(1, N + 1, dtype=np.float64) - 0.5
    return nodes, mids


def _u_poly(x):
    """Manufactured solution u = x^2 (1-x)^2."""
    return x * x * (1.0 - x) ** 2


def _u_antiderivative(x):
    return x ** 3 / 3.0 - x ** 4 / 2.0 + x ** 5 / 5.0


def manufactured(variant: int, N: int, r: int):
    """Right-hand side and exact nodal values for u = x^2 (1-x)^2 with g = u on Omega_I.

    Row p: b_p = (6/h) [2 delta u(x_p) - int_{x_p-delta}^{x_p+delta} u(y) dy]
                 - sum over exterior points q of entry(p, q) u(x_q),
    i.e. eta_h f(x_p) with f = -L_delta u (section 2.2, eq. (2.5); eta_h = 6/(gamma h) so
    the kernel constant cancels), minus the constrained values moved to the right-hand side
    with the same row stencil (eqs. (2.7)-(2.8), read row by row). delta = r h.
    Returns (b, u_exact) in the unknown ordering of the module docstring.
    """
    return manufactured_rhs(variant, N, r, _u_poly, _u_antiderivative)


def collocation_points(N: int) -> np.ndarray:
    """Coordinates x_p of the unknowns (nodes, then midpoints), in [0, 1]."""
    nodes, mids = grid_points(N)
    return np.concatenate([nodes, mids]) / N


def exterior_points(N: int, r: int):
    """The constrained points of Omega_I within the horizon, at half steps: left x = -j h/2
    and right x = 1 + j h/2 for j = 0..2r (x = 0 and x = 1 included)."""
    h = 1.0 / N
    j = np.arange(2 * r + 1)
    return -j * 0.5 * h, 1.0 + j * 0.5 * h


def exterior_rhs(variant: int, N: int, r: int, g_left, g_right) -> np.ndarray:
    """Minus the couplings of each row to the constrained exterior values (eqs.
    (2.7)-(2.8), read row by row with the row's own stencil): -sum_q entry(p, q) g(x_q).
    g_left[j], g_right[j]: values at the points of :func:`exterior_points`."""
    nodes, mids = grid_points(N)
    rows = [(x, True) for x in nodes] + [(x, False) for x in mids]
    out = np.zeros(len(rows))
    for p, (xp, is_node) in enumerate(rows):
        xp2 = int(round(2 * xp))
        for j in range(2 * r + 1):
            for q2, gv in ((-j, g_left[j]), (2 * N + j, g_right[j])):
                dist2 = q2 - xp2
                if abs(dist2) > 2 * r + 1:
                    continue
                w = stencil_entry(variant, is_node, dist2, r)
                if w != 0.0:
                    out[p] -= w * gv
    return out


def manufactured_rhs(variant: int, N: int, r: int, u, U):
    """The right-hand side of :func:`manufactured` for any smooth u with antiderivative U
    (callables of x): eta_h (-L_delta u)(x_p) minus the exterior couplings of g = u."""
    h = 1.0 / N
    delta = r * h
    nodes, mids = grid_points(N)
    rows = [(x, True) for x in nodes] + [(x, False) for x in mids]
    b = np.empty(len(rows))
    uex = np.empty(len(rows))
    # all grid points (units of h) from -r to N + r in half steps; exterior = outside (0, N)
    all2 = np.arange(-2 * r, 2 * (N + r) + 1)          # twice the coordinate
    ext2 = all2[(all2 <= 0) | (all2 >= 2 * N)]
    for p, (xp, is_node) in enumerate(rows):
        x = xp * h
        integ = U(x + delta) - U(x - delta)
        val = (6.0 / h) * (2.0 * delta * u(x) - integ)
        xp2 = int(round(2 * xp))
        for q2 in ext2:
            dist2 = q2 - xp2
            if abs(dist2) > 2 * r + 1:
                continue
            w = stencil_entry(variant, is_node, dist2, r)
            if w != 0.0:
                val -= w * u(q2 * 0.5 * h)
        b[p] = val
        uex[p] = u(x)
    return b, uex
