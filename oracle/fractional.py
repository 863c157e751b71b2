"""Fractional kernel with a horizon: gamma(|s|) = gamma0 |s|^{-(1+2a)} for |s| < delta.

Test infrastructure only (see the package docstring).

The paper defines only the constant kernel with a horizon (section 2.2); this module states the
reading used for the fractional family named in the benchmark configurations: the collocation
of -L_delta u, L_delta u(x) = int_{|s|<delta} gamma(|s|) (u(x+s) - u(x)) ds, with the piecewise
quadratic basis, each entry written as an exact integral,

    A_pq = 6 int_{|sigma|<r} |sigma|^{-(1+2a)} [phi_q(x_p) - phi_q(x_p + sigma)] dsigma

(units of h, r = floor(delta / h)); the factor 6 and the units make a = -1/2 (the constant
kernel) reproduce the printed coefficients of section 2.2, and the SPD system collocates its
midpoint rows on the mesh shifted by h/2 as eq. (2.10) does. Integrals are evaluated exactly
with sympy (rational exponent), term by term over the powers of s, for -1/2 <= a < 1. For
a < 1/2 every integral converges. For 1/2 <= a < 1 the linear term of the basis next to the
singularity gives int_0 s^{-2a} ds, which diverges; the entry is then its Hadamard finite
part, the analytic continuation in a: int_0^c s^{e-1} ds = c^e / e also for e < 0, and
log c (units of h) for e = 0 (a = 1/2). PARITY UNPINNED by the paper: the pins are
mathematical (a = -1/2 gives the printed matrix; the stencil is exact on 1, x, x^2, which
holds for the finite parts too since continuation in a is linear; symmetry of the SPD system).
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np
import sympy as sp

from .model import SPD, grid_points

_S = sp.Symbol("s", real=True)


def _basis(node_type: bool, c: sp.Rational):
    """Pieces (lo, hi, expression in s) of the basis function centred at c (units of h)."""
    if node_type:
        t = _S - (c - 1)
        u = (c + 1) - _S
        return [(c - 1, c, t * (2 * t - 1)), (c, c + 1, u * (2 * u - 1))]
    half = sp.Rational(1, 2)
    return [(c - half, c + half, 4 * (_S - (c - half)) * ((c + half) - _S))]


def _int_power(k, g, lo, hi):
    """int_lo^hi t^{k-g} dt for 0 <= lo < hi; at t = 0 with k - g <= -1 the Hadamard finite
    part (the antiderivative t^e / e or log t is taken as 0 there)."""
    e = k + 1 - g

    def F(t):
        if t == 0:
            return sp.Integer(0)
        return sp.log(t) if e == 0 else t ** e / e

    return F(hi) - F(lo)


def _int_weighted(expr, lo, hi, g):
    """Exact int_lo^hi expr(s) |s|^{-g} ds (a finite part where it diverges at s = 0), split
    at s = 0 into integrals over t = |s| >= 0 of the polynomial's powers."""
    tot = sp.Integer(0)
    if hi > 0:
        poly = sp.Poly(sp.expand(expr), _S)
        for (k,), c in poly.terms():
            tot += c * _int_power(k, g, max(lo, 0), hi)
    if lo < 0:
        poly = sp.Poly(sp.expand(expr.subs(_S, -_S)), _S)  # s = -t
        for (k,), c in poly.terms():
            tot += c * _int_power(k, g, max(-hi, 0), -lo)
    return tot


@lru_cache(maxsize=None)
def entry(variant: int, row_is_node: bool, dist2: int, r: int, a: sp.Rational) -> float:
    """A_pq for a row of the given type and a column at twice-distance dist2 = 2 (x_p - x_q)."""
    g = 1 + 2 * a
    col_is_node = (dist2 % 2 == 0) == row_is_node
    node_type = (not col_is_node) if (variant == SPD and not row_is_node) else col_is_node
    c = -sp.Rational(dist2, 2)
    R = sp.Integer(r)
    tot = sp.Integer(0)
    if dist2 == 0:
        sup = 1 if node_type else sp.Rational(1, 2)
        for lo, hi, ex in _basis(node_type, c):
            lo, hi = max(lo, -R), min(hi, R)
            if hi > lo:
                tot += _int_weighted(1 - ex, lo, hi, g)
        if R > sup:
            tot += _int_weighted(sp.Integer(1), sup, R, g) + _int_weighted(sp.Integer(1), -R, -sup, g)
        return float(6 * tot)
    for lo, hi, ex in _basis(node_type, c):
        lo, hi = max(lo, -R), min(hi, R)
        if hi > lo:
            tot += _int_weighted(ex, lo, hi, g)
    return float(-6 * tot)


def assemble(variant: int, N: int, r: int, a) -> np.ndarray:
    """Dense matrix in the unknown ordering of section 2.2 (nodes, then midpoints)."""
    a = sp.Rational(a)
    nodes, mids = grid_points(N)
    pts = [(int(2 * x), True) for x in nodes] + [(int(2 * x), False) for x in mids]
    n = len(pts)
    M = np.empty((n, n))
    for i, (p2, pnode) in enumerate(pts):
        for j, (q2, _) in enumerate(pts):
            d2 = p2 - q2
            M[i, j] = entry(variant, pnode, d2, r, a) if abs(d2) <= 2 * r + 2 else 0.0
    return M


def stencil(variant: int, row_is_node: bool, r: int, a):
    """The row's full stencil: (twice-distances, entries) over every grid point in reach."""
    a = sp.Rational(a)
    d2s = list(range(-(2 * r + 2), 2 * r + 3))
    return d2s, [entry(variant, row_is_node, d, r, a) for d in d2s]
