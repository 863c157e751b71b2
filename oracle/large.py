"""Finest-level operator for sizes where a dense matrix does not fit (FP64).

Test infrastructure only (see the package docstring).

The four blocks of eq. (2.9) / eq. (2.10) are Toeplitz; each is described here
by its first column and first row exactly as printed in section 2.2 (Matlab toeplitz(c, r)
semantics: entry (i, j) is c[i-j] for i >= j and r[j-i] otherwise). Two uses:

* ``rows``: selected dense rows of the finest matrix, O(n) per row;
* ``matvec``: the product A u with each Toeplitz block applied as a convolution computed by
  scipy's FFT (the library FFT stands for the convolution step of section 3.2, eq. (3.4)).
"""
from __future__ import annotations

import numpy as np
from scipy.signal import fftconvolve

from .model import NONSYM, SPD, _fit, coefficients


def block_lists(variant: int, N: int, r: int) -> dict:
    """First column / first row of A, B, C, D (section 2.2) as arrays."""
    cf = coefficients(r)
    a_int, a_half, c, d = cf["a_int"], cf["a_half"], cf["c"], cf["d"]
    out = {}
    colA = np.array(_fit(a_int, N - 1))
    out["A"] = (colA, colA)
    colB = np.array(_fit(a_half, N - 1))
    rowB = np.array(_fit([a_half[0]] + list(a_half), N))
    out["B"] = (colB, rowB)
    if variant == SPD:
        out["C"] = (rowB.copy(), colB.copy())          # C = B^T
        colD = np.array(_fit(a_int, N))
    elif variant == NONSYM:
        out["C"] = (np.array(_fit([c[0]] + list(c), N)), np.array(_fit(c, N - 1)))
        colD = np.array(_fit(d, N))
    else:
        raise ValueError("variant")
    out["D"] = (colD, colD)
    return out


def _toeplitz_row(col, row, i):
    """Row i (0-based) of toeplitz(col, row)."""
    n = len(row)
    j = np.arange(n)
    return np.where(j <= i, col[np.clip(i - j, 0, len(col) - 1)], row[np.clip(j - i, 0, n - 1)])


def rows(variant: int, N: int, r: int, idx) -> np.ndarray:
    """Dense rows idx (0-based, in the unknown ordering v then w) of the finest matrix."""
    bl = block_lists(variant, N, r)
    out = np.empty((len(idx), 2 * N - 1))
    for k, i in enumerate(idx):
        if i < N - 1:
            out[k, :N - 1] = _toeplitz_row(*bl["A"], i)
            out[k, N - 1:] = _toeplitz_row(*bl["B"], i)
        else:
            ii = i - (N - 1)
            out[k, :N - 1] = _toeplitz_row(*bl["C"], ii)
            out[k, N - 1:] = _toeplitz_row(*bl["D"], ii)
    return out


def _toeplitz_matvec(col, row, x):
    """toeplitz(col, row) @ x as a linear convolution (library FFT)."""
    M, n = len(col), len(row)
    g = np.concatenate([row[::-1][:n - 1], col])     # g[k] = T-entry at d = k - (n-1)
    y = fftconvolve(x, g)
    return y[n - 1:n - 1 + M]


def matvec(variant: int, N: int, r: int, u: np.ndarray) -> np.ndarray:
    """A u for the finest matrix of order 2N - 1."""
    bl = block_lists(variant, N, r)
    v, w = u[:N - 1], u[N - 1:]
    top = _toeplitz_matvec(*bl["A"], v) + _toeplitz_matvec(*bl["B"], w)
    bot = _toeplitz_matvec(*bl["C"], v) + _toeplitz_matvec(*bl["D"], w)
    return np.concatenate([top, bot])
