"""Oracle of the fractional kernel with a horizon (a reading of this build; the paper defines
only the constant kernel): pinned to the printed matrix at a = -1/2 and to exactness on
quadratics. Parity of the fractional entries is otherwise unpinned by the paper."""
import numpy as np
import pytest
import sympy as sp

from oracle import fractional, model
from oracle.model import NONSYM, SPD


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("N,r", [(8, 1), (16, 3), (16, 5)])
def test_a_minus_half_is_the_printed_matrix(variant, N, r):
    A = fractional.assemble(variant, N, r, sp.Rational(-1, 2))
    assert np.max(np.abs(A - model.assemble(variant, N, r))) <= 1e-12


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("a", [sp.Rational(-1, 4), sp.Integer(0), sp.Rational(1, 4),
                               sp.Rational(2, 5)])
@pytest.mark.parametrize("r", [1, 3])
def test_stencil_exact_on_quadratics(variant, a, r):
    """sum_q A_pq u(x_q) = 6 int |s|^{-(1+2a)} [u(x_p) - u(x_p + s)] ds for u = 1, s, s^2 (units
    of h, row at the origin): 0, 0 and -12 r^{2-2a} / (2-2a)."""
    g = 1 + 2 * a
    expected_x2 = float(-12 * sp.Integer(r) ** (3 - g) / (3 - g))
    for row_is_node in (True, False):
        d2s, w = fractional.stencil(variant, row_is_node, r, a)
        x = -np.array(d2s) / 2.0  # column coordinate relative to the row
        w = np.array(w)
        assert abs(w.sum()) <= 1e-10 * np.abs(w).sum()
        assert abs((w * x).sum()) <= 1e-10 * np.abs(w).sum()
        assert abs((w * x * x).sum() - expected_x2) <= 1e-10 * abs(expected_x2)


@pytest.mark.parametrize("a", [sp.Integer(0), sp.Rational(1, 4)])
def test_spd_system_symmetric_positive(a):
    A = fractional.assemble(SPD, 16, 3, a)
    assert np.max(np.abs(A - A.T)) <= 1e-12 * np.abs(A).max()
    np.linalg.cholesky(A)
