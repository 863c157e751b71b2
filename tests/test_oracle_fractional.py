"""Oracle of the fractional kernel with a horizon (a reading of this build; the paper defines
only the constant kernel): pinned to the printed matrix at a = -1/2, to exactness on
quadratics, entry by entry (a < 1/2) to the convergent integral of its definition and
(a >= 1/2) to Hadamard's definition of the finite part, both evaluated by adaptive quadrature
on the basis functions. Parity of the fractional entries is otherwise unpinned by the paper."""
import numpy as np
import pytest
import sympy as sp
from scipy.integrate import quad

from oracle import fractional, model
from oracle.model import NONSYM, SPD


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("N,r", [(8, 1), (16, 3), (16, 5)])
def test_a_minus_half_is_the_printed_matrix(variant, N, r):
    A = fractional.assemble(variant, N, r, sp.Rational(-1, 2))
    assert np.max(np.abs(A - model.assemble(variant, N, r))) <= 1e-12


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("a", [sp.Rational(-1, 4), sp.Integer(0), sp.Rational(1, 4),
                               sp.Rational(2, 5), sp.Rational(1, 2), sp.Rational(3, 4),
                               sp.Rational(9, 10)])
@pytest.mark.parametrize("r", [1, 3])
def test_stencil_exact_on_quadratics(variant, a, r):
    """sum_q A_pq u(x_q) = 6 int |s|^{-(1+2a)} [u(x_p) - u(x_p + s)] ds for u = 1, s, s^2 (units
    of h, row at the origin): 0, 0 and -12 r^{2-2a} / (2-2a) (convergent for every a < 1; for
    a >= 1/2 the entries are finite parts and the identities still hold)."""
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


@pytest.mark.parametrize("a", [sp.Rational(1, 2), sp.Rational(3, 4)])
def test_spd_system_symmetric_indefinite_for_finite_parts(a):
    """a >= 1/2: the finite-part system is still symmetric but has negative eigenvalues."""
    A = fractional.assemble(SPD, 16, 3, a)
    assert np.max(np.abs(A - A.T)) <= 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() < 0.0


def _lagrange_basis(node_type, c):
    """Quadratic Lagrange basis function centred at c (units of h): a vertex of the elements
    [c-1, c] and [c, c+1], or the midpoint of [c-1/2, c+1/2]."""
    def phi(y):
        # evaluated in the element's own coordinate v (measured from its left end, which is a
        # half-integer and so subtracted exactly), so that values next to an element end keep
        # their relative accuracy
        if node_type:
            if c <= y <= c + 1:
                v = y - c
                return 2 * (v - 0.5) * (v - 1)
            if c - 1 <= y < c:
                v = y - (c - 1)
                return 2 * (v - 0.5) * v
            return 0.0
        if c - 0.5 <= y <= c + 0.5:
            v = y - (c - 0.5)
            return -4 * v * (v - 1)
        return 0.0
    return phi


def _hadamard_entry(variant, row_is_node, dist2, r, a, eps=1e-3):
    """6 f.p. int_{-r}^{r} |s|^{-g} [phi_q(0) - phi_q(s)] ds, g = 1 + 2a, by Hadamard's
    definition: on each side lim_{e->0} of int_e^r f(t) t^{-g} dt plus f'(0) e^{2-g} / (2-g)
    (f'(0) log e for g = 2), f(t) = phi_q(0) - phi_q(+-t). The truncated integrals come from
    adaptive quadrature on the basis function itself; the remaining error, exactly a multiple
    of e^{3-g} (f is quadratic on [0, 1/2]), is removed by one Richardson step in e."""
    g = 1 + 2 * a
    col_is_node = (dist2 % 2 == 0) == row_is_node
    node_type = (not col_is_node) if (variant == SPD and not row_is_node) else col_is_node
    phi = _lagrange_basis(node_type, -dist2 / 2)
    brk = [k / 2 for k in range(1, 2 * r)]
    total = 0.0
    for sgn in (1.0, -1.0):
        def f(t):
            return phi(0.0) - phi(sgn * t)
        f1 = (-3 * f(0.0) + 4 * f(0.25) - f(0.5)) / 0.5  # exact for a quadratic on [0, 1/2]

        def E(e):
            pts = [e] + [b for b in brk if b > e] + [float(r)]
            val = sum(quad(lambda t: f(t) * t ** (-g), lo, hi, epsabs=0, epsrel=1e-13,
                           limit=200)[0] for lo, hi in zip(pts[:-1], pts[1:]))
            return val + (f1 * np.log(e) if g == 2 else f1 * e ** (2 - g) / (2 - g))
        q = 4.0 ** (3 - g)
        total += (q * E(eps) - E(4 * eps)) / (q - 1)
    return 6 * total


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("a", [sp.Rational(1, 2), sp.Rational(3, 4), sp.Rational(9, 10)])
@pytest.mark.parametrize("r", [1, 3])
def test_finite_parts_follow_hadamards_definition(variant, a, r):
    """Every entry of both row types equals the finite part computed from its definition."""
    for row_is_node in (True, False):
        d2s, w = fractional.stencil(variant, row_is_node, r, a)
        scale = max(abs(x) for x in w)
        for d2, wo in zip(d2s, w):
            ref = _hadamard_entry(variant, row_is_node, d2, r, float(a))
            assert abs(ref - wo) <= 1e-10 * scale, (row_is_node, d2)


def _convergent_entry(variant, row_is_node, dist2, r, a):
    """6 int_{-r}^{r} |s|^{-g} [phi_q(0) - phi_q(s)] ds, g = 1 + 2a < 2: an ordinary integral (the
    bracket vanishes linearly at s = 0), by adaptive quadrature on each piece between the basis
    function's breakpoints (half steps), no finite-part term. On the piece next to s = 0 the
    substitution t = u^k, k = 1 / (2 - g), makes the integrand smooth."""
    g = 1 + 2 * a
    col_is_node = (dist2 % 2 == 0) == row_is_node
    node_type = (not col_is_node) if (variant == SPD and not row_is_node) else col_is_node
    phi = _lagrange_basis(node_type, -dist2 / 2)
    pts = [k / 2 for k in range(1, 2 * r)] + [float(r)]
    k = 1.0 / (2.0 - g)
    total = 0.0
    for sgn in (1.0, -1.0):
        def f(t):
            return phi(0.0) - phi(sgn * t)
        # on [0, 1/2] the bracket is the quadratic f1 t + f2 t^2 (no breakpoint inside; its
        # coefficients from two samples, where they carry no cancellation), and with t = u^k the
        # integrand k (f1 + f2 u^k) is smooth
        f1 = 8.0 * f(0.25) - 2.0 * f(0.5)
        f2 = 8.0 * f(0.5) - 16.0 * f(0.25)
        total += quad(lambda u: k * (f1 + f2 * u ** k), 0.0, 0.5 ** (2 - g), epsrel=1e-13)[0]
        for lo, hi in zip(pts[:-1], pts[1:]):
            total += quad(lambda t: f(t) * t ** (-g), lo, hi, epsrel=1e-13, limit=400)[0]
    return 6 * total


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("a", [sp.Rational(-1, 4), sp.Integer(0), sp.Rational(1, 4),
                               sp.Rational(2, 5)])
@pytest.mark.parametrize("r", [1, 3])
def test_entries_follow_the_convergent_integral(variant, a, r):
    """a < 1/2: every entry of both row types equals its defining integral (which converges)."""
    for row_is_node in (True, False):
        d2s, w = fractional.stencil(variant, row_is_node, r, a)
        scale = max(abs(x) for x in w)
        for d2, wo in zip(d2s, w):
            ref = _convergent_entry(variant, row_is_node, d2, r, float(a))
            assert abs(ref - wo) <= 1e-10 * scale, (row_is_node, d2, ref, wo)
