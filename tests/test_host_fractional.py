"""Host set-up of the fractional kernel (kernel = 1, exponent a = kernel_a) against the oracle:
every level's dense matrix (finest: the exact-integral entries; coarse: dense Galerkin R A P)."""
import numpy as np
import pytest
import sympy as sp

import paper_2202_11288_gb300 as tpc
from oracle import amg, fractional
from oracle.model import NONSYM, SPD


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("a", [sp.Integer(0), sp.Rational(1, 4), sp.Rational(2, 5),
                               sp.Rational(1, 2), sp.Rational(3, 4), sp.Rational(9, 10)])
def test_levels_match_oracle(variant, a):
    K, r = 5, 3
    N = 1 << K
    A = fractional.assemble(variant, N, r, a)
    H = amg.Hierarchy(A, kc=3)
    p = tpc.tpc_default_params(variant=variant, kernel=1, kernel_a=float(a))
    for k in range(K, 2, -1):
        Ak = tpc.tpc_host_dense_level(r / N, 1.0 / N, k, params=p)
        assert np.max(np.abs(Ak - H.A[k])) <= 1e-11 * np.abs(H.A[k]).max(), k


def test_fractional_exponent_limits():
    with pytest.raises(tpc.TpcError) as ei:
        tpc.tpc_host_dense_level(0.25, 1 / 16, 4,
                                 params=tpc.tpc_default_params(kernel=1, kernel_a=1.0))
    assert ei.value.code == tpc.TPC_ENOTSUP
    with pytest.raises(tpc.TpcError):
        tpc.tpc_host_dense_level(0.25, 1 / 16, 4,
                                 params=tpc.tpc_default_params(kernel=1, kernel_a=-0.75))
    with pytest.raises(tpc.TpcError):
        tpc.tpc_host_dense_level(0.25, 1 / 16, 4, params=tpc.tpc_default_params(kernel=2))


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("a", [sp.Rational(1, 4), sp.Rational(3, 4)])
def test_entries_at_the_full_size_horizon(variant, a):
    """r = 209715 (the benchmark's horizon ratio; N = 2^18, delta = 0.8): the host's finest
    entries (closed forms next to the singularity, Gauss-Legendre farther) equal the oracle's
    exact integrals at sampled twice-distances, near, in the middle and at the end of the
    horizon, and zero beyond it."""
    K, delta = 18, 0.8
    N = 1 << K
    r = int(delta * N)
    p = tpc.tpc_default_params(variant=variant, kernel=1, kernel_a=float(a))
    L = tpc.tpc_host_hierarchy(delta, 1.0 / N, 12, params=p)[0]
    Nk = L["N"]

    def node_row(d2):  # finest_form's layout: A at even, B at odd twice-distances
        return L["A"][d2 // 2 + Nk - 1] if d2 % 2 == 0 else L["B"][(d2 - 1) // 2 + Nk]

    def mid_row(d2):  # D at even, C at odd twice-distances
        return L["D"][d2 // 2 + Nk - 1] if d2 % 2 == 0 else L["C"][(d2 + 1) // 2 + Nk - 2]

    scale = abs(node_row(0))
    for d2 in [0, 1, -1, 2, -2, 3, -3, 7, -8, 100, -101, r, -r, r + 1, 2 * r - 1, -(2 * r - 1),
               2 * r, -2 * r, 2 * r + 1, -(2 * r + 1), 2 * r + 2, 2 * r + 3, -(2 * r + 3)]:
        for row_is_node, f in ((True, node_row), (False, mid_row)):
            ref = fractional.entry(variant, row_is_node, d2, r, a)
            assert abs(f(d2) - ref) <= 1e-13 * scale, (row_is_node, d2)
