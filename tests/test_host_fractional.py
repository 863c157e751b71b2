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
