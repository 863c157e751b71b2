"""Host set-up with the geometric transfer (tpc_params.transfer = TPC_TRANSFER_GEOMETRIC, an
option of this build): every level's dense matrix equals the oracle's dense Galerkin product
with the same transfer."""
import numpy as np
import pytest
import sympy as sp

import paper_2202_11288_gb300 as tpc
from oracle import amg, fractional, model
from oracle.model import NONSYM, SPD


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("a", [None, sp.Rational(1, 4), sp.Rational(3, 4)])
@pytest.mark.parametrize("K,r", [(6, 5), (7, 2)])
def test_levels_match_oracle(variant, a, K, r):
    N = 1 << K
    A = model.assemble(variant, N, r) if a is None else fractional.assemble(variant, N, r, a)
    H = amg.Hierarchy(A, kc=3, transfer="geometric")
    kw = {} if a is None else {"kernel": 1, "kernel_a": float(a)}
    p = tpc.tpc_default_params(variant=variant, transfer=tpc.TPC_TRANSFER_GEOMETRIC, **kw)
    scale = np.abs(A).max()  # coarse entries can cancel far below the finest ones (a >= 1/2)
    for k in range(K, 2, -1):
        Ak = tpc.tpc_host_dense_level(r / N, 1.0 / N, k, params=p)
        assert np.max(np.abs(Ak - H.A[k])) <= 1e-12 * scale, k


def test_shifted_system():
    K, r, shift = 6, 5, 7.5
    N = 1 << K
    A = model.assemble(SPD, N, r) + shift * np.eye(2 * N - 1)
    H = amg.Hierarchy(A, kc=3, transfer="geometric")
    p = tpc.tpc_default_params(transfer=tpc.TPC_TRANSFER_GEOMETRIC, shift=shift)
    for k in range(K, 2, -1):
        Ak = tpc.tpc_host_dense_level(r / N, 1.0 / N, k, params=p)
        assert np.max(np.abs(Ak - H.A[k])) <= 1e-12 * np.abs(H.A[k]).max(), k


def test_transfer_limits():
    assert tpc.tpc_default_params().transfer == tpc.TPC_TRANSFER_PAPER
    with pytest.raises(tpc.TpcError) as ei:
        tpc.tpc_host_dense_level(0.25, 1 / 16, 4, params=tpc.tpc_default_params(transfer=2))
    assert ei.value.code == tpc.TPC_EINVAL
    with pytest.raises(tpc.TpcError) as ei:
        tpc.tpc_host_dense_level(
            0.25, 1 / 16, 4, params=tpc.tpc_default_params(
                variant=tpc.TPC_WEAKLY, kernel_a=0.5, transfer=tpc.TPC_TRANSFER_GEOMETRIC))
    assert ei.value.code == tpc.TPC_ENOTSUP


@pytest.mark.parametrize("variant", [SPD, NONSYM])
def test_coarse_levels_are_one_toeplitz_sequence_at_size(variant):
    """N = 2^16, delta = 0.05, fractional a = 1/4: every coarse level of the geometric
    hierarchy is Toeplitz in position order, i.e. one sequence c(d2) read through the block
    layout: A and D are c at even twice-distances, B and C at odd ones, and the Cross continues
    them (p, q, xi, zeta, o are the same sequence at the next offsets)."""
    K = 16
    N = 1 << K
    p = tpc.tpc_default_params(variant=variant, kernel=1, kernel_a=0.25,
                               transfer=tpc.TPC_TRANSFER_GEOMETRIC)
    levels = tpc.tpc_host_hierarchy(0.05, 1.0 / N, K - 6, params=p)
    for L in levels[1:]:
        n = L["N"]
        A, B, C, D = L["A"], L["B"], L["C"], L["D"]
        s = np.abs(A).max()
        assert np.max(np.abs(A - D)) <= 1e-14 * s
        # tB[d] = c(2d - 1), tC[d] = c(2d + 1): C at offset d equals B at offset d + 1
        assert np.max(np.abs(C[:-1] - B[1:])) <= 1e-14 * s
        i = np.arange(1, n + 1)
        c_odd = lambda k: B[(k + 1) // 2 + n - 1]   # c(k) for odd k, -(2n-3) <= k <= 2n-3
        c_even = lambda k: A[k // 2 + n - 1]        # c(k) for even k, |k| <= 2n-2
        assert np.max(np.abs(L["p"][:-1] - c_odd(2 * i[:-1] - 1))) <= 1e-14 * s
        assert np.max(np.abs(L["xi"][:-1] - c_even(2 * i[:-1]))) <= 1e-14 * s
        assert abs(L["o"] - A[n - 1]) <= 1e-14 * s
