"""Host setup of the weakly singular model (section 2.1, eq. (2.3)) against the oracle, no
GPU: every level's dense matrix (finest: A_h; coarse: the dense Galerkin R A P of Algorithm 2),
the right-hand side pieces and the BDF4 coefficients."""
import math

import numpy as np
import pytest

import paper_2202_11288_gb300 as tpc
from oracle import amg, weakly


@pytest.mark.parametrize("gamma", [0.0, 0.5, 0.9])
def test_levels_match_dense_galerkin(gamma):
    K = 6
    N = 1 << K
    p = tpc.tpc_default_params(variant=tpc.TPC_WEAKLY, kernel_a=gamma)
    A = weakly.assemble(N, gamma)
    H = amg.Hierarchy(A, kc=3)
    for k in range(K, 2, -1):
        Ak = tpc.tpc_host_dense_level(0.1, 1.0 / N, k, params=p)
        ref = H.A[k]
        assert np.max(np.abs(Ak - ref)) <= 1e-12 * np.max(np.abs(ref)), k


def test_shift_and_band_structure():
    """The shift adds sigma to the diagonal; coarse levels differ from a Toeplitz-plus-Cross
    matrix by a tridiagonal (the Galerkin image of the diagonal D)."""
    N, gamma, sigma = 32, 0.5, 7.25
    p0 = tpc.tpc_default_params(variant=tpc.TPC_WEAKLY, kernel_a=gamma)
    p1 = tpc.tpc_default_params(variant=tpc.TPC_WEAKLY, kernel_a=gamma, shift=sigma)
    A0 = tpc.tpc_host_dense_level(0.1, 1.0 / N, 5, params=p0)
    A1 = tpc.tpc_host_dense_level(0.1, 1.0 / N, 5, params=p1)
    assert np.allclose(A1 - A0, sigma * np.eye(A0.shape[0]), rtol=0, atol=1e-12)


@pytest.mark.parametrize("gamma", [0.0, 0.5, 0.9])
def test_rhs_and_bdf4_coefficients(gamma):
    N = 32
    h = 1.0 / N
    p = tpc.tpc_default_params(variant=tpc.TPC_WEAKLY, kernel_a=gamma)
    x = np.array(weakly.points(N)) / (2.0 * N)
    f = weakly.phi(x) + weakly.L_phi(x, gamma)
    G = tpc.tpc_collocation_rhs(0.1, h, f, np.array([weakly.phi(0.0)]),
                                np.array([weakly.phi(1.0)]), params=p)
    K0, KN = weakly.boundary_columns(N, gamma)
    ref = weakly.eta(N, gamma) * f + K0 * weakly.phi(0.0) + KN * weakly.phi(1.0)
    assert np.max(np.abs(G - ref)) <= 1e-12 * np.max(np.abs(ref))
    sigma, hs = tpc.tpc_bdf4_coefficients(0.1, h, h, params=p)
    assert math.isclose(hs, weakly.eta(N, gamma) / h, rel_tol=1e-14)
    assert math.isclose(sigma, 25.0 * weakly.eta(N, gamma) / (12.0 * h), rel_tol=1e-14)


def test_weakly_exponent_validated():
    with pytest.raises(tpc.TpcError):
        tpc.tpc_host_dense_level(0.1, 1 / 16, 4,
                                 params=tpc.tpc_default_params(variant=tpc.TPC_WEAKLY,
                                                               kernel_a=1.0))
