"""Host entry points of the time stepping (no GPU): the collocation right-hand side and the
BDF4 coefficients against the oracle (section 5, eq. (5.1); section 2.2 eqs. (2.5) and
(2.7)-(2.8))."""
import math

import numpy as np
import pytest

import paper_2202_11288_gb300 as tpc
from oracle import model, timestep
from oracle.model import NONSYM, SPD


def phi(x):
    return (1.0 + x) ** 6


def Phi(x):
    return (1.0 + x) ** 7 / 7.0


def source_f(N, r):
    """phi - L_delta phi at the collocation points, closed form (gamma = 3 / (r h)^3)."""
    h = 1.0 / N
    delta = r * h
    gamma = 3.0 / delta ** 3
    x = np.concatenate([np.arange(1, N), np.arange(1, N + 1) - 0.5]) / N
    return phi(x) - gamma * (Phi(x + delta) - Phi(x - delta) - 2.0 * delta * phi(x))


def exterior(N, r):
    j = np.arange(2 * r + 1)
    return phi(-j * 0.5 / N), phi(1.0 + j * 0.5 / N)


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("N,r", [(8, 1), (16, 3), (32, 8), (64, 16), (32, 40)])
def test_collocation_rhs_matches_oracle_source(variant, N, r):
    delta, h = r / N, 1.0 / N
    p = tpc.tpc_default_params(variant=variant)
    gl, gr = exterior(N, r)
    G = tpc.tpc_collocation_rhs(delta, h, source_f(N, r), gl, gr, params=p)
    G_ref = timestep.source_vector(variant, N, r)
    assert np.max(np.abs(G - G_ref)) <= 1e-11 * np.max(np.abs(G_ref))


@pytest.mark.parametrize("variant", [SPD, NONSYM])
def test_collocation_rhs_exterior_part_alone(variant):
    N, r = 32, 5
    gl, gr = exterior(N, r)
    ext = tpc.tpc_collocation_rhs(r / N, 1.0 / N, None, gl, gr,
                                  params=tpc.tpc_default_params(variant=variant))
    ref = model.exterior_rhs(variant, N, r, gl, gr)
    assert np.array_equal(ext == 0, ref == 0)
    assert np.allclose(ext, ref, rtol=1e-13, atol=0)
    f_only = tpc.tpc_collocation_rhs(r / N, 1.0 / N, np.ones(2 * N - 1), None, None,
                                     params=tpc.tpc_default_params(variant=variant))
    assert np.allclose(f_only, timestep.eta_h(N, r), rtol=1e-15, atol=0)


def test_bdf4_coefficients():
    for N, r in ((32, 8), (256, 16)):
        h, tau = 1.0 / N, 1.0 / N
        sigma, hs = tpc.tpc_bdf4_coefficients(r * h, h, tau)
        eta = timestep.eta_h(N, r)
        assert math.isclose(sigma, 25.0 * eta / (12.0 * tau), rel_tol=1e-15)
        assert math.isclose(hs, eta / tau, rel_tol=1e-15)
    sigma, hs = tpc.tpc_bdf4_coefficients(0.25, 1 / 32, 1 / 32,
                                          params=tpc.tpc_default_params(gamma0=2.0))
    assert math.isclose(hs, 6.0 / (2.0 / 32) * 32, rel_tol=1e-15)


def test_time_stepping_arguments_rejected():
    with pytest.raises(tpc.TpcError):
        tpc.tpc_bdf4_coefficients(0.25, 1 / 32, 0.0)
    with pytest.raises(tpc.TpcError):
        tpc.tpc_bdf4_coefficients(0.25, 0.3, 0.1)
    with pytest.raises(tpc.TpcError):
        tpc.tpc_collocation_rhs(0.25, 1 / 32, params=tpc.tpc_default_params(gamma0=-1.0))
