"""Host setup of the library (C++, no GPU) against the oracle's dense Galerkin hierarchy."""
import numpy as np
import pytest

import paper_2202_11288_gb300 as tpc
from oracle import amg, model
from oracle.model import NONSYM, SPD


def _compare(level, ref, tol):
    N = ref["N"]
    assert level["N"] == N
    scale = max(np.abs(ref["A"]).max(), abs(ref["o"]))
    for key in ("A", "B", "C", "D", "p", "q", "xi", "zeta"):
        np.testing.assert_allclose(level[key], ref[key], rtol=0, atol=tol * scale, err_msg=key)
    assert abs(level["o"] - ref["o"]) <= tol * scale


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("K,delta", [(5, 0.125), (6, 0.125), (7, 0.125), (6, 0.01),
                                     (6, 0.3), (5, 1.4), (7, 0.05)])
def test_generator_hierarchy_matches_dense_galerkin(variant, K, delta):
    N = 1 << K
    h = 1.0 / N
    r = model.horizon_ratio(delta, h)
    kc = 1
    H = amg.Hierarchy(model.assemble(variant, N, r), kc=kc)
    p = tpc.tpc_default_params(variant=variant, coarsest_level=kc)
    levels = tpc.tpc_host_hierarchy(delta, h, 0, p)
    assert len(levels) == K - kc + 1
    for i, lev in enumerate(levels):
        k = K - i
        ref = amg.split_cross(H.A[k])
        _compare(lev, ref, 0.0 if k == K else 1e-13)


def test_shift_adds_to_the_finest_diagonal():
    K, delta, sigma = 6, 0.125, 3.25
    N = 1 << K
    A = model.assemble(SPD, N, model.horizon_ratio(delta, 1.0 / N)) + sigma * np.eye(2 * N - 1)
    H = amg.Hierarchy(A, kc=3)
    levels = tpc.tpc_host_hierarchy(delta, 1.0 / N, 0, tpc.tpc_default_params(shift=sigma))
    for i, lev in enumerate(levels):
        _compare(lev, amg.split_cross(H.A[K - i]), 1e-13)


def test_levels_argument_sets_the_coarsest_level():
    levels = tpc.tpc_host_hierarchy(0.125, 2.0 ** -7, 3)
    assert [l["N"] for l in levels] == [127, 63, 31]


@pytest.mark.parametrize("kw,delta,h,levels,code", [
    ({}, 0.1, 0.3, 0, tpc.TPC_EINVAL),                 # h not a power of two
    ({}, -0.1, 2.0 ** -6, 0, tpc.TPC_EINVAL),          # delta <= 0
    ({"coarsest_level": 7}, 0.1, 2.0 ** -6, 0, tpc.TPC_EINVAL),   # kc > K
    ({"coarsest_level": 0}, 0.1, 2.0 ** -6, 0, tpc.TPC_EINVAL),
    ({}, 0.1, 2.0 ** -6, 5, tpc.TPC_EINVAL),           # more levels than K - kc + 1
    ({"variant": 5}, 0.1, 2.0 ** -6, 0, tpc.TPC_EINVAL),
    ({"kernel": 1, "kernel_a": 1.0}, 0.1, 2.0 ** -6, 0, tpc.TPC_ENOTSUP),
    ({"kernel": 2}, 0.1, 2.0 ** -6, 0, tpc.TPC_EINVAL),
    ({"omega_pre": 2.5}, 0.1, 2.0 ** -6, 0, tpc.TPC_EINVAL),
    ({"m1": 0}, 0.1, 2.0 ** -6, 0, tpc.TPC_EINVAL),
])
def test_invalid_arguments_are_rejected(kw, delta, h, levels, code):
    with pytest.raises(tpc.TpcError) as ei:
        tpc.tpc_host_hierarchy(delta, h, levels, tpc.tpc_default_params(**kw))
    assert ei.value.code == code
    assert tpc.tpc_last_error()


def test_horizon_ratio_rule():
    # r = floor(delta/h) (r = 1 when delta <= h): first column of A is a_0 = 12 r - 2
    for delta, h, r in [(0.125, 2.0 ** -7, 16), (0.05, 2.0 ** -14, 819), (0.001, 2.0 ** -6, 1),
                        (0.2, 2.0 ** -10, 204)]:
        assert model.horizon_ratio(delta, h) == r
        lev = tpc.tpc_host_hierarchy(delta, h, 0)[0]
        assert lev["A"][lev["N"] - 1] == 12 * r - 2


def test_poison_flag_is_validated():
    assert tpc.tpc_default_params().poison == 0
    with pytest.raises(tpc.TpcError) as ei:
        tpc.tpc_host_dense_level(0.25, 1 / 16, 4, params=tpc.tpc_default_params(poison=2))
    assert ei.value.code == tpc.TPC_EINVAL
