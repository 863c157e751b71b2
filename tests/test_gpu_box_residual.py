"""The finest residual r = b - A u formed from prefix sums over the runs of equal generator values
(tpc_residual on a handle with box_residual), against the FFT product of the same handle and
against the oracle.

Tolerance: the products' FP64 bound, ||r - r_ref|| <= 1e-12 ||A||_1 ||x||, for seeded uniform
operands, smooth operands and operands with a large mean (the case where the prefix sums are
largest compared with the box sums).
"""
import numpy as np
import pytest

import paper_2202_11288_gb300 as tpc
from oracle import amg, large, model
from oracle.model import NONSYM, SPD
from synth import uniform_pm1

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _operands(n, seed):
    i = np.arange(1, n + 1)
    return [uniform_pm1(n, seed), np.sin(np.pi * i / (n + 1)), 1000.0 + uniform_pm1(n, seed + 1)]


def _norm1(variant, N, r):
    bl = large.block_lists(variant, N, r)
    g = {k: np.abs(c).sum() + np.abs(rw[1:]).sum() for k, (c, rw) in bl.items()}
    return max(g["A"] + g["C"], g["B"] + g["D"])


@pytest.mark.parametrize("variant", [SPD, NONSYM])
def test_box_residual_full_size_matches_fft_and_oracle(variant):
    K, delta = 22, 0.05
    N = 1 << K
    r = model.horizon_ratio(delta, 1.0 / N)
    S = tpc.Solver(delta, 2.0 ** -K, variant=variant)
    try:
        assert tpc.tpc_uses_box_residual(S.handle) == 1
        n = S.n
        norm1 = _norm1(variant, N, r)
        b = uniform_pm1(n, 91)
        bd = _dev(b)
        for j, x in enumerate(_operands(n, 90)):
            xd = _dev(x)
            rd = torch.empty_like(xd)
            S.residual(xd, bd, rd)
            yd = torch.empty_like(xd)
            S.apply(K, xd, yd)
            res = _host(rd)
            fft = b - _host(yd)
            ref = b - large.matvec(variant, N, r, x)
            bound = 1e-12 * norm1 * np.linalg.norm(x)
            assert np.linalg.norm(res - ref) <= bound, (j, np.linalg.norm(res - ref) / bound)
            assert np.linalg.norm(res - fft) <= bound, (j, np.linalg.norm(res - fft) / bound)
    finally:
        S.close()


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("K,delta,kw", [(7, 0.125, {}), (10, 0.05, {}), (9, 0.3, {}),
                                        (8, 0.125, {"shift": 1234.5}),
                                        (9, 0.05, {"transfer": tpc.TPC_TRANSFER_GEOMETRIC}),
                                        (6, 2.0, {})])
def test_box_residual_matches_dense_oracle(variant, K, delta, kw):
    """Small sizes against the oracle's dense matrix (shift sigma I added as in the BDF4 steps;
    delta = 2 takes a horizon wider than the domain)."""
    N = 1 << K
    r = model.horizon_ratio(delta, 1.0 / N)
    A = model.assemble(variant, N, r) + kw.get("shift", 0.0) * np.eye(2 * N - 1)
    S = tpc.Solver(delta, 2.0 ** -K, variant=variant, **kw)
    try:
        assert tpc.tpc_uses_box_residual(S.handle) == 1
        norm1 = np.abs(A).sum(0).max()
        b = uniform_pm1(S.n, 7)
        for x in _operands(S.n, 3):
            rd = torch.empty(S.n, dtype=torch.float64, device="cuda")
            S.residual(_dev(x), _dev(b), rd)
            err = np.linalg.norm(_host(rd) - (b - A @ x))
            assert err <= 1e-12 * norm1 * np.linalg.norm(x), err
    finally:
        S.close()


def test_fft_residual_where_generators_vary():
    """The fractional kernel's generators vary with the distance: the handle keeps the FFT
    residual, which still equals b - A x of the oracle's dense Galerkin-free finest matrix."""
    from oracle import fractional
    K, delta, a = 9, 0.125, 0.25
    N = 1 << K
    r = model.horizon_ratio(delta, 1.0 / N)
    S = tpc.Solver(delta, 2.0 ** -K, kernel=1, kernel_a=a)
    try:
        assert tpc.tpc_uses_box_residual(S.handle) == 0
        A = fractional.assemble(SPD, N, r, a)
        x, b = uniform_pm1(S.n, 4), uniform_pm1(S.n, 5)
        rd = torch.empty(S.n, dtype=torch.float64, device="cuda")
        S.residual(_dev(x), _dev(b), rd)
        err = np.linalg.norm(_host(rd) - (b - A @ x))
        assert err <= 1e-12 * np.abs(A).sum(0).max() * np.linalg.norm(x)
    finally:
        S.close()


def test_box_residual_off_gives_the_fft_residual_and_the_same_solve():
    K, delta = 12, 0.05
    b = uniform_pm1((1 << (K + 1)) - 1, 11)
    out = {}
    for box in (0, 1):
        S = tpc.Solver(delta, 2.0 ** -K, box_residual=box)
        try:
            assert tpc.tpc_uses_box_residual(S.handle) == box
            xd = torch.zeros(S.n, dtype=torch.float64, device="cuda")
            rc, it, rel = S.solve(_dev(b), xd, tol=1e-10)
            assert rc == tpc.TPC_OK and rel < 1e-10
            out[box] = (it, _host(xd))
        finally:
            S.close()
    assert out[0][0] == out[1][0]
    assert np.linalg.norm(out[0][1] - out[1][1]) <= 1e-10 * np.linalg.norm(out[0][1])


def test_box_residual_rejects_aliasing():
    S = tpc.Solver(0.125, 2.0 ** -7)
    try:
        x = torch.zeros(S.n, dtype=torch.float64, device="cuda")
        with pytest.raises(tpc.TpcError):
            S.residual(x, x.clone(), x)
    finally:
        S.close()
