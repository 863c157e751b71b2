"""Mixed precision (FP32 V-cycles inside FP64 iterative refinement) against the FP64 oracle.

FP32 products: one forward and one inverse FFT of length m in FP32 carry an absolute error of
order eps32 * log2(m) * ||c|| ||x|| (eps32 = 6e-8), plus the rounding of x and of the spectra;
the bound used is 2e-6 * log2(m) normwise, ||y - y_ref|| <= 2e-6 log2(m) ||A||_1 ||x||.
Solutions: the FP64 residual reaches 1e-10, and the distance to the oracle's direct FP64
solution is within cond(A) * 1e-10 (two solutions with relative residual 1e-10 can differ by
that much).
"""
import numpy as np
import pytest

import paper_2202_11288_gb300 as tpc
from oracle import amg, large, model
from oracle.model import NONSYM, SPD
from synth import uniform_pm1

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(x, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("K,delta", [(7, 0.125), (11, 0.05)])
def test_fp32_products_every_level(variant, K, delta):
    S = tpc.Solver(delta, 2.0 ** -K, variant=variant, precision=tpc.TPC_MIXED)
    try:
        N = 1 << K
        H = amg.Hierarchy(model.assemble(variant, N, model.horizon_ratio(delta, 1.0 / N)), kc=3)
        for k in range(K, H.kc, -1):
            A = H.A[k]
            n = A.shape[0]
            x = uniform_pm1(n, 300 + k)
            yd = torch.empty(n, dtype=torch.float32, device="cuda")
            S.apply_f32(k, dev(x, torch.float32), yd)
            y = host(yd)
            ref = A @ x
            bound = 2e-6 * (k + 1) * np.abs(A).sum(0).max() * np.linalg.norm(x)
            assert np.linalg.norm(y - ref) <= bound, (k, np.linalg.norm(y - ref) / bound)
    finally:
        S.close()


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("inner", [1, 4])
def test_mixed_solve_matches_fp64_oracle(variant, inner):
    K, delta = 9, 0.125
    N = 1 << K
    A = model.assemble(variant, N, model.horizon_ratio(delta, 1.0 / N))
    b = uniform_pm1(2 * N - 1, 12)
    S = tpc.Solver(delta, 1.0 / N, variant=variant, precision=tpc.TPC_MIXED, inner_cycles=inner)
    try:
        xd = torch.zeros(2 * N - 1, dtype=torch.float64, device="cuda")
        rc, it, rel = S.solve(dev(b), xd, tol=1e-10)
        x = host(xd)
    finally:
        S.close()
    assert rc == tpc.TPC_OK and rel < 1e-10
    assert np.linalg.norm(b - A @ x) <= 1.01e-10 * np.linalg.norm(b)
    x_ref = np.linalg.solve(A, b)
    cond = np.linalg.cond(A)
    err = np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref)
    assert err <= cond * 1e-10, (err, cond)
    if inner == 4:
        assert it <= 5           # FP64 residuals per solve


def test_mixed_and_fp64_agree_on_the_manufactured_problem():
    """N = 256, delta = 1/8: both solvers reach the same discretisation error of the scheme
    (within 1 %), and differ from each other by at most cond(A) * tol * max|x|."""
    K, delta, tol = 8, 0.125, 1e-12
    N = 1 << K
    r = model.horizon_ratio(delta, 1.0 / N)
    A = model.assemble(SPD, N, r)
    b, uex = model.manufactured(SPD, N, r)
    out = []
    for prec in (tpc.TPC_FP64, tpc.TPC_MIXED):
        S = tpc.Solver(delta, 1.0 / N, precision=prec)
        try:
            xd = torch.zeros(2 * N - 1, dtype=torch.float64, device="cuda")
            rc, it, rel = S.solve(dev(b), xd, tol=tol)
            assert rc == tpc.TPC_OK and rel < tol
            out.append(host(xd))
        finally:
            S.close()
    e64, e32 = (np.max(np.abs(x - uex)) for x in out)
    assert abs(e32 - e64) <= 0.01 * e64
    cond = np.linalg.cond(A)
    assert np.max(np.abs(out[0] - out[1])) <= cond * tol * np.max(np.abs(out[0]))


def test_mixed_full_size_solve():
    """N = 2^22, delta = 0.05: the mixed solver reaches 1e-10, checked by the oracle's FFT
    product of the finest matrix."""
    K, delta = 22, 0.05
    N = 1 << K
    r = model.horizon_ratio(delta, 1.0 / N)
    S = tpc.Solver(delta, 2.0 ** -K, precision=tpc.TPC_MIXED)
    try:
        b = uniform_pm1(S.n, 0)
        xd = torch.zeros(S.n, dtype=torch.float64, device="cuda")
        rc, it, rel = S.solve(dev(b), xd, tol=1e-10)
        assert rc == tpc.TPC_OK and rel < 1e-10 and it <= 6
        res = b - large.matvec(SPD, N, r, host(xd))
        assert np.linalg.norm(res) <= 1.05e-10 * np.linalg.norm(b)
    finally:
        S.close()


def test_fp32_product_needs_mixed_handle():
    S = tpc.Solver(0.125, 2.0 ** -7)
    try:
        x = torch.zeros(S.n, dtype=torch.float32, device="cuda")
        with pytest.raises(tpc.TpcError):
            S.apply_f32(7, x, x.clone())
    finally:
        S.close()
