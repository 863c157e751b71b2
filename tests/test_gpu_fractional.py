"""GPU path with the fractional kernel (kernel = 1; a reading of this build, see
oracle/fractional.py) against the oracle: products at every level, V-cycle iterates, and a
mixed-precision solve; for a >= 1/2 (finite-part entries, indefinite system) the iterates of
the diverging V-cycle and its reported non-convergence. The kernels are those of the constant
kernel (same banded Toeplitz-plus-Cross structure, other coefficients); tolerances as in
tests/test_gpu_parity.py."""
import numpy as np
import pytest
import sympy as sp

import paper_2202_11288_gb300 as tpc
from oracle import amg, fractional
from oracle.model import NONSYM, SPD
from synth import uniform_pm1

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(x, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("a", [sp.Integer(0), sp.Rational(1, 4), sp.Rational(1, 2),
                               sp.Rational(3, 4)])
def test_products_every_level(variant, a):
    K, r = 7, 16
    N = 1 << K
    A = fractional.assemble(variant, N, r, a)
    H = amg.Hierarchy(A, kc=3)
    S = tpc.Solver(r / N, 1.0 / N, variant=variant, kernel=1, kernel_a=float(a),
                   precision=tpc.TPC_MIXED)
    try:
        for k in range(K, H.kc, -1):
            Ak = H.A[k]
            x = uniform_pm1(Ak.shape[0], 70 + k)
            nrm = np.abs(Ak).sum(0).max() * np.linalg.norm(x)
            y = torch.empty(Ak.shape[0], dtype=torch.float64, device="cuda")
            S.apply(k, dev(x), y)
            y32 = torch.empty(Ak.shape[0], dtype=torch.float32, device="cuda")
            S.apply_f32(k, dev(x, torch.float32), y32)
            torch.cuda.synchronize()
            ref = Ak @ x
            assert np.linalg.norm(y.cpu().numpy() - ref) <= 1e-12 * nrm, k
            assert np.linalg.norm(y32.cpu().numpy().astype(np.float64) - ref) <= 2e-6 * (k + 1) * nrm, k
    finally:
        S.close()


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("a", [sp.Rational(1, 4), sp.Rational(1, 2), sp.Rational(3, 4)])
def test_vcycle_iterates_match_oracle(variant, a):
    """Iterates after 1 and 3 cycles (for a = 1/2 the residual grows about sevenfold a cycle)."""
    K, r = 7, 16
    N = 1 << K
    H = amg.Hierarchy(fractional.assemble(variant, N, r, a), kc=3)
    b = uniform_pm1(2 * N - 1, 9)
    _, _, _, its = amg.solve(H, b, tol=0.0, max_iters=3)
    for ncyc in (1, 3):
        S = tpc.Solver(r / N, 1.0 / N, variant=variant, kernel=1, kernel_a=float(a),
                       max_iters=ncyc)
        try:
            x = torch.zeros(2 * N - 1, dtype=torch.float64, device="cuda")
            S.solve(dev(b), x, tol=0.0)
            torch.cuda.synchronize()
            ref = its[ncyc - 1]
            assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref), ncyc
        finally:
            S.close()


def test_mixed_solve_converges():
    """N = 2^14, delta = 0.05, a = 1/4: the mixed solver reaches 1e-10, checked by the FP64
    product of the handle."""
    K, delta = 14, 0.05
    S = tpc.Solver(delta, 2.0 ** -K, kernel=1, kernel_a=0.25, precision=tpc.TPC_MIXED)
    try:
        b = dev(uniform_pm1(S.n, 3))
        x = torch.zeros_like(b)
        rc, it, rel = S.solve(b, x, tol=1e-10)
        assert rc == tpc.TPC_OK and rel < 1e-10
        y = torch.empty_like(b)
        S.apply(K, x, y)
        torch.cuda.synchronize()
        assert (torch.linalg.norm(b - y) / torch.linalg.norm(b)).item() < 1.05e-10
    finally:
        S.close()


def test_finite_part_solve_reports_non_convergence():
    """a = 1/2, N = 2^7, delta = 1/8: the V-cycle diverges (indefinite system); the solver stops
    at max_iters with TPC_ENOTCONV and a relative residual above 1."""
    K, r = 7, 16
    N = 1 << K
    S = tpc.Solver(r / N, 1.0 / N, kernel=1, kernel_a=0.5, max_iters=20)
    try:
        b = dev(uniform_pm1(S.n, 4))
        x = torch.zeros_like(b)
        rc, it, rel = S.solve(b, x, tol=1e-10)
        assert rc == tpc.TPC_ENOTCONV and it == 20 and rel > 1.0
    finally:
        S.close()


def test_non_finite_residual_and_right_hand_side_are_reported():
    """a = 1/2 grows the residual about sevenfold a cycle: given enough iterations it overflows
    and the solve stops with TPC_EDIVERGED; a right-hand side with a NaN is refused with
    TPC_EINVAL. The handle and the context stay usable afterwards."""
    K, r = 7, 16
    N = 1 << K
    S = tpc.Solver(r / N, 1.0 / N, kernel=1, kernel_a=0.5, max_iters=2000)
    try:
        b = dev(uniform_pm1(S.n, 4))
        x = torch.zeros_like(b)
        with pytest.raises(tpc.TpcError) as ei:
            S.solve(b, x, tol=1e-10)
        assert ei.value.code == tpc.TPC_EDIVERGED
        bad = b.clone()
        bad[3] = float("nan")
        with pytest.raises(tpc.TpcError) as ei:
            S.solve(bad, x, tol=1e-10)
        assert ei.value.code == tpc.TPC_EINVAL
    finally:
        S.close()
    C = tpc.Solver(r / N, 1.0 / N)
    try:
        b = dev(uniform_pm1(C.n, 5))
        x = torch.zeros_like(b)
        rc, it, rel = C.solve(b, x, tol=1e-10)
        assert rc == tpc.TPC_OK and rel < 1e-10
    finally:
        C.close()
