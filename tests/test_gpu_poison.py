"""Buffers filled with NaN at allocation (tpc_params.poison = 1): every value the library reads
must have been written first, so a poisoned handle gives bit-for-bit the results of a clean
one. A value read before it is written would turn the results into NaN."""
import numpy as np
import pytest

import paper_2202_11288_gb300 as tpc
from synth import uniform_pm1

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [  # (variant, delta, K, kernel_a, shift)
    (tpc.TPC_SPD, 0.125, 9, 0.0, 0.0),    # every level fits one block (single-block bottom)
    (tpc.TPC_NONSYM, 0.1, 14, 0.0, 0.0),  # strided levels above the bottom
    (tpc.TPC_SPD, 0.05, 19, 0.0, 0.0),    # both occupancy instances (m <= 2^18 and above)
    (tpc.TPC_WEAKLY, 0.1, 10, 0.5, 3.0),  # tridiagonal band, per-entry weights (shifted)
]


def _run(variant, delta, K, a, shift, precision, poison):
    S = tpc.Solver(delta, 2.0 ** -K, variant=variant, kernel_a=a, shift=shift,
                   precision=precision, poison=poison)
    try:
        b = torch.tensor(uniform_pm1(S.n, 31), device="cuda")
        x = torch.zeros_like(b)
        rc, it, rel = S.solve(b, x, tol=1e-10)
        ys = []
        for k in range(S.K, S.kc, -1):
            xk = torch.tensor(uniform_pm1(S.level_size(k), 40 + k), device="cuda")
            y = torch.empty_like(xk)
            S.apply(k, xk, y)
            ys.append(y.cpu().numpy())
            if precision == tpc.TPC_MIXED:
                y32 = torch.empty_like(xk, dtype=torch.float32)
                S.apply_f32(k, xk.float(), y32)
                ys.append(y32.cpu().numpy())
        torch.cuda.synchronize()
        return rc, it, rel, x.cpu().numpy(), ys
    finally:
        S.close()


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("precision", [tpc.TPC_FP64, tpc.TPC_MIXED])
def test_poisoned_buffers_change_nothing(case, precision):
    clean = _run(*case, precision, 0)
    poisoned = _run(*case, precision, 1)
    assert clean[0] == tpc.TPC_OK and clean[2] < 1e-10
    assert poisoned[:3] == clean[:3]
    assert np.array_equal(poisoned[3], clean[3])
    for yp, yc in zip(poisoned[4], clean[4]):
        assert np.all(np.isfinite(yp))
        assert np.array_equal(yp, yc)
