"""The set-up autotuner of the three-pass FFT products: the factorisation m = R1 x L of every
level's transform and the tile width of its strided passes. The factorisation changes the
order of the radix steps (every choice is the same transform, to rounding) and the width which
block transforms which column; so a solve with the tuned plans agrees with the fixed rule's to
rounding (FP64), or within the solver tolerance (mixed precision), and two handles of one
process with the same level sizes use the same plans (the process-wide table) and agree
bitwise. Every candidate plan is checked against the oracle in tests/test_gpu_fft_plans.py."""
import numpy as np
import pytest

import paper_2202_11288_gb300 as tpc
from synth import uniform_pm1

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("precision", [tpc.TPC_FP64, tpc.TPC_MIXED])
@pytest.mark.parametrize("variant", [tpc.TPC_SPD, tpc.TPC_NONSYM])
def test_autotune_agrees_with_the_fixed_rule(precision, variant):
    K, delta = 18, 0.05
    results = []
    for autotune in (0, 1):
        S = tpc.Solver(delta, 2.0 ** -K, variant=variant, precision=precision, autotune=autotune)
        try:
            b = torch.tensor(uniform_pm1(S.n, 31), device="cuda")
            x = torch.zeros_like(b)
            rc, it, rel = S.solve(b, x, tol=1e-10)
            assert rc == tpc.TPC_OK
            results.append((x.cpu().numpy(), it, rel))
        finally:
            S.close()
    x0, x1 = results[0][0], results[1][0]
    diff = np.max(np.abs(x0 - x1)) / np.max(np.abs(x0))
    if precision == tpc.TPC_FP64:
        # FP64 products differ in the rounding of one entry: the iterates stay within 1e-12
        assert diff <= 1e-12 and results[0][1] == results[1][1], (diff, results[0][1:])
    else:
        # FP32 products differ at the FP32 rounding level; both solutions meet the FP64
        # residual tolerance 1e-10, so they differ by at most cond(A) * 1e-10 (cond < 1e3 here)
        assert diff <= 1e-7 and abs(results[0][1] - results[1][1]) <= 1, (diff, results[0][1:])


def test_tuned_widths_shared_by_handles():
    K, delta = 17, 0.1
    xs = []
    for _ in range(2):
        S = tpc.Solver(delta, 2.0 ** -K, precision=tpc.TPC_MIXED, autotune=1)
        try:
            b = torch.tensor(uniform_pm1(S.n, 7), device="cuda")
            x = torch.zeros_like(b)
            rc, it, rel = S.solve(b, x, tol=1e-10)
            assert rc == tpc.TPC_OK
            xs.append(x.cpu().numpy())
        finally:
            S.close()
    assert np.array_equal(xs[0], xs[1])


def test_autotune_rejects_other_values():
    with pytest.raises(tpc.TpcError):
        tpc.Solver(0.05, 2.0 ** -12, autotune=2)
