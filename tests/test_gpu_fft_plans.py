"""FFT plans of the three-pass products: every factorisation m = R1 x L the set-up autotuner may
choose (log2 L the rule's value or one off it), with the register-resident FP32 kernels where
they take it and the general kernels elsewhere, forced through the process-wide plan table
(tpc_tune_set), element by element against the oracle's FFT-convolution product of the printed
Toeplitz blocks (section 2.2, eq. (2.9) / eq. (2.10)).

Tolerances as the other product tests: FP64 ||y - y_ref|| <= 1e-12 ||A||_1 ||x||; FP32
||y - y_ref|| <= 2e-6 log2(m) ||A||_1 ||x||.
"""
import numpy as np
import pytest

import paper_2202_11288_gb300 as tpc
from oracle import large, model
from oracle.model import NONSYM, SPD
from synth import uniform_pm1

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rule(logm):
    """The fixed rule's factorisation and tile width (log2 L, log2 C)."""
    logL = min(12, (logm + 1) // 2)
    logR1 = logm - logL
    return logL, max(0, min(4, 13 - logR1, logL - 9))


def width_rule(logm, logL):
    logR1 = logm - logL
    return max(0, min(4, 13 - logR1, logL - 9))


def reg_ok(logm, logL):
    return 20 <= logm <= 23 and logm - logL in (10, 11) and 10 <= logL <= 12


def candidates(logm):
    base = rule(logm)[0]
    out = []
    for d in (0, 1, -1):
        logL = base + d
        if d and not (7 <= logL <= 12 and 6 <= logm - logL <= 11):
            continue
        out.append(logL)
    return out


def pin_rule(word):
    for logm in range(13, 24):
        logL, logC = rule(logm)
        tpc.tpc_tune_set(word, logm, logL, logC, int(word == 4 and reg_ok(logm, logL)))


@pytest.fixture
def plan_table():
    tpc.tpc_tune_reset()
    yield
    tpc.tpc_tune_reset()


def _norm1(variant, N, r):
    bl = large.block_lists(variant, N, r)

    def gen_sum(name):
        col, row = bl[name]
        return np.abs(col).sum() + np.abs(row[1:]).sum()

    return max(gen_sum("A") + gen_sum("C"), gen_sum("B") + gen_sum("D"))


CASES = [(K, logL, v) for K in range(12, 23) for logL in candidates(K + 1)
         for v in ((SPD, NONSYM) if K <= 19 else (SPD,))]


@pytest.mark.parametrize("K,logL,variant", CASES)
def test_fp32_product_of_every_candidate_plan(plan_table, K, logL, variant):
    logm = K + 1
    pin_rule(4)
    pin_rule(8)
    reg = int(reg_ok(logm, logL))
    tpc.tpc_tune_set(4, logm, logL, width_rule(logm, logL), reg)
    assert tpc.tpc_tune_get(4, logm) == (logL, 2 if reg else width_rule(logm, logL), reg)
    delta = 0.05
    N = 1 << K
    r = model.horizon_ratio(delta, 1.0 / N)
    S = tpc.Solver(delta, 2.0 ** -K, variant=variant, precision=tpc.TPC_MIXED, autotune=1)
    try:
        x = uniform_pm1(S.n, 40 + K).astype(np.float32).astype(np.float64)
        xd = torch.tensor(x, dtype=torch.float32, device="cuda")
        yd = torch.empty_like(xd)
        S.apply_f32(K, xd, yd)
        torch.cuda.synchronize()
        y = yd.cpu().numpy().astype(np.float64)
        ref = large.matvec(variant, N, r, x)
        err = np.linalg.norm(y - ref)
        bound = 2e-6 * logm * _norm1(variant, N, r) * np.linalg.norm(x)
        assert np.isfinite(err) and err <= bound, (logL, reg, err / bound)
    finally:
        S.close()


@pytest.mark.parametrize("K,logL", [(K, logL) for K in (12, 15, 18, 21) for logL in candidates(K + 1)])
@pytest.mark.parametrize("logC", [0, None])
def test_fp64_product_of_every_candidate_plan(plan_table, K, logL, logC):
    logm = K + 1
    pin_rule(8)
    c = width_rule(logm, logL) if logC is None else logC
    tpc.tpc_tune_set(8, logm, logL, c, 0)
    delta = 0.05
    N = 1 << K
    r = model.horizon_ratio(delta, 1.0 / N)
    S = tpc.Solver(delta, 2.0 ** -K, variant=NONSYM, precision=tpc.TPC_FP64, autotune=1)
    try:
        x = uniform_pm1(S.n, 60 + K)
        xd = torch.tensor(x, device="cuda")
        yd = torch.empty_like(xd)
        S.apply(K, xd, yd)
        torch.cuda.synchronize()
        y = yd.cpu().numpy()
        ref = large.matvec(NONSYM, N, r, x)
        err = np.linalg.norm(y - ref)
        assert err <= 1e-12 * _norm1(NONSYM, N, r) * np.linalg.norm(x), (logL, c, err)
    finally:
        S.close()


def test_solve_with_the_other_plans_everywhere(plan_table):
    """Every three-pass level on the factorisation one off the rule (where there is one): the
    mixed solve reaches 1e-10 and agrees with the rule's to within what the tolerance allows."""
    K, delta = 20, 0.05
    b = torch.tensor(uniform_pm1((1 << (K + 1)) - 1, 77), device="cuda")
    sols = []
    for shifted in (False, True):
        tpc.tpc_tune_reset()
        pin_rule(4)
        pin_rule(8)
        if shifted:
            for logm in range(13, K + 2):
                alt = [l for l in candidates(logm) if l != rule(logm)[0]]
                if alt:
                    tpc.tpc_tune_set(4, logm, alt[0], width_rule(logm, alt[0]),
                                     int(reg_ok(logm, alt[0])))
        S = tpc.Solver(delta, 2.0 ** -K, precision=tpc.TPC_MIXED, autotune=1)
        try:
            x = torch.zeros_like(b)
            rc, it, rel = S.solve(b, x, tol=1e-10)
            assert rc == tpc.TPC_OK and rel < 1e-10
            sols.append(x.cpu().numpy())
        finally:
            S.close()
    diff = np.max(np.abs(sols[0] - sols[1])) / np.max(np.abs(sols[0]))
    assert diff <= 1e-7, diff


def test_plan_table_rejects_out_of_range_entries(plan_table):
    assert tpc.tpc_tune_get(4, 17) is None
    for args in [(4, 12, 7, 0, 0), (4, 17, 6, 0, 0), (4, 17, 13, 0, 0), (4, 23, 11, 0, 0),
                 (4, 17, 9, 5, 0), (8, 21, 11, 0, 1), (4, 19, 10, 0, 1), (2, 17, 9, 0, 0)]:
        with pytest.raises(tpc.TpcError):
            tpc.tpc_tune_set(*args)
    tpc.tpc_tune_set(4, 22, 12, 0, 1)
    assert tpc.tpc_tune_get(4, 22) == (12, 2, 1)
