"""Flexible GMRES outer iteration (tpc_params.outer = TPC_OUTER_FGMRES) against the oracle.

FP64: the iterate after each restart cycle equals the oracle's FGMRES iterate (oracle/krylov.py,
the oracle V-cycle as preconditioner, the same step counts) to 1e-9 relative. Mixed precision:
the solution reaches relative residual 1e-10 and the direct (LU) solution of the oracle's
matrix to within what the conditioning allows. The fractional nonsymmetric case where the
stationary iteration diverges converges.
"""
import numpy as np
import pytest

import paper_2202_11288_gb300 as tpc
from oracle import amg, fractional, krylov, model
from oracle.model import NONSYM, SPD
from synth import uniform_pm1

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def constant_system(variant, K, delta):
    N = 1 << K
    return model.assemble(variant, N, model.horizon_ratio(delta, 1.0 / N))


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("K,delta,steps", [(7, 0.125, 4), (10, 0.05, 6), (10, 0.2, 3)])
def test_fp64_restart_cycles_match_oracle(variant, K, delta, steps):
    A = constant_system(variant, K, delta)
    H = amg.Hierarchy(A, kc=3)
    prec = lambda v: amg.vcycle(H, H.K, v)
    b = uniform_pm1(A.shape[0], 31 + K)
    S = tpc.Solver(delta, 2.0 ** -K, variant=variant, precision=tpc.TPC_FP64,
                   outer=tpc.TPC_OUTER_FGMRES, inner_cycles=steps, max_iters=1)
    try:
        x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
        rc, it, rel = S.solve(dev(b), x, tol=1e-14)
        assert it == 1 and tpc.tpc_last_solve_cycles(S.handle) == steps
        u1, _, _ = krylov.restart_cycle(A, b, np.zeros_like(b), prec, steps)
        got = host(x)
        assert np.linalg.norm(got - u1) <= 1e-9 * np.linalg.norm(u1)
        # a second cycle: its step count is the solver's choice, read back from the cycle count
        S2 = tpc.Solver(delta, 2.0 ** -K, variant=variant, precision=tpc.TPC_FP64,
                        outer=tpc.TPC_OUTER_FGMRES, inner_cycles=steps, max_iters=2)
        try:
            x2 = torch.zeros_like(x)
            rc, it, rel = S2.solve(dev(b), x2, tol=1e-14)
            c2 = tpc.tpc_last_solve_cycles(S2.handle) - steps
            assert it == 2 and 1 <= c2 <= steps
            u2, _, _ = krylov.restart_cycle(A, b, u1, prec, c2)
            assert np.linalg.norm(host(x2) - u2) <= 1e-9 * np.linalg.norm(u2)
        finally:
            S2.close()
    finally:
        S.close()


@pytest.mark.parametrize("precision", [tpc.TPC_FP64, tpc.TPC_MIXED])
@pytest.mark.parametrize("variant", [SPD, NONSYM])
def test_solution_matches_direct_solve_in_fewer_vcycles(precision, variant):
    K, delta = 10, 0.05
    A = constant_system(variant, K, delta)
    b = uniform_pm1(A.shape[0], 5)
    x_lu = np.linalg.solve(A, b)
    res = {}
    for outer in (tpc.TPC_OUTER_VCYCLE, tpc.TPC_OUTER_FGMRES):
        S = tpc.Solver(delta, 2.0 ** -K, variant=variant, precision=precision, outer=outer)
        try:
            x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
            rc, it, rel = S.solve(dev(b), x, tol=1e-10)
            assert rc == tpc.TPC_OK and rel < 1e-10
            res[outer] = (host(x), tpc.tpc_last_solve_cycles(S.handle))
            # the residual the solver reports is the true one
            r = b - A @ res[outer][0]
            assert abs(np.linalg.norm(r) / np.linalg.norm(b) - rel) <= 1e-3 * rel + 1e-15
        finally:
            S.close()
    xk, cyc_k = res[tpc.TPC_OUTER_FGMRES]
    cond_bound = 1e-10 * np.linalg.cond(A)
    assert np.linalg.norm(xk - x_lu) <= cond_bound * np.linalg.norm(x_lu)
    assert cyc_k <= res[tpc.TPC_OUTER_VCYCLE][1]


@pytest.mark.parametrize("precision", [tpc.TPC_FP64, tpc.TPC_MIXED])
def test_fractional_nonsymmetric_converges_where_the_stationary_iteration_diverges(precision):
    """a = 0.45, nonsymmetric, geometric transfer, K = 9: the stationary iteration diverges,
    FGMRES reaches 1e-10 and the LU solution."""
    K, delta, a = 9, 0.1, 0.45
    N = 1 << K
    A = fractional.assemble(NONSYM, N, int(np.floor(delta * N)), a)
    b = uniform_pm1(A.shape[0], 8)
    kw = dict(variant=tpc.TPC_NONSYM, kernel=1, kernel_a=a, transfer=tpc.TPC_TRANSFER_GEOMETRIC,
              precision=precision)
    S = tpc.Solver(delta, 2.0 ** -K, max_iters=40, **kw)
    try:
        x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
        try:
            rc, it, rel = S.solve(dev(b), x, tol=1e-10)
            assert not (rc == tpc.TPC_OK and rel < 1e-10)
        except tpc.TpcError as e:
            assert e.code == tpc.TPC_EDIVERGED
    finally:
        S.close()
    S = tpc.Solver(delta, 2.0 ** -K, outer=tpc.TPC_OUTER_FGMRES, inner_cycles=12, **kw)
    try:
        x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
        rc, it, rel = S.solve(dev(b), x, tol=1e-10)
        assert rc == tpc.TPC_OK and rel < 1e-10
        x_lu = np.linalg.solve(A, b)
        assert np.linalg.norm(host(x) - x_lu) <= 1e-10 * np.linalg.cond(A) * np.linalg.norm(x_lu)
    finally:
        S.close()


def test_large_mixed_solve_and_repeatability():
    """N = 2^20 (register-resident FP32 kernels on the finest levels): FGMRES reaches 1e-10 in
    no more V-cycles than the stationary iteration, and a repeated solve is bitwise equal."""
    K, delta = 20, 0.05
    n = (1 << (K + 1)) - 1
    b = torch.tensor(uniform_pm1(n, 12), device="cuda")
    cyc = {}
    for outer in (tpc.TPC_OUTER_VCYCLE, tpc.TPC_OUTER_FGMRES):
        S = tpc.Solver(delta, 2.0 ** -K, precision=tpc.TPC_MIXED, outer=outer)
        try:
            x = torch.zeros_like(b)
            rc, it, rel = S.solve(b, x, tol=1e-10)
            assert rc == tpc.TPC_OK and rel < 1e-10
            cyc[outer] = tpc.tpc_last_solve_cycles(S.handle)
            if outer == tpc.TPC_OUTER_FGMRES:
                x2 = torch.zeros_like(b)
                S.solve(b, x2, tol=1e-10)
                assert torch.equal(x, x2)
        finally:
            S.close()
    assert cyc[tpc.TPC_OUTER_FGMRES] <= cyc[tpc.TPC_OUTER_VCYCLE]


def test_outer_parameter_is_checked():
    with pytest.raises(tpc.TpcError):
        tpc.Solver(0.1, 2.0 ** -8, outer=5)
    with pytest.raises(tpc.TpcError):
        tpc.Solver(0.1, 2.0 ** -8, outer=tpc.TPC_OUTER_FGMRES, inner_cycles=33)
