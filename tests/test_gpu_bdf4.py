"""Time stepping on the GPU (section 5, eq. (5.1)): each step is tpc_bdf4_step on a handle
whose shift is sigma = 25 eta_h / (12 tau). The final errors are compared with the values the
paper prints in Tables 2 and 3 and the final level with the oracle's dense time stepping.

Tolerances: each shifted solve stops at a residual 1e-12 relative to its initial residual
(the previous level as initial guess); the shifted matrix is well conditioned (sigma dominates
the spectrum of A), so a step's solution error is of order 1e-12 times the change of the
solution per step, and over N steps the final level differs from the oracle's exact LU steps by
well under 1e-11 of max|u| (max|u| = 64 e). The printed errors (five digits) are met to three
units of their last digit."""
import math
import os

import numpy as np
import pytest

import paper_2202_11288_gb300 as tpc
from oracle import timestep
from oracle.model import NONSYM, SPD

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "bdf4_tables.txt")


def table_rows():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                v, N, d, e = line.split()
                N = int(N)
                r = N // 4 if d == "1/4" else int(math.floor(math.sqrt(N)))
                rows.append((SPD if v == "spd" else NONSYM, N, r, float(e)))
    return rows


def phi(x):
    return (1.0 + x) ** 6


def Phi(x):
    return (1.0 + x) ** 7 / 7.0


def collocation_x(N):
    return np.concatenate([np.arange(1, N), np.arange(1, N + 1) - 0.5]) / N


def run_gpu(variant, N, r, precision=tpc.TPC_FP64, tol=1e-12):
    h = tau = 1.0 / N
    delta = r * h
    p = tpc.tpc_default_params(variant=variant)
    sigma, hs = tpc.tpc_bdf4_coefficients(delta, h, tau, params=p)
    x = collocation_x(N)
    gamma = 3.0 / delta ** 3
    f = phi(x) - gamma * (Phi(x + delta) - Phi(x - delta) - 2.0 * delta * phi(x))
    j = np.arange(2 * r + 1)
    G = tpc.tpc_collocation_rhs(delta, h, f, phi(-j * 0.5 * h), phi(1.0 + j * 0.5 * h), params=p)
    S = tpc.Solver(delta, h, variant=variant, shift=sigma, precision=precision)
    try:
        g = torch.tensor(G, device="cuda")
        U = [torch.tensor(np.exp(k * tau) * phi(x), device="cuda") for k in range(4)]
        iters = []
        for k in range(4, N + 1):
            out = U[0]  # the oldest level is overwritten (it is read first)
            rc, it, rel = S.bdf4_step(U[3], U[2], U[1], U[0], hs, g, math.exp(k * tau), out,
                                      tol=tol)
            assert rc == tpc.TPC_OK, (k, rc, rel)
            iters.append(it)
            U = U[1:] + [out]
        torch.cuda.synchronize()
        UT = U[-1].cpu().numpy()
    finally:
        S.close()
    err = float(np.max(np.abs(UT - math.exp(N * tau) * phi(x))))
    return err, UT, iters


@pytest.mark.parametrize("variant,N,r,printed", table_rows())
def test_bdf4_on_gpu_matches_tables_and_oracle(variant, N, r, printed):
    err, UT, iters = run_gpu(variant, N, r)
    unit = 10.0 ** (math.floor(math.log10(printed)) - 4)
    _, U_ref = timestep.bdf4(variant, N, r)
    diff = np.max(np.abs(UT - U_ref)) / np.max(np.abs(U_ref))
    assert abs(err - printed) <= 3 * unit, (err, printed, diff, np.mean(iters))
    assert diff <= 1e-11, (diff, np.mean(iters))


def test_bdf4_mixed_precision():
    """FP32 V-cycles inside FP64 refinement give the same final level (N = 64, delta = 1/4)."""
    err64, U64, _ = run_gpu(SPD, 64, 16)
    err32, U32, _ = run_gpu(SPD, 64, 16, precision=tpc.TPC_MIXED)
    assert np.max(np.abs(U32 - U64)) <= 1e-11 * np.max(np.abs(U64))
    assert abs(err32 - 7.3840e-07) <= 3e-11


def test_bdf4_step_arguments():
    S = tpc.Solver(0.25, 1 / 32, shift=100.0)
    try:
        u = torch.zeros(S.n, dtype=torch.float64, device="cuda")
        with pytest.raises(tpc.TpcError):
            S.bdf4_step(u, u, u, None, 1.0, None, 1.0, u)
        with pytest.raises(tpc.TpcError):
            S.bdf4_step(u, u, u, u, float("nan"), None, 1.0, u)
        rc, it, rel = S.bdf4_step(u, u, u, u, 1.0, None, 1.0, u)  # zero data: zero solution
        assert rc == tpc.TPC_OK and torch.count_nonzero(u).item() == 0
    finally:
        S.close()
