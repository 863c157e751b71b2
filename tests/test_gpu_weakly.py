"""GPU path of the weakly singular model (section 2.1, eq. (2.3)) against the oracle:
products at every level (FFT for the Toeplitz part plus the tridiagonal band), V-cycle iterates,
and the BDF4 time stepping of Table 1.

Tolerances: products as in tests/test_gpu_parity.py (1e-12 ||A||_1 ||x|| in FP64, 2e-6 (k+1)
||A||_1 ||x|| in FP32); iterates 1e-10 relative after the same number of cycles; Table 1 as in
tests/test_oracle_weakly.py (five units of the last printed digit for N <= 128, 1 % at N = 256)
plus 2e-12 max|u| for the steps solved to 1e-12 (relative to their initial residual), and the
final level within 1e-11 max|u| of the oracle's."""
import math
import os

import numpy as np
import pytest

import paper_2202_11288_gb300 as tpc
from oracle import amg, weakly
from synth import uniform_pm1

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "bdf4_table1.txt")


def dev(x, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


@pytest.mark.parametrize("gamma", [0.0, 0.5, 0.9])
@pytest.mark.parametrize("K", [7, 9])
def test_products_every_level(gamma, K):
    N = 1 << K
    shift = 3.0
    A = weakly.assemble(N, gamma) + shift * np.eye(2 * N - 1)
    H = amg.Hierarchy(A, kc=3)
    S = tpc.Solver(0.1, 1.0 / N, variant=tpc.TPC_WEAKLY, kernel_a=gamma, shift=shift,
                   precision=tpc.TPC_MIXED)
    try:
        for k in range(K, H.kc, -1):
            Ak = H.A[k]
            x = uniform_pm1(Ak.shape[0], 40 + k)
            y = torch.empty(Ak.shape[0], dtype=torch.float64, device="cuda")
            S.apply(k, dev(x), y)
            torch.cuda.synchronize()
            ref = Ak @ x
            nrm = np.abs(Ak).sum(0).max() * np.linalg.norm(x)
            assert np.linalg.norm(y.cpu().numpy() - ref) <= 1e-12 * nrm, k
            y32 = torch.empty(Ak.shape[0], dtype=torch.float32, device="cuda")
            S.apply_f32(k, dev(x, torch.float32), y32)
            torch.cuda.synchronize()
            err32 = np.linalg.norm(y32.cpu().numpy().astype(np.float64) - ref)
            assert err32 <= 2e-6 * (k + 1) * nrm, k
    finally:
        S.close()


@pytest.mark.parametrize("gamma", [0.0, 0.5])
def test_vcycle_iterates_match_oracle(gamma):
    """Shifted system of one BDF4 step (sigma = 25 eta / (12 h)), omega = (1, 1/2) as in
    section 5: the GPU's iterates after 1, 2, 3 cycles equal the oracle's."""
    K = 9
    N = 1 << K
    sigma = 25.0 * weakly.eta(N, gamma) / 12.0 * N
    A = weakly.assemble(N, gamma) + sigma * np.eye(2 * N - 1)
    H = amg.Hierarchy(A, kc=3)
    b = uniform_pm1(2 * N - 1, 5)
    _, _, _, its = amg.solve(H, b, tol=0.0, max_iters=3, omega_pre=1.0, omega_post=0.5)
    for ncyc in (1, 2, 3):
        S = tpc.Solver(0.1, 1.0 / N, variant=tpc.TPC_WEAKLY, kernel_a=gamma, shift=sigma,
                       omega_pre=1.0, omega_post=0.5, max_iters=ncyc)
        try:
            x = torch.zeros(2 * N - 1, dtype=torch.float64, device="cuda")
            S.solve(dev(b), x, tol=0.0)
            torch.cuda.synchronize()
            ref = its[ncyc - 1]
            assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref), ncyc
        finally:
            S.close()


def L_phi(x, gamma):
    """L (1+x)^6 = int_0^1 ((1+x)^6 - (1+y)^6) |x - y|^{-gamma} dy in closed form."""
    s = 0.0
    for k in range(1, 7):
        ck = math.comb(6, k) * (1.0 + x) ** (6 - k)
        s -= ck * ((1.0 - x) ** (k + 1 - gamma) + (-1) ** k * x ** (k + 1 - gamma)) / (k + 1 - gamma)
    return s


def table_rows():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                g, N, e = line.split()
                rows.append((float(g), int(N), float(e)))
    return rows


@pytest.mark.parametrize("gamma,N,printed", table_rows())
def test_bdf4_table_1_on_gpu(gamma, N, printed):
    h = tau = 1.0 / N
    p = tpc.tpc_default_params(variant=tpc.TPC_WEAKLY, kernel_a=gamma)
    sigma, hs = tpc.tpc_bdf4_coefficients(0.1, h, tau, params=p)
    x = np.concatenate([np.arange(1, N), np.arange(1, N + 1) - 0.5]) / N
    phi = (1.0 + x) ** 6
    G = tpc.tpc_collocation_rhs(0.1, h, phi + L_phi(x, gamma), np.array([1.0]),
                                np.array([64.0]), params=p)
    S = tpc.Solver(0.1, h, variant=tpc.TPC_WEAKLY, kernel_a=gamma, shift=sigma)
    try:
        g = dev(G)
        U = [dev(math.exp(k * tau) * phi) for k in range(4)]
        for k in range(4, N + 1):
            out = U[0]
            rc, it, rel = S.bdf4_step(U[3], U[2], U[1], U[0], hs, g, math.exp(k * tau), out,
                                      tol=1e-12)
            assert rc == tpc.TPC_OK, (k, rc, rel)
            U = U[1:] + [out]
        torch.cuda.synchronize()
        UT = U[-1].cpu().numpy()
    finally:
        S.close()
    umax = float(np.max(np.abs(math.e * phi)))
    if N <= 128:
        _, U_ref = weakly.bdf4(N, gamma)
        assert np.max(np.abs(UT - U_ref)) <= 1e-11 * umax
    err = float(np.max(np.abs(UT - math.e * phi)))
    unit = 10.0 ** (math.floor(math.log10(printed)) - 4)
    # the oracle's tolerance plus what steps solved to 1e-12 (relative) may leave: 2e-12 max|u|
    tol = (5 * unit if N <= 128 else 0.01 * printed) + 2e-12 * umax
    assert abs(err - printed) <= tol, (err, printed)
