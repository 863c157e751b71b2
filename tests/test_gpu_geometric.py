"""GPU path with the geometric transfer (tpc_params.transfer = TPC_TRANSFER_GEOMETRIC, an
option of this build) against the oracle with the same transfer: products at every level,
V-cycle iterates (FP64: whole-level and strided kernels, both smoothing counts), and the
fractional-kernel solves the paper's transfer slows down."""
import numpy as np
import pytest
import sympy as sp

import paper_2202_11288_gb300 as tpc
from oracle import amg, fractional, model
from oracle.model import NONSYM, SPD
from synth import uniform_pm1

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GEO = tpc.TPC_TRANSFER_GEOMETRIC


def dev(x, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def _matrix(variant, N, r, a):
    return model.assemble(variant, N, r) if a is None else fractional.assemble(variant, N, r, a)


def _kw(a):
    return {} if a is None else {"kernel": 1, "kernel_a": float(a)}


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("a", [None, sp.Rational(1, 4)])
def test_products_every_level(variant, a):
    K, r = 10, 40
    N = 1 << K
    H = amg.Hierarchy(_matrix(variant, N, r, a), kc=3, transfer="geometric")
    S = tpc.Solver(r / N, 1.0 / N, variant=variant, transfer=GEO, precision=tpc.TPC_MIXED,
                   **_kw(a))
    try:
        for k in range(K, H.kc, -1):
            Ak = H.A[k]
            x = uniform_pm1(Ak.shape[0], 90 + k)
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
@pytest.mark.parametrize("a", [None, sp.Rational(1, 4)])
@pytest.mark.parametrize("K,r", [(7, 16), (10, 40)])
@pytest.mark.parametrize("m2", [1, 0])
def test_vcycle_iterates_match_oracle(variant, a, K, r, m2):
    N = 1 << K
    H = amg.Hierarchy(_matrix(variant, N, r, a), kc=3, transfer="geometric")
    b = uniform_pm1(2 * N - 1, 19)
    _, _, _, its = amg.solve(H, b, tol=0.0, max_iters=3, m2=m2)
    for ncyc in (1, 3):
        S = tpc.Solver(r / N, 1.0 / N, variant=variant, transfer=GEO, max_iters=ncyc, m2=m2,
                       **_kw(a))
        try:
            x = torch.zeros(2 * N - 1, dtype=torch.float64, device="cuda")
            S.solve(dev(b), x, tol=0.0)
            torch.cuda.synchronize()
            ref = its[ncyc - 1]
            assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref), ncyc
        finally:
            S.close()


@pytest.mark.parametrize("variant", [SPD, NONSYM])
def test_fractional_solves_converge_at_the_constant_kernels_rate(variant):
    """N = 2^14, delta = 0.05, a = 1/4: FP64 solve within 15 V-cycles and the mixed solve within
    4 FP64 residuals (its FP32 inner solves stop at a rounding floor that grows with the
    condition number), both to 1e-10; with the paper's transfer the FP64 solve takes about 150."""
    K, delta = 14, 0.05
    b = dev(uniform_pm1((1 << (K + 1)) - 1, 8))
    for prec in (tpc.TPC_FP64, tpc.TPC_MIXED):
        S = tpc.Solver(delta, 2.0 ** -K, variant=variant, kernel=1, kernel_a=0.25,
                       transfer=GEO, precision=prec)
        try:
            x = torch.zeros_like(b)
            rc, it, rel = S.solve(b, x, tol=1e-10)
            assert rc == tpc.TPC_OK and rel < 1e-10
            assert it <= (15 if prec == tpc.TPC_FP64 else 4)
            y = torch.empty_like(b)
            S.apply(K, x, y)
            torch.cuda.synchronize()
            assert (torch.linalg.norm(b - y) / torch.linalg.norm(b)).item() < 1.05e-10
        finally:
            S.close()


def test_server_mix_with_the_geometric_transfer_equals_lone_solves():
    """A server whose handles use the geometric transfer, fed constant- and fractional-kernel
    requests (a budget small enough to evict): every result equals, bit for bit and with the
    same iteration count, the lone solve of the same request."""
    import time
    keys = [(SPD, 0.05, 10, 1, 0.25), (NONSYM, 0.1, 11, 1, 0.3), (SPD, 0.2, 9, 0, 0.0),
            (NONSYM, 0.05, 12, 1, 0.1)]
    reqs = []
    for i in range(12):
        v, d, K, kk, a = keys[i % len(keys)]
        n = (1 << (K + 1)) - 1
        b = torch.tensor(uniform_pm1(n, 300 + i)).pin_memory()
        reqs.append((v, d, K, kk, a, b, torch.zeros(n, dtype=torch.float64).pin_memory()))
    srv = tpc.Server(hbm_budget_bytes=4 << 20, max_inflight=3, precision=tpc.TPC_MIXED,
                     transfer=GEO)
    try:
        tickets = {srv.submit(v, d, 2.0 ** -K, b, x, 1e-10, kk, a): i
                   for i, (v, d, K, kk, a, b, x) in enumerate(reqs)}
        got, t0 = [], time.time()
        while len(got) < len(reqs) and time.time() - t0 < 120:
            got += srv.poll(64, wait_ms=50)
        assert len(got) == len(reqs)
    finally:
        srv.close()
    for r in got:
        v, d, K, kk, a, b, x = reqs[tickets[r["ticket"]]]
        assert r["status"] == tpc.TPC_OK and r["relres"] < 1e-10
        S = tpc.Solver(d, 2.0 ** -K, variant=v, kernel=kk, kernel_a=a, transfer=GEO,
                       precision=tpc.TPC_MIXED)
        try:
            xa = np.zeros(b.numel())
            rc, it, rel = S.solve_host(b.numpy(), xa, tol=1e-10)
        finally:
            S.close()
        assert it == r["iters"] and rel == r["relres"]
        assert np.array_equal(xa, x.numpy())
