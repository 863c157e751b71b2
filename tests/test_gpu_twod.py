"""2-D Toeplitz-like-plus-Cross solver (tpc2d_*, through the C ABI) against the 2-D oracle
(oracle/twod.py: dense assembly from the exact 1-D integrals, dense Galerkin with R (x) R).

Tolerances as for 1-D: FP64 products 1e-12 ||A2||_1 ||x|| (and 1e-12 plain relative for uniform
operands), FP32 products 2e-6 log2(m) ||A2||_1 ||x||, V-cycle iterates and solutions 1e-10
relative after the same number of cycles.
"""
import numpy as np
import pytest

import paper_2202_11288_gb300 as tpc
from oracle import large, model, twod
from oracle.model import NONSYM, SPD
from synth import uniform_pm1

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(x, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64)


@pytest.fixture(scope="module")
def oracle5():
    out = {}
    for variant in (SPD, NONSYM):
        N = 32
        r = model.horizon_ratio(0.125, 1.0 / N)
        out[variant] = twod.Hierarchy(twod.assemble(variant, N, r), kc=3)
    return out


@pytest.mark.parametrize("variant", [SPD, NONSYM])
def test_products_every_level_fp64_and_fp32(oracle5, variant):
    K, delta = 5, 0.125
    H = oracle5[variant]
    S = tpc.Solver2D(delta, 2.0 ** -K, variant=variant, precision=tpc.TPC_MIXED)
    try:
        for k in range(K, H.kc, -1):
            A = H.A[k]
            nn = A.shape[0]
            norm1 = np.abs(A).sum(0).max()
            n = int(round(nn ** 0.5))
            xs = [uniform_pm1(nn, 60 + k),
                  np.outer(np.sin(np.pi * np.arange(1, n + 1) / (n + 1)),
                           np.cos(np.pi * np.arange(1, n + 1) / (n + 1))).ravel()]
            for j, x in enumerate(xs):
                ref = A @ x
                yd = torch.empty(nn, dtype=torch.float64, device="cuda")
                S.apply(k, _dev(x), yd)
                err = np.linalg.norm(_host(yd) - ref)
                assert err <= 1e-12 * norm1 * np.linalg.norm(x), (k, j, err)
                if j == 0:
                    assert err <= 1e-12 * np.linalg.norm(ref)
                x32 = x.astype(np.float32).astype(np.float64)
                yd32 = torch.empty(nn, dtype=torch.float32, device="cuda")
                S.apply_f32(k, _dev(x32, torch.float32), yd32)
                err32 = np.linalg.norm(_host(yd32) - A @ x32)
                assert err32 <= 2e-6 * (k + 1) * norm1 * np.linalg.norm(x32), (k, j, err32)
    finally:
        S.close()


def _norm1_bound(variant, N, r):
    """||A2||_1 <= 2 ||A||_1 + ||A||_1^2 / d from the 1-D blocks (A2 = A(x)I + I(x)A - A(x)A/d)."""
    bl = large.block_lists(variant, N, r)
    g = {k: np.abs(c).sum() + np.abs(rw[1:]).sum() for k, (c, rw) in bl.items()}
    a1 = max(g["A"] + g["C"], g["B"] + g["D"])
    return 2.0 * a1 + a1 * a1 / (12.0 * r)


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("K,delta", [(6, 0.1), (9, 0.1), (11, 0.1)])
def test_finest_product_large(variant, K, delta):
    """Finest level against the oracle's product d (U - M U M^T) (1-D FFT convolutions)."""
    N = 1 << K
    r = model.horizon_ratio(delta, 1.0 / N)
    S = tpc.Solver2D(delta, 2.0 ** -K, variant=variant, precision=tpc.TPC_MIXED)
    try:
        nn = S.nn
        x = uniform_pm1(nn, 70 + K)
        ref = twod.matvec_large(variant, N, r, x)
        norm1 = _norm1_bound(variant, N, r)
        yd = torch.empty(nn, dtype=torch.float64, device="cuda")
        S.apply(K, _dev(x), yd)
        err = np.linalg.norm(_host(yd) - ref)
        assert err <= 1e-12 * norm1 * np.linalg.norm(x), err
        x32 = x.astype(np.float32).astype(np.float64)
        yd32 = torch.empty(nn, dtype=torch.float32, device="cuda")
        S.apply_f32(K, _dev(x32, torch.float32), yd32)
        err32 = np.linalg.norm(_host(yd32) - twod.matvec_large(variant, N, r, x32))
        assert err32 <= 2e-6 * (K + 1) * norm1 * np.linalg.norm(x32), err32
    finally:
        S.close()


@pytest.mark.parametrize("variant", [SPD, NONSYM])
def test_vcycle_iterate(oracle5, variant):
    K, delta = 5, 0.125
    H = oracle5[variant]
    S = tpc.Solver2D(delta, 2.0 ** -K, variant=variant)
    try:
        nn = S.nn
        rhs = uniform_pm1(nn, 8)
        ed = torch.empty(nn, dtype=torch.float64, device="cuda")
        S.vcycle(_dev(rhs), ed)
        ref = twod.vcycle(H, K, rhs)
        assert np.linalg.norm(_host(ed) - ref) <= 1e-10 * np.linalg.norm(ref)
    finally:
        S.close()


@pytest.mark.parametrize("variant", [SPD, NONSYM])
def test_solve_fp64_iterates_and_mixed(oracle5, variant):
    K, delta = 5, 0.125
    H = oracle5[variant]
    A = H.A[K]
    b = uniform_pm1(A.shape[0], 9)
    u, it_ref, rel_ref, iterates = twod.solve(H, b, tol=1e-10)
    S = tpc.Solver2D(delta, 2.0 ** -K, variant=variant)
    try:
        xd = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
        rc, it, rel = S.solve(_dev(b), xd, tol=1e-10)
        x = _host(xd)
    finally:
        S.close()
    assert rc == tpc.TPC_OK and rel < 1e-10 and it == it_ref
    assert np.linalg.norm(x - iterates[it - 1]) <= 1e-10 * np.linalg.norm(iterates[it - 1])
    S = tpc.Solver2D(delta, 2.0 ** -K, variant=variant, precision=tpc.TPC_MIXED)
    try:
        xd = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
        rc, it, rel = S.solve(_dev(b), xd, tol=1e-10)
        xm = _host(xd)
    finally:
        S.close()
    assert rc == tpc.TPC_OK and rel < 1e-10
    assert np.linalg.norm(b - A @ xm) <= 1.01e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("variant", [SPD, NONSYM])
def test_mixed_solve_larger(variant):
    """N = 2^9 per axis (1023^2 unknowns), delta = 0.1: the mixed solver reaches 1e-10, checked
    with the oracle's product."""
    K, delta = 9, 0.1
    N = 1 << K
    r = model.horizon_ratio(delta, 1.0 / N)
    S = tpc.Solver2D(delta, 2.0 ** -K, variant=variant, precision=tpc.TPC_MIXED)
    try:
        b = uniform_pm1(S.nn, 10)
        xd = torch.zeros(S.nn, dtype=torch.float64, device="cuda")
        rc, it, rel = S.solve(_dev(b), xd, tol=1e-10)
        assert rc == tpc.TPC_OK and rel < 1e-10
        res = b - twod.matvec_large(variant, N, r, _host(xd))
        assert np.linalg.norm(res) <= 1.05e-10 * np.linalg.norm(b)
    finally:
        S.close()


def test_setup_rejects_what_it_does_not_build():
    with pytest.raises(tpc.TpcError) as ei:
        tpc.Solver2D(0.1, 2.0 ** -12)                       # m = 8192 per axis
    assert ei.value.code == tpc.TPC_EINVAL
    with pytest.raises(tpc.TpcError) as ei:
        tpc.Solver2D(0.1, 2.0 ** -8, kernel=1, kernel_a=0.25)
    assert ei.value.code == tpc.TPC_ENOTSUP
    with pytest.raises(tpc.TpcError) as ei:
        tpc.Solver2D(0.1, 2.0 ** -8, variant=tpc.TPC_WEAKLY, kernel_a=0.5)
    assert ei.value.code == tpc.TPC_EINVAL


@pytest.mark.parametrize("variant", [SPD, NONSYM])
def test_fgmres_restart_cycle_matches_oracle(oracle5, variant):
    """The flexible GMRES outer iteration of the 2-D solver (FP64): the iterate after one restart
    cycle of 4 steps equals the oracle's (oracle/krylov.py with the 2-D oracle V-cycle), and the
    solve reaches 1e-10 in no more V-cycles than the stationary iteration."""
    from oracle import krylov
    K, delta = 5, 0.125
    H = oracle5[variant]
    A = H.A[K]
    b = uniform_pm1(A.shape[0], 19)
    u1, _, _ = krylov.restart_cycle(A, b, np.zeros_like(b), lambda v: twod.vcycle(H, K, v), 4)
    S = tpc.Solver2D(delta, 2.0 ** -K, variant=variant, outer=tpc.TPC_OUTER_FGMRES,
                     inner_cycles=4, max_iters=1)
    try:
        xd = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
        rc, it, rel = S.solve(_dev(b), xd, tol=1e-14)
        assert it == 1
        assert np.linalg.norm(_host(xd) - u1) <= 1e-9 * np.linalg.norm(u1)
    finally:
        S.close()
    cycles = {}
    for outer in (tpc.TPC_OUTER_VCYCLE, tpc.TPC_OUTER_FGMRES):
        S = tpc.Solver2D(delta, 2.0 ** -K, variant=variant, outer=outer, inner_cycles=6)
        try:
            xd = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
            rc, it, rel = S.solve(_dev(b), xd, tol=1e-10)
            assert rc == tpc.TPC_OK and rel < 1e-10
            assert np.linalg.norm(b - A @ _host(xd)) <= 1.01e-10 * np.linalg.norm(b)
            cycles[outer] = S.last_cycles()
        finally:
            S.close()
    assert cycles[tpc.TPC_OUTER_FGMRES] <= cycles[tpc.TPC_OUTER_VCYCLE]


def test_fgmres_mixed_on_a_slowly_converging_horizon():
    """r = 1 (delta = h): the stationary 2-D V-cycle iteration needs about a hundred V-cycles;
    the mixed FGMRES solve reaches 1e-10 in far fewer, checked with the oracle's product."""
    K, delta = 6, 2.0 ** -6
    N = 1 << K
    res = {}
    for outer in (tpc.TPC_OUTER_VCYCLE, tpc.TPC_OUTER_FGMRES):
        S = tpc.Solver2D(delta, 2.0 ** -K, variant=NONSYM, precision=tpc.TPC_MIXED, outer=outer,
                         inner_cycles=8, max_iters=200)
        try:
            b = uniform_pm1(S.nn, 23)
            xd = torch.zeros(S.nn, dtype=torch.float64, device="cuda")
            rc, it, rel = S.solve(_dev(b), xd, tol=1e-10)
            assert rc == tpc.TPC_OK and rel < 1e-10
            x = _host(xd)
            r = b - twod.matvec_large(NONSYM, N, 1, x)
            assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b)
            res[outer] = S.last_cycles()
        finally:
            S.close()
    assert 2 * res[tpc.TPC_OUTER_FGMRES] <= res[tpc.TPC_OUTER_VCYCLE], res
