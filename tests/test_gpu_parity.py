"""GPU path (through the C ABI) against the oracle, element by element.

Tolerances (FP64): matrix-vector products 1e-12 normwise, ||y - y_ref|| <= 1e-12 ||A||_1 ||x||,
and 1e-12 plain relative for seeded uniform[-1,1) operands; V-cycle iterates and solutions
1e-10 relative after the same number of cycles.
"""
import numpy as np
import pytest

import paper_2202_11288_gb300 as tpc
from oracle import amg, large, model
from oracle.model import NONSYM, SPD
from synth import uniform_pm1

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def oracle_hierarchy(variant, K, delta, kc=3, shift=0.0):
    N = 1 << K
    A = model.assemble(variant, N, model.horizon_ratio(delta, 1.0 / N))
    if shift:
        A = A + shift * np.eye(A.shape[0])
    return amg.Hierarchy(A, kc=kc)


@pytest.fixture(scope="module")
def solvers():
    cache = {}

    def get(variant, K, delta, **kw):
        key = (variant, K, delta, tuple(sorted(kw.items())))
        if key not in cache:
            cache[key] = tpc.Solver(delta, 2.0 ** -K, variant=variant, **kw)
        return cache[key]

    yield get
    for s in cache.values():
        s.close()


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("K,delta", [(7, 0.125), (10, 0.05), (11, 0.2)])
def test_matvec_every_level(solvers, variant, K, delta):
    """tpc_apply at every level (single-CTA and three-kernel pipelines) vs dense R A P."""
    S = solvers(variant, K, delta)
    H = oracle_hierarchy(variant, K, delta)
    for k in range(K, H.kc, -1):
        A = H.A[k]
        n = A.shape[0]
        norm1 = np.abs(A).sum(0).max()
        xs = [uniform_pm1(n, 100 + k), np.sin(np.pi * np.arange(1, n + 1) / (n + 1))]
        for j, x in enumerate(xs):
            yd = torch.empty(n, dtype=torch.float64, device="cuda")
            S.apply(k, dev(x), yd)
            y = host(yd)
            ref = A @ x
            err = np.linalg.norm(y - ref)
            assert err <= 1e-12 * norm1 * np.linalg.norm(x), (k, j, err)
            if j == 0:
                assert err <= 1e-12 * np.linalg.norm(ref), (k, err / np.linalg.norm(ref))


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("K,delta,kw", [(7, 0.125, {}), (10, 0.05, {}),
                                        (8, 0.125, {"omega_pre": 1.0, "omega_post": 0.5}),
                                        (8, 0.125, {"m1": 2, "m2": 3}),
                                        (6, 0.125, {"coarsest_level": 1})])
def test_vcycle_iterate(solvers, variant, K, delta, kw):
    """One V-cycle of Algorithm 2 (tpc_vcycle) vs the oracle's recursive dense V-cycle."""
    S = solvers(variant, K, delta, **kw)
    H = oracle_hierarchy(variant, K, delta, kc=kw.get("coarsest_level", 3))
    vc = {k: kw[k] for k in ("m1", "m2", "omega_pre", "omega_post") if k in kw}
    n = H.A[K].shape[0]
    r = uniform_pm1(n, 7)
    ed = torch.empty(n, dtype=torch.float64, device="cuda")
    S.vcycle(dev(r), ed)
    e = host(ed)
    ref = amg.vcycle(H, K, r, **vc)
    assert np.linalg.norm(e - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("rhs", ["uniform", "manufactured"])
@pytest.mark.parametrize("K", [7, 9])
def test_solve_matches_oracle_iterates(solvers, variant, rhs, K):
    """tpc_solve to 1e-10: same number of cycles as the oracle, same iterate to 1e-10."""
    delta = 0.125
    S = solvers(variant, K, delta)
    H = oracle_hierarchy(variant, K, delta)
    N = 1 << K
    r = model.horizon_ratio(delta, 1.0 / N)
    if rhs == "uniform":
        b = uniform_pm1(2 * N - 1, 3)
    else:
        b, _ = model.manufactured(variant, N, r)
    xd = torch.zeros(2 * N - 1, dtype=torch.float64, device="cuda")
    rc, it, rel = S.solve(dev(b), xd, tol=1e-10)
    x = host(xd)
    u, it_ref, rel_ref, iterates = amg.solve(H, b, tol=1e-10)
    assert rc == tpc.TPC_OK and rel < 1e-10
    assert it == it_ref
    assert np.linalg.norm(x - iterates[it - 1]) <= 1e-10 * np.linalg.norm(iterates[it - 1])
    A = H.A[K]
    assert np.linalg.norm(b - A @ x) <= 1.01e-10 * np.linalg.norm(b)


def test_manufactured_solution_accuracy(solvers):
    """The GPU solution of the manufactured problem has the discretisation error of the
    scheme (order 4 at fixed delta): error at N=512 about 16x below N=256."""
    errs = []
    for K in (8, 9):
        N = 1 << K
        r = model.horizon_ratio(0.125, 1.0 / N)
        b, uex = model.manufactured(SPD, N, r)
        S = solvers(SPD, K, 0.125)
        xd = torch.zeros(2 * N - 1, dtype=torch.float64, device="cuda")
        S.solve(dev(b), xd, tol=1e-13)
        errs.append(np.max(np.abs(host(xd) - uex)))
    assert 3.8 < np.log2(errs[0] / errs[1]) < 4.2


@pytest.mark.parametrize("K,delta,kw", [
    (3, 0.125, {"coarsest_level": 3}),   # one level: the coarse solve alone
    (4, 0.125, {}),                      # two-grid
    (5, 1.4, {}),                        # r = 44 > N: truncated bands
    (12, 0.25, {"variant": NONSYM}),
    (6, 0.125, {"shift": 2.5}),
])
def test_edge_cases_converge(solvers, K, delta, kw):
    kw = dict(kw)
    variant = kw.pop("variant", SPD)
    S = solvers(variant, K, delta, **kw)
    H = oracle_hierarchy(variant, K, delta, kc=kw.get("coarsest_level", 3),
                         shift=kw.get("shift", 0.0))
    n = (1 << (K + 1)) - 1
    b = uniform_pm1(n, 9)
    xd = torch.zeros(n, dtype=torch.float64, device="cuda")
    rc, it, rel = S.solve(dev(b), xd, tol=1e-10)
    x = host(xd)
    assert rc == tpc.TPC_OK
    A = H.A[K]
    assert np.linalg.norm(b - A @ x) <= 1.01e-10 * np.linalg.norm(b)
    if K == kw.get("coarsest_level", -1):
        assert it == 1


def test_small_horizon_iterates_match(solvers):
    """delta < h (r = 1): the paper's transfers converge slowly there (the oracle needs more
    than 300 cycles at N = 256), so compare the iterate after a fixed number of cycles."""
    K, delta, cycles = 8, 0.001, 25
    S = solvers(SPD, K, delta, max_iters=cycles)
    H = oracle_hierarchy(SPD, K, delta)
    n = (1 << (K + 1)) - 1
    b = uniform_pm1(n, 9)
    xd = torch.zeros(n, dtype=torch.float64, device="cuda")
    rc, it, rel = S.solve(dev(b), xd, tol=1e-10)
    _, it_ref, rel_ref, iterates = amg.solve(H, b, tol=1e-10, max_iters=cycles)
    assert rc == tpc.TPC_ENOTCONV and it == it_ref == cycles
    ref = iterates[-1]
    assert np.linalg.norm(host(xd) - ref) <= 1e-10 * np.linalg.norm(ref)
    assert abs(rel - rel_ref) <= 1e-8 * rel_ref


def test_zero_rhs_initial_guess_and_host_buffers(solvers):
    S = solvers(SPD, 9, 0.125)
    n = S.n
    b = uniform_pm1(n, 4)
    # b = 0: nothing to do
    xd = torch.full((n,), 5.0, dtype=torch.float64, device="cuda")
    rc, it, rel = S.solve(torch.zeros(n, dtype=torch.float64, device="cuda"), xd)
    assert rc == tpc.TPC_OK and it == 0 and not host(xd).any()
    # device solve, then the host-buffer entry point: identical bits
    xd = torch.zeros(n, dtype=torch.float64, device="cuda")
    S.solve(dev(b), xd)
    xh = np.zeros(n)
    rc2, it2, rel2 = S.solve_host(b, xh)
    assert np.array_equal(host(xd), xh)
    # repeated solves are bitwise reproducible
    xd2 = torch.zeros(n, dtype=torch.float64, device="cuda")
    S.solve(dev(b), xd2)
    assert torch.equal(xd, xd2)
    # resume: 1e-5 from zero, then 1e-5 relative to the restart residual from that iterate
    _, it_full, _ = S.solve(dev(b), xd2, tol=1e-10)
    xr = torch.zeros(n, dtype=torch.float64, device="cuda")
    rc_a, it_a, _ = S.solve(dev(b), xr, tol=1e-5)
    rc_b, it_b, _ = S.solve(dev(b), xr, tol=1e-5, use_x0=True)
    assert rc_a == rc_b == tpc.TPC_OK
    assert abs(it_a + it_b - it_full) <= 1
    H = oracle_hierarchy(SPD, 9, 0.125)
    assert np.linalg.norm(b - H.A[9] @ host(xr)) <= 2e-10 * np.linalg.norm(b)


def test_not_converged_status(solvers):
    S = solvers(SPD, 8, 0.125, max_iters=2)
    b = uniform_pm1(S.n, 1)
    xd = torch.zeros(S.n, dtype=torch.float64, device="cuda")
    rc, it, rel = S.solve(dev(b), xd, tol=1e-12)
    assert rc == tpc.TPC_ENOTCONV and it == 2 and rel > 1e-12


def test_bad_arguments(solvers):
    S = solvers(SPD, 7, 0.125)
    x = torch.zeros(S.n, dtype=torch.float64, device="cuda")
    with pytest.raises(tpc.TpcError):
        S.apply(3, x, x.clone())        # coarsest level is held as an inverse
    with pytest.raises(tpc.TpcError):
        S.apply(7, x, x)                # aliasing
    with pytest.raises(tpc.TpcError):
        S.apply(9, x, x.clone())        # level out of range
    with pytest.raises(tpc.TpcError) as ei:
        tpc.Solver(0.05, 2.0 ** -23)    # m = 2^24 is beyond this build's plans
    assert ei.value.code == tpc.TPC_ENOTSUP


def test_full_size_finest_product_and_solve():
    """N = 2^22, delta = 0.05 (8,388,607 unknowns, r = 209715): sampled rows of the finest
    product against the oracle's rows, the whole product against the oracle's FFT
    convolution, and a solve whose residual the oracle recomputes."""
    K, delta = 22, 0.05
    N = 1 << K
    r = model.horizon_ratio(delta, 1.0 / N)
    S = tpc.Solver(delta, 2.0 ** -K)
    try:
        n = S.n
        x = uniform_pm1(n, 21)
        yd = torch.empty(n, dtype=torch.float64, device="cuda")
        S.apply(K, dev(x), yd)
        y = host(yd)
        rows = [0, 1, 2, r - 1, r, r + 1, N // 2, N - 3, N - 2, N - 1, N, N + 1, N + r,
                n // 2 + 12345, n - 2, n - 1]
        R = large.rows(SPD, N, r, rows)
        ref_rows = R @ x
        scale = np.abs(R).sum(1) * np.abs(x).max()
        assert np.all(np.abs(y[rows] - ref_rows) <= 1e-12 * scale)
        ref = large.matvec(SPD, N, r, x)
        assert np.linalg.norm(y - ref) <= 1e-12 * np.linalg.norm(ref)
        b = uniform_pm1(n, 0)
        xd = torch.zeros(n, dtype=torch.float64, device="cuda")
        rc, it, rel = S.solve(dev(b), xd, tol=1e-10)
        assert rc == tpc.TPC_OK and rel < 1e-10 and it <= 20
        res = b - large.matvec(SPD, N, r, host(xd))
        assert np.linalg.norm(res) <= 1.05e-10 * np.linalg.norm(b)
    finally:
        S.close()
