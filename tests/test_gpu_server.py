"""Request server (continuous batching): every result is the same alone and in the mix.

Requests of several problems are submitted at once into a server with few slots and a tight
device-memory budget (so hierarchies are evicted and rebuilt); each result must equal, bit for
bit and with the same iteration count, the solve of the same request alone on its own handle.
"""
import time

import numpy as np
import pytest

import paper_2202_11288_gb300 as tpc
from synth import uniform_pm1

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# (variant, delta, K, kernel, a); the last key differs from the first only in its kernel, so a
# hierarchy must not be shared across kernels
KEYS = [(tpc.TPC_SPD, 0.05, 10, 0, 0.0), (tpc.TPC_NONSYM, 0.1, 11, 0, 0.0),
        (tpc.TPC_SPD, 0.2, 9, 0, 0.0), (tpc.TPC_SPD, 0.125, 12, 0, 0.0),
        (tpc.TPC_NONSYM, 0.3, 10, 0, 0.0), (tpc.TPC_SPD, 0.05, 10, 1, 0.25)]


def _wait_all(srv, count, timeout_s=120.0):
    got = []
    t0 = time.time()
    while len(got) < count and time.time() - t0 < timeout_s:
        got += srv.poll(64, wait_ms=50)
    return got


def test_server_results_equal_alone_with_eviction():
    rng = np.random.default_rng(3)
    reqs = []
    for i in range(24):
        v, d, K, kk, a = KEYS[i % len(KEYS)] if i < len(KEYS) else KEYS[int(rng.integers(len(KEYS)))]
        n = (1 << (K + 1)) - 1
        b = torch.tensor(uniform_pm1(n, 700 + i)).pin_memory()
        x = torch.zeros(n, dtype=torch.float64).pin_memory()
        reqs.append((v, d, K, kk, a, b, x))
    # a budget below the six hierarchies' total (about 6 MB), so the LRU eviction runs
    srv = tpc.Server(hbm_budget_bytes=4 << 20, max_inflight=4, precision=tpc.TPC_MIXED)
    try:
        tickets = {srv.submit(v, d, 2.0 ** -K, b, x, 1e-10, kk, a): i
                   for i, (v, d, K, kk, a, b, x) in enumerate(reqs)}
        res = _wait_all(srv, len(reqs))
        assert len(res) == len(reqs)
        assert srv.outstanding() == 0
    finally:
        srv.close()
    for r in res:
        i = tickets[r["ticket"]]
        v, d, K, kk, a, b, x = reqs[i]
        assert r["status"] == tpc.TPC_OK and r["relres"] < 1e-10
        assert r["latency_s"] >= r["queue_s"] >= 0.0
        S = tpc.Solver(d, 2.0 ** -K, variant=v, kernel=kk, kernel_a=a, precision=tpc.TPC_MIXED)
        try:
            xa = np.zeros(b.numel())
            rc, it, rel = S.solve_host(b.numpy(), xa, tol=1e-10)
        finally:
            S.close()
        assert it == r["iters"] and rel == r["relres"]
        assert np.array_equal(xa, x.numpy())


def test_server_rejects_a_problem_larger_than_its_budget():
    srv = tpc.Server(hbm_budget_bytes=1 << 20, max_inflight=2)
    try:
        K = 12
        n = (1 << (K + 1)) - 1
        b, x = np.ones(n), np.zeros(n)
        srv.submit(tpc.TPC_SPD, 0.1, 2.0 ** -K, b, x)
        res = _wait_all(srv, 1)
        assert len(res) == 1 and res[0]["status"] == tpc.TPC_ENOMEM
    finally:
        srv.close()


def test_server_mix_of_2d_fractional_and_transfers_equals_alone():
    """2-D requests, a fractional kernel under the geometric transfer, requests that differ only
    in their transfer or their outer iteration: each result equals its lone solve bit for bit,
    and the occupancy statistics are consistent."""
    # (dim, variant, delta, K, kernel, a, transfer, outer); the last two keys repeat earlier ones
    # but for the outer iteration, so hierarchies must not be shared across it
    VC, FG = tpc.TPC_OUTER_VCYCLE, tpc.TPC_OUTER_FGMRES
    keys = [(2, tpc.TPC_SPD, 0.1, 6, 0, 0.0, tpc.TPC_TRANSFER_PAPER, VC),
            (2, tpc.TPC_NONSYM, 0.2, 5, 0, 0.0, tpc.TPC_TRANSFER_PAPER, VC),
            (1, tpc.TPC_SPD, 0.1, 11, 1, 0.3, tpc.TPC_TRANSFER_GEOMETRIC, VC),
            (1, tpc.TPC_SPD, 0.08, 10, 0, 0.0, tpc.TPC_TRANSFER_PAPER, VC),
            (1, tpc.TPC_SPD, 0.08, 10, 0, 0.0, tpc.TPC_TRANSFER_GEOMETRIC, VC),
            (2, tpc.TPC_NONSYM, 0.2, 5, 0, 0.0, tpc.TPC_TRANSFER_PAPER, FG),
            (1, tpc.TPC_SPD, 0.08, 10, 0, 0.0, tpc.TPC_TRANSFER_PAPER, FG)]
    reqs = []
    for i in range(21):
        dim, v, d, K, kk, a, tr, oi = keys[i % len(keys)]
        n1 = (1 << (K + 1)) - 1
        n = n1 * n1 if dim == 2 else n1
        b = torch.tensor(uniform_pm1(n, 900 + i)).pin_memory()
        x = torch.zeros(n, dtype=torch.float64).pin_memory()
        reqs.append((keys[i % len(keys)], b, x))
    srv = tpc.Server(max_inflight=6, precision=tpc.TPC_MIXED)
    try:
        srv.stats(reset=True)
        tickets = {srv.submit(v, d, 2.0 ** -K, b, x, 1e-10, kk, a, dim=dim, transfer=tr,
                              outer=oi): i
                   for i, ((dim, v, d, K, kk, a, tr, oi), b, x) in enumerate(reqs)}
        res = _wait_all(srv, len(reqs))
        assert len(res) == len(reqs)
        st = srv.stats()
    finally:
        srv.close()
    assert st["admitted"] == len(reqs) and st["setups"] == len(keys) and st["evictions"] == 0
    assert 0.0 < st["busy_s"] <= st["elapsed_s"]
    assert st["inflight_s"] >= st["busy_s"] and 1 <= st["max_inflight_seen"] <= 6
    for r in res:
        i = tickets[r["ticket"]]
        (dim, v, d, K, kk, a, tr, oi), b, x = reqs[i]
        assert r["status"] == tpc.TPC_OK and r["relres"] < 1e-10, (i, r)
        bd = b.cuda()
        xd = torch.zeros_like(bd)
        if dim == 2:
            S = tpc.Solver2D(d, 2.0 ** -K, variant=v, precision=tpc.TPC_MIXED, outer=oi)
        else:
            S = tpc.Solver(d, 2.0 ** -K, variant=v, kernel=kk, kernel_a=a, transfer=tr,
                           precision=tpc.TPC_MIXED, outer=oi)
        try:
            rc, it, rel = S.solve(bd, xd, tol=1e-10)
        finally:
            S.close()
        assert it == r["iters"] and rel == r["relres"], (i, it, r)
        assert torch.equal(xd.cpu(), x), i
