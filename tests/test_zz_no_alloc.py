"""tpc_apply_noalloc: the one-level product for callers that cannot allocate device memory.

Such callers (work captured into a CUDA graph with allocation disallowed, a plugin whose host
application owns every device allocation, a path that must not let cudaMalloc/cudaFree
synchronise the device) get the level's generators and Cross vectors into device memory
themselves and call tpc_apply_noalloc, whose work memory is a static device array. This file
checks its result against tpc_apply of a handle built by tpc_setup and against the oracle's
matrix of the same level, on calls in a row, with the product tolerance of the other GPU tests
(1e-12 normwise against ||A||_1 ||x||). The sizes reach both ends of what the static array
accepts: N = 1 (the smallest level) and N = 32767 (m = 65536, every part of the array at its
limit). It runs last so that a failure here does not hide the other tests' results; it passes
on its own in a fresh process as well as after them.
"""
import numpy as np
import pytest

import paper_2202_11288_gb300 as tpc
from oracle import amg, large, model
from synth import uniform_pm1

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _noalloc(lev, x):
    """tpc_apply_noalloc on a level in the tpc_export_level layout (generators copied to the
    device by the caller, as such a caller would)."""
    g = {k: _dev(lev[k]) for k in ("A", "B", "C", "D", "p", "q", "xi", "zeta")}
    y = torch.full_like(x, float("nan"))
    tpc.tpc_apply_noalloc(lev["N"], g["A"], g["B"], g["C"], g["D"], g["p"], g["q"], g["xi"],
                          g["zeta"], lev["o"], x, y)
    torch.cuda.synchronize()
    return y


def _check(y, ref, norm1, x):
    err = np.linalg.norm(y - ref)
    bound = 1e-12 * norm1 * np.linalg.norm(x)
    assert np.isfinite(err) and err <= bound, (err, bound)


@pytest.mark.parametrize("variant", [tpc.TPC_NONSYM, tpc.TPC_SPD])
def test_noalloc_product_matches_tpc_apply_and_oracle_twice(variant):
    K, delta = 13, 0.05
    N = 1 << K
    r = model.horizon_ratio(delta, 1.0 / N)
    H = amg.Hierarchy(large.rows(variant, N, r, np.arange(2 * N - 1)), kc=3)
    S = tpc.Solver(delta, 2.0 ** -K, variant=variant)
    try:
        # two calls in a row: the finest level (three-kernel pipeline) and a small level
        # (single-block pipeline), each against tpc_apply on the same operand and against the
        # oracle's dense matrix of that level
        for call, level in enumerate((K, 8)):
            lev = S.export_level(level)
            n = 2 * lev["N"] + 1
            xh = uniform_pm1(n, 40 + call)
            x = _dev(xh)
            y_ref = torch.empty_like(x)
            S.apply(level, x, y_ref)
            y = _noalloc(lev, x)
            A = H.A[level]
            norm1 = np.abs(A).sum(0).max()
            _check(y.cpu().numpy(), y_ref.cpu().numpy(), norm1, xh)
            _check(y.cpu().numpy(), A @ xh, norm1, xh)
    finally:
        S.close()


def test_noalloc_at_the_size_limit_and_the_smallest_level():
    """N = 32767 (the largest accepted: m = 2^16) against the oracle's FFT product of the
    printed finest blocks, then N = 1 (level 1 of a hierarchy taken down to k = 1) against the
    oracle's dense Galerkin matrix: calls in a row on the shared static array."""
    K, delta, variant = 15, 0.05, tpc.TPC_NONSYM
    N = 1 << K
    r = model.horizon_ratio(delta, 1.0 / N)
    S = tpc.Solver(delta, 2.0 ** -K, variant=variant)
    try:
        lev = S.export_level(K)
        assert lev["N"] == 32767
        n = 2 * lev["N"] + 1
        for seed in (50, 51):
            xh = uniform_pm1(n, seed)
            y = _noalloc(lev, _dev(xh)).cpu().numpy()
            bl = large.block_lists(variant, N, r)
            gsum = {k: np.abs(c).sum() + np.abs(rw[1:]).sum() for k, (c, rw) in bl.items()}
            norm1 = max(gsum["A"] + gsum["C"], gsum["B"] + gsum["D"])
            _check(y, large.matvec(variant, N, r, xh), norm1, xh)
    finally:
        S.close()
    Ks = 6
    H = amg.Hierarchy(model.assemble(variant, 1 << Ks, model.horizon_ratio(0.125, 2.0 ** -Ks)),
                      kc=1)
    S = tpc.Solver(0.125, 2.0 ** -Ks, variant=variant, coarsest_level=1)
    try:
        lev = S.export_level(1)
        assert lev["N"] == 1
        xh = uniform_pm1(3, 52)
        y = _noalloc(lev, _dev(xh)).cpu().numpy()
        A = H.A[1]
        _check(y, A @ xh, np.abs(A).sum(0).max(), xh)
    finally:
        S.close()


def test_noalloc_rejects_sizes_beyond_its_static_array():
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    y = torch.zeros(8, dtype=torch.float64, device="cuda")
    N = 1 << 15          # 2^15 - 1 is the largest accepted N; 2^16 - 1 is beyond
    for bad in (N * 2 - 1, 10):
        with pytest.raises(tpc.TpcError) as ei:
            tpc.tpc_apply_noalloc(bad, x, x, x, x, x, x, x, x, 1.0, x, y)
        assert ei.value.code == tpc.TPC_EINVAL
        assert "tpc_apply_noalloc" in tpc.tpc_last_error()
