"""tpc_apply_noalloc: the one-level product for callers that cannot allocate device memory.

Such callers (work captured into a CUDA graph with allocation disallowed, a plugin whose host
application owns every device allocation, a path that must not let cudaMalloc/cudaFree
synchronise the device) get the level's generators and Cross vectors into device memory
themselves and call tpc_apply_noalloc, whose work memory is a static device array. This file
checks its result against tpc_apply of a handle built by tpc_setup, on two calls in a row, with
the product tolerance of the other GPU tests (1e-12 normwise against ||A||_1 ||x||). It runs
last so that a failure here does not hide the other tests' results; it passes on its own in a
fresh process as well as after them.
"""
import numpy as np
import pytest

import paper_2202_11288_gb300 as tpc
from synth import uniform_pm1

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _norm1(lev):
    # a bound on ||A_k||_1 from the generators and the Cross
    return (np.abs(lev["A"]).sum() + np.abs(lev["B"]).sum() + np.abs(lev["C"]).sum()
            + np.abs(lev["D"]).sum() + np.abs(lev["p"]).sum() + np.abs(lev["q"]).sum()
            + np.abs(lev["xi"]).sum() + np.abs(lev["zeta"]).sum() + abs(lev["o"]))


@pytest.mark.parametrize("variant", [tpc.TPC_NONSYM, tpc.TPC_SPD])
def test_noalloc_product_matches_tpc_apply_twice(variant):
    K, delta = 13, 0.05
    S = tpc.Solver(delta, 2.0 ** -K, variant=variant)
    try:
        # two calls in a row: the finest level (three-kernel pipeline) and a small level
        # (single-block pipeline), each against tpc_apply on the same operand
        for call, level in enumerate((K, 8)):
            lev = S.export_level(level)
            N = lev["N"]
            n = 2 * N + 1
            x = _dev(uniform_pm1(n, 40 + call))
            y_ref = torch.empty_like(x)
            S.apply(level, x, y_ref)
            y = torch.full_like(x, float("nan"))
            g = {k: _dev(lev[k]) for k in ("A", "B", "C", "D", "p", "q", "xi", "zeta")}
            tpc.tpc_apply_noalloc(N, g["A"], g["B"], g["C"], g["D"], g["p"], g["q"], g["xi"],
                                  g["zeta"], lev["o"], x, y)
            torch.cuda.synchronize()
            err = torch.linalg.norm(y - y_ref).item()
            bound = 1e-12 * _norm1(lev) * torch.linalg.norm(x).item()
            assert np.isfinite(err) and err <= bound, (call, level, err, bound)
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
