"""Batched solves of uneven independent instances (tpc_solve_batch) against solving each alone.

Every instance runs the arithmetic of tpc_solve on its own handle, so the results must be
bitwise identical to the lone solves, with the same iteration counts, for any mix of sizes,
variants and precisions.
"""
import numpy as np
import pytest

import paper_2202_11288_gb300 as tpc
from oracle import amg, model
from synth import uniform_pm1

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SPECS = [  # (K, delta, variant, precision)
    (8, 0.125, tpc.TPC_SPD, tpc.TPC_FP64),
    (10, 0.05, tpc.TPC_NONSYM, tpc.TPC_FP64),
    (12, 0.2, tpc.TPC_SPD, tpc.TPC_MIXED),
    (9, 0.3, tpc.TPC_NONSYM, tpc.TPC_MIXED),
    (14, 0.05, tpc.TPC_SPD, tpc.TPC_MIXED),
    (11, 0.1, tpc.TPC_SPD, tpc.TPC_FP64),
    (4, 0.125, tpc.TPC_SPD, tpc.TPC_FP64),
]


def test_batch_equals_alone_bitwise():
    solvers = [tpc.Solver(d, 2.0 ** -K, variant=v, precision=p) for K, d, v, p in SPECS]
    try:
        bs = [torch.tensor(uniform_pm1(S.n, 50 + i), device="cuda") for i, S in enumerate(solvers)]
        alone = []
        for S, b in zip(solvers, bs):
            x = torch.zeros_like(b)
            rc, it, rel = S.solve(b, x, tol=1e-10)
            assert rc == tpc.TPC_OK
            alone.append((x, it, rel))
        xs = [torch.full_like(b, 7.0) for b in bs]
        rc, its, rels, sts = tpc.tpc_solve_batch([S.handle for S in solvers], bs, xs, tol=1e-10)
        assert rc == tpc.TPC_OK and all(s == tpc.TPC_OK for s in sts)
        for (xa, ita, rela), xb, itb, relb in zip(alone, xs, its, rels):
            assert itb == ita and relb == rela
            assert torch.equal(xa, xb)
        # and the FP64 ones are right: compare the smallest with the oracle's iterate
        K, d, v, p = SPECS[0]
        N = 1 << K
        H = amg.Hierarchy(model.assemble(v, N, model.horizon_ratio(d, 1.0 / N)), kc=3)
        _, it_ref, _, iterates = amg.solve(H, bs[0].cpu().numpy(), tol=1e-10)
        ref = iterates[it_ref - 1]
        assert np.linalg.norm(xs[0].cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref)
    finally:
        for S in solvers:
            S.close()


def test_batch_edge_cases():
    S = tpc.Solver(0.125, 2.0 ** -7)
    try:
        rc, its, rels, sts = tpc.tpc_solve_batch([], [], [])
        assert rc == tpc.TPC_OK and its == []
        b = torch.tensor(uniform_pm1(S.n, 1), device="cuda")
        x1, x2 = torch.zeros_like(b), torch.zeros_like(b)
        with pytest.raises(tpc.TpcError):
            tpc.tpc_solve_batch([S.handle, S.handle], [b, b], [x1, x2])
    finally:
        S.close()
