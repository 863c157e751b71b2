"""Stage-batched solves (tpc_batch_*): one launch per V-cycle stage over all instances of a group.

Each instance must compute exactly what its lone tpc_solve computes (bitwise equal iterates),
converged instances and instances with fewer inner cycles are masked per stage, handles that
cannot be grouped are solved beside the groups, and a device-side grid barrier whose wait cannot
be satisfied gives up and reports instead of hanging.
"""
import numpy as np
import pytest

import paper_2202_11288_gb300 as tpc
from synth import uniform_pm1

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _specs():
    # (K, delta, variant, kernel, a): several members per group (same K and system), levels
    # whose products are single-block (K <= 11) and three-pass (K >= 12), both systems, different
    # horizons within a group; a fractional-kernel instance that cannot be grouped (its
    # generators are not piecewise constant, so its residual is the FFT product)
    return [(10, 0.05, 0, 0, 0.0), (10, 0.2, 0, 0, 0.0), (10, 0.11, 0, 0, 0.0),
            (13, 0.05, 1, 0, 0.0), (13, 0.21, 1, 0, 0.0),
            (14, 0.07, 0, 0, 0.0), (14, 0.15, 0, 0, 0.0), (14, 0.03, 0, 0, 0.0),
            (12, 0.1, 0, 1, 0.25)]


def _solvers(specs):
    return [tpc.Solver(d, 2.0 ** -K, variant=v, kernel=k, kernel_a=a, precision=tpc.TPC_MIXED,
                       transfer=(tpc.TPC_TRANSFER_GEOMETRIC if k else tpc.TPC_TRANSFER_PAPER))
            for K, d, v, k, a in specs]


MODES = [tpc.TPC_BATCH_AUTO, tpc.TPC_BATCH_COOPERATIVE, tpc.TPC_BATCH_THREE_PASS]


@pytest.mark.parametrize("mode", MODES)
def test_stage_batched_equals_lone_solves_bitwise(mode):
    specs = _specs()
    solvers = _solvers(specs)
    try:
        bs = [torch.tensor(uniform_pm1(S.n, 800 + i), device="cuda") for i, S in enumerate(solvers)]
        lone = []
        for S, b in zip(solvers, bs):
            x = torch.zeros_like(b)
            rc, it, rel = S.solve(b, x, tol=1e-10)
            assert rc == tpc.TPC_OK and rel < 1e-10
            lone.append((it, x.clone()))
        B = tpc.Batch([S.handle for S in solvers])
        try:
            B.set_product_mode(mode)
            assert B.groups() == 3 and B.grouped_instances() == 8
            for rep in range(2):                      # twice: graphs are reused
                xs = [torch.full_like(b, float("nan")) for b in bs]
                rc, its, rels, sts = B.solve(bs, xs, tol=1e-10)
                assert rc == tpc.TPC_OK, (rc, sts)
                for i, (it, x) in enumerate(lone):
                    assert its[i] == it, (i, its[i], it)
                    assert rels[i] < 1e-10
                    assert torch.equal(xs[i], x), (rep, i)
        finally:
            B.close()
    finally:
        for S in solvers:
            S.close()


@pytest.mark.parametrize("mode", [tpc.TPC_BATCH_COOPERATIVE, tpc.TPC_BATCH_THREE_PASS])
def test_stage_batched_masks_converged_instances(mode):
    """Instances that converge in different numbers of outer iterations (a right-hand side that
    is already solved needs none) keep their own results while the group goes on."""
    solvers = _solvers([(12, 0.05, 0, 0, 0.0), (12, 0.09, 0, 0, 0.0)])
    try:
        b0 = torch.tensor(uniform_pm1(solvers[0].n, 3), device="cuda")
        b1 = torch.zeros(solvers[1].n, dtype=torch.float64, device="cuda")   # x = 0 at once
        B = tpc.Batch([S.handle for S in solvers])
        try:
            B.set_product_mode(mode)
            assert B.groups() == 1
            xs = [torch.full_like(b0, 7.0), torch.full_like(b1, 7.0)]
            rc, its, rels, sts = B.solve([b0, b1], xs, tol=1e-10)
            assert rc == tpc.TPC_OK and its[1] == 0 and its[0] >= 1
            assert torch.count_nonzero(xs[1]).item() == 0
            x_ref = torch.zeros_like(b0)
            rc, it, rel = solvers[0].solve(b0, x_ref, tol=1e-10)
            assert it == its[0] and torch.equal(xs[0], x_ref)
        finally:
            B.close()
    finally:
        for S in solvers:
            S.close()


def test_product_mode_switch_keeps_results():
    """Switching the product mode between solves drops the captured graphs; results stay bitwise."""
    solvers = _solvers([(13, 0.05, 0, 0, 0.0), (13, 0.12, 0, 0, 0.0)])
    try:
        bs = [torch.tensor(uniform_pm1(S.n, 40 + i), device="cuda") for i, S in enumerate(solvers)]
        B = tpc.Batch([S.handle for S in solvers])
        try:
            out = []
            for mode in (tpc.TPC_BATCH_THREE_PASS, tpc.TPC_BATCH_COOPERATIVE, tpc.TPC_BATCH_AUTO):
                B.set_product_mode(mode)
                xs = [torch.zeros_like(b) for b in bs]
                rc, its, rels, sts = B.solve(bs, xs, tol=1e-10)
                assert rc == tpc.TPC_OK
                out.append(xs)
            for xs in out[1:]:
                assert all(torch.equal(a, b) for a, b in zip(out[0], xs))
            with pytest.raises(tpc.TpcError):
                B.set_product_mode(7)
        finally:
            B.close()
    finally:
        for S in solvers:
            S.close()


def test_grid_wait_gives_up_and_reports():
    """A barrier no block can reach: every wait stops after its poll limit, the flag is raised,
    no block passes, and the context stays usable."""
    gave_up, passed = tpc.tpc_grid_wait_selftest(2000)
    assert gave_up == 1 and passed == 0
    x = torch.ones(1000, dtype=torch.float64, device="cuda")
    assert float((x * 2).sum()) == 2000.0


def test_batch_with_2d_instances_equals_lone_solves():
    """2-D instances beside the groups and the lone 1-D instances: every result is bitwise the
    lone tpc2d_solve / tpc_solve result."""
    specs = [(12, 0.05, 0, 0, 0.0), (12, 0.2, 0, 0, 0.0), (11, 0.1, 0, 1, 0.3)]
    solvers = _solvers(specs)
    twod = [tpc.Solver2D(d, 2.0 ** -K, variant=v, precision=tpc.TPC_MIXED)
            for K, d, v in [(6, 0.1, tpc.TPC_SPD), (5, 0.2, tpc.TPC_NONSYM), (7, 0.15, tpc.TPC_SPD)]]
    try:
        bs = [torch.tensor(uniform_pm1(S.n, 60 + i), device="cuda") for i, S in enumerate(solvers)]
        bs += [torch.tensor(uniform_pm1(S.nn, 70 + i), device="cuda") for i, S in enumerate(twod)]
        lone = []
        for S, b in zip(solvers + twod, bs):
            x = torch.zeros_like(b)
            rc, it, rel = S.solve(b, x, tol=1e-10)
            assert rc == tpc.TPC_OK and rel < 1e-10
            lone.append((it, rel, x))
        B = tpc.Batch([S.handle for S in solvers], [S.handle for S in twod])
        try:
            assert B.groups() == 1 and B.grouped_instances() == 2
            xs = [torch.full_like(b, float("nan")) for b in bs]
            rc, its, rels, sts = B.solve(bs, xs, tol=1e-10)
            assert rc == tpc.TPC_OK, (rc, sts)
            for i, (it, rel, x) in enumerate(lone):
                assert its[i] == it and rels[i] == rel, (i, its[i], it)
                assert torch.equal(xs[i], x), i
        finally:
            B.close()
    finally:
        for S in solvers + twod:
            S.close()
