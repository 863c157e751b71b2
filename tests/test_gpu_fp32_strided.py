"""FP32 products on the levels that take the multi-kernel (strided) pipeline, element by element
against the FP64 oracle.

In FP32 a level's product is one launch only while m = 2N + 2 <= 4096; larger levels run the
forward strided pass, the contiguous-block kernel (instances with log2 L = 10, 11, 12 fixed at
compile time and the general one) and the inverse strided pass; levels with m <= 2^18 use the
instances compiled for three resident blocks per SM. These tests reach every one of them:

* every level of K = 12, 13, 14 (m = 2^13 .. 2^15 on top, single-block below), both systems,
  against the oracle's dense Galerkin matrices R A P (eq. (3.2), eq. (3.6));
* the finest level of K = 18 .. 22 (m = 2^19 .. 2^23: log2 L = 10, 10, 11, 11, 12), both
  systems, against the oracle's FFT-convolution product of the printed Toeplitz blocks
  (section 2.2, eq. (2.9) / eq. (2.10)).

Tolerance: one forward and one inverse FFT of length m in FP32, plus the rounding of x and of
the spectra, carry an absolute error of order eps32 log2(m) ||A|| ||x|| (eps32 = 6e-8); the
bound is ||y - y_ref|| <= 2e-6 log2(m) ||A||_1 ||x||, the bound of the other FP32 tests.
"""
import numpy as np
import pytest

import paper_2202_11288_gb300 as tpc
from oracle import amg, large, model
from oracle.model import NONSYM, SPD
from synth import uniform_pm1

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _f32(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float32, device="cuda")


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64)


def _operands(n, seed):
    """A seeded uniform[-1,1) operand and a smooth one (its product is far below ||A|| ||x||)."""
    return [uniform_pm1(n, seed), np.sin(np.pi * np.arange(1, n + 1) / (n + 1))]


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("K", [12, 13, 14])
def test_fp32_products_every_level_strided(variant, K):
    delta = 0.05
    N = 1 << K
    r = model.horizon_ratio(delta, 1.0 / N)
    A_fine = large.rows(variant, N, r, np.arange(2 * N - 1))   # the printed blocks, densely
    H = amg.Hierarchy(A_fine, kc=3)
    del A_fine
    S = tpc.Solver(delta, 2.0 ** -K, variant=variant, precision=tpc.TPC_MIXED)
    try:
        for k in range(K, H.kc, -1):
            A = H.A[k]
            n = A.shape[0]
            norm1 = np.abs(A).sum(0).max()
            for j, x in enumerate(_operands(n, 500 + k)):
                xr = x.astype(np.float32).astype(np.float64)   # the operand the GPU sees
                yd = torch.empty(n, dtype=torch.float32, device="cuda")
                S.apply_f32(k, _f32(xr), yd)
                y = _host(yd)
                ref = A @ xr
                bound = 2e-6 * (k + 1) * norm1 * np.linalg.norm(xr)
                err = np.linalg.norm(y - ref)
                assert np.isfinite(err) and err <= bound, (k, j, err / bound)
    finally:
        S.close()


def _norm1_bound(variant, N, r):
    """||A||_1 of the finest matrix, from its Toeplitz blocks: the largest column sum of
    [A; C] and [B; D] taken over full generators (exact once N > 2r)."""
    bl = large.block_lists(variant, N, r)

    def gen_sum(name):
        col, row = bl[name]
        return np.abs(col).sum() + np.abs(row[1:]).sum()

    return max(gen_sum("A") + gen_sum("C"), gen_sum("B") + gen_sum("D"))


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("K", [18, 19, 20, 21, 22])
def test_fp32_finest_product_large(variant, K):
    delta = 0.05
    N = 1 << K
    r = model.horizon_ratio(delta, 1.0 / N)
    S = tpc.Solver(delta, 2.0 ** -K, variant=variant, precision=tpc.TPC_MIXED)
    try:
        n = S.n
        norm1 = _norm1_bound(variant, N, r)
        for j, x in enumerate(_operands(n, 700 + K)):
            xr = x.astype(np.float32).astype(np.float64)
            yd = torch.empty(n, dtype=torch.float32, device="cuda")
            S.apply_f32(K, _f32(xr), yd)
            y = _host(yd)
            ref = large.matvec(variant, N, r, xr)
            bound = 2e-6 * (K + 1) * norm1 * np.linalg.norm(xr)
            err = np.linalg.norm(y - ref)
            assert np.isfinite(err) and err <= bound, (K, j, err / bound)
    finally:
        S.close()
