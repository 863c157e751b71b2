"""The large-size finest-level oracle agrees with the dense assembly it restates."""
import numpy as np
import pytest

from oracle import large, model
from oracle.model import NONSYM, SPD
from synth import uniform_pm1


@pytest.mark.parametrize("variant", [SPD, NONSYM])
@pytest.mark.parametrize("N,r", [(16, 3), (64, 8), (32, 40)])
def test_rows_and_fft_matvec_match_dense(variant, N, r):
    A = model.assemble(variant, N, r)
    idx = list(range(A.shape[0]))
    assert np.array_equal(large.rows(variant, N, r, idx), A)
    u = uniform_pm1(A.shape[0], 5)
    y = large.matvec(variant, N, r, u)
    assert np.linalg.norm(y - A @ u) <= 1e-13 * np.abs(A).sum(0).max() * np.linalg.norm(u)
