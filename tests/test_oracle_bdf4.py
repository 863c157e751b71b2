"""The oracle's time stepping (eq. (5.1), section 5) against the errors the paper prints in
Tables 2 and 3 (tests/golden/bdf4_tables.txt). These pin, together, the printed coefficients
of both systems, the exterior couplings moved to the right-hand side, the kernel constant
gamma = 3 / delta^3 with delta = r h, and the BDF4 recurrence: all sixteen printed errors are
reproduced to within one unit of their last printed digit."""
import math
import os

import numpy as np
import pytest

from oracle import model, timestep
from oracle.model import NONSYM, SPD

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "bdf4_tables.txt")


def table_rows():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                v, N, d, e = line.split()
                N = int(N)
                r = N // 4 if d == "1/4" else int(math.floor(math.sqrt(N)))
                rows.append((SPD if v == "spd" else NONSYM, N, r, d, float(e)))
    return rows


def last_digit_unit(e):
    return 10.0 ** (math.floor(math.log10(e)) - 4)


@pytest.mark.parametrize("variant,N,r,d,printed", table_rows())
def test_bdf4_error_matches_tables_2_and_3(variant, N, r, d, printed):
    err, _ = timestep.bdf4(variant, N, r)
    assert abs(err - printed) <= last_digit_unit(printed), (err, printed)


def test_bdf4_fourth_order_in_tau_and_h():
    """delta = 1/4 fixed: the error falls by about 2^4 per refinement (section 5)."""
    errs = [timestep.bdf4(SPD, N, N // 4)[0] for N in (16, 32, 64)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(3.8 < q < 4.2 for q in rates), rates


def test_planted_mistakes_miss_the_table():
    """The pin is sensitive: a wrong BDF4 history weight, the exterior couplings dropped, or the
    nominal delta in gamma for delta = sqrt(h) each move the N = 32 error far off the table."""
    N, r, printed = 32, 8, 1.1628e-05
    h = 1.0 / N
    tau = h
    eta = timestep.eta_h(N, r)
    A = model.assemble(SPD, N, r)
    M = A + 25.0 * eta / (12.0 * tau) * np.eye(A.shape[0])
    x = model.collocation_points(N)
    G_full = timestep.source_vector(SPD, N, r)
    G_noext = G_full - model.exterior_rhs(SPD, N, r, *[timestep.phi(p) for p in
                                                        model.exterior_points(N, r)])

    def run(G, w3):
        U = [np.exp(j * tau) * timestep.phi(x) for j in range(4)]
        for k in range(4, N + 1):
            hist = 4.0 * U[-1] - 3.0 * U[-2] + w3 * U[-3] - 0.25 * U[-4]
            U.append(np.linalg.solve(M, (eta / tau) * hist + np.exp(k * tau) * G))
            U.pop(0)
        return float(np.max(np.abs(U[-1] - np.exp(1.0) * timestep.phi(x))))

    assert abs(run(G_full, 4.0 / 3.0) - printed) <= last_digit_unit(printed)
    assert abs(run(G_full, 1.0) - printed) > 100 * last_digit_unit(printed)
    assert abs(run(G_noext, 4.0 / 3.0) - printed) > 100 * last_digit_unit(printed)
    # gamma from the nominal delta = sqrt(h) instead of r h (N = 32: r = 5, delta_eff = 5/32)
    err_nominal, _ = timestep.bdf4(SPD, 32, 5, gamma=3.0 / math.sqrt(1.0 / 32) ** 3)
    assert abs(err_nominal - 2.5257e-05) > 100 * last_digit_unit(2.5257e-05)


def test_exterior_rhs_is_the_manufactured_boundary_part():
    """model.exterior_rhs with g = u reproduces the exterior part of model.manufactured."""
    for variant in (SPD, NONSYM):
        N, r = 16, 3
        b, _ = model.manufactured(variant, N, r)
        x = model.collocation_points(N)
        h, delta = 1.0 / N, r / N
        u = lambda y: y * y * (1.0 - y) ** 2          # noqa: E731
        U = lambda y: y ** 3 / 3 - y ** 4 / 2 + y ** 5 / 5  # noqa: E731
        interior = (6.0 / h) * (2.0 * delta * u(x) - (U(x + delta) - U(x - delta)))
        ext = model.exterior_rhs(variant, N, r, *[u(p) for p in model.exterior_points(N, r)])
        assert np.allclose(interior + ext, b, rtol=0, atol=1e-9 * np.abs(b).max())
