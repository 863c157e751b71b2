"""The process-wide FFT plan table (tpc_tune_get / tpc_tune_set / tpc_tune_reset): host logic,
no GPU. The GPU side (every candidate plan against the oracle) is tests/test_gpu_fft_plans.py."""
import pytest

import paper_2202_11288_gb300 as tpc


@pytest.fixture(autouse=True)
def empty_table():
    tpc.tpc_tune_reset()
    yield
    tpc.tpc_tune_reset()


def test_set_get_reset():
    assert tpc.tpc_tune_get(4, 18) is None
    tpc.tpc_tune_set(4, 18, 10, 1, 0)
    tpc.tpc_tune_set(8, 18, 9, 0, 0)
    assert tpc.tpc_tune_get(4, 18) == (10, 1, 0)
    assert tpc.tpc_tune_get(8, 18) == (9, 0, 0)      # per precision
    tpc.tpc_tune_set(4, 18, 9, 0, 0)                  # overwrite
    assert tpc.tpc_tune_get(4, 18) == (9, 0, 0)
    tpc.tpc_tune_reset()
    assert tpc.tpc_tune_get(4, 18) is None and tpc.tpc_tune_get(8, 18) is None


def test_register_resident_entries_take_four_columns():
    for logm, logL in ((20, 10), (21, 10), (21, 11), (22, 11), (22, 12), (23, 12)):
        tpc.tpc_tune_set(4, logm, logL, 0, 1)
        assert tpc.tpc_tune_get(4, logm) == (logL, 2, 1)


@pytest.mark.parametrize("args", [
    (4, 12, 6, 0, 0),     # below the three-pass sizes
    (4, 24, 12, 0, 0),    # above
    (4, 17, 6, 0, 0),     # L < 2^7
    (4, 17, 12, 0, 0),    # R1 < 2^6
    (4, 23, 11, 0, 0),    # R1 > 2^11
    (4, 19, 9, 4, 0),     # R1 x 2^logC > 8192
    (4, 17, 9, -1, 0),    # width out of range
    (4, 19, 10, 0, 1),    # register-resident kernels start at m = 2^20
    (4, 22, 13, 0, 1),    # L > 2^12
    (8, 22, 11, 0, 1),    # FP64 has no register-resident kernels
    (4, 18, 9, 0, 2),     # reg is 0 or 1
    (3, 18, 9, 0, 0),     # word is 4 or 8
])
def test_out_of_range_entries_are_refused(args):
    with pytest.raises(tpc.TpcError):
        tpc.tpc_tune_set(*args)
    assert tpc.tpc_tune_get(4, args[1]) is None if args[0] == 4 else True


def test_get_refuses_a_bad_word():
    with pytest.raises(tpc.TpcError):
        tpc.tpc_tune_get(2, 18)
