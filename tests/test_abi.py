"""The C-ABI library loads without a GPU and exports every symbol its header declares."""
import ctypes
import os
import re

import pytest

import paper_2202_11288_gb300 as tpc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "tpcamg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tpc(?:2d)?_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_binding_names():
    assert sorted(tpc.EXPORTED) == _declared()


def test_library_exports_every_declared_symbol():
    L = ctypes.CDLL(tpc.LIB_PATH)
    for name in _declared():
        assert hasattr(L, name), name


def test_device_calls_fail_cleanly_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(tpc.TpcError) as ei:
        tpc.tpc_setup(0.125, 2.0 ** -7, stream=0)
    assert ei.value.code == tpc.TPC_ECUDA
    assert tpc.lib().tpc_level_size(None, 7) == 0
    tpc.lib().tpc_destroy(None)


def test_server_and_batch_fail_cleanly_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(tpc.TpcError) as ei:
        tpc.Server(hbm_budget_bytes=1 << 20)
    assert ei.value.code == tpc.TPC_ECUDA
    rc, its, rels, sts = tpc.tpc_solve_batch([], [], [])  # an empty batch needs no device
    assert rc == tpc.TPC_OK and its == [] and sts == []
    tpc.lib().tpc_server_destroy(None)
