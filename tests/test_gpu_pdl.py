"""Programmatic dependent launch (the solve's kernels wait for their predecessor with
griddepcontrol.wait): results are bitwise those of plain stream order. A child process with
TPC_PDL=0 (read once, at the first launch) solves the same problems; every solution and
iteration count must agree exactly."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import paper_2202_11288_gb300 as tpc
from synth import uniform_pm1

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import paper_2202_11288_gb300 as tpc
from synth import uniform_pm1
cases = json.loads(sys.argv[2])
out = []
for K, delta, prec, outer in cases:
    S = tpc.Solver(delta, 2.0 ** -K, precision=prec, outer=outer, autotune=0)
    b = torch.tensor(uniform_pm1(S.n, 1000 + K), device="cuda")
    x = torch.zeros_like(b)
    rc, it, rel = S.solve(b, x, tol=1e-10)
    out.append((it, x.cpu().numpy().tobytes().hex()))
    S.close()
print(json.dumps(out))
"""

CASES = [(12, 0.05, tpc.TPC_MIXED, tpc.TPC_OUTER_VCYCLE), (16, 0.1, tpc.TPC_FP64, tpc.TPC_OUTER_VCYCLE),
         (20, 0.05, tpc.TPC_MIXED, tpc.TPC_OUTER_VCYCLE), (18, 0.05, tpc.TPC_MIXED, tpc.TPC_OUTER_FGMRES)]


def _solve(env):
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, json.dumps(CASES)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_pdl_results_equal_plain_stream_order():
    env_on = dict(os.environ)
    env_on.pop("TPC_PDL", None)
    env_off = dict(os.environ, TPC_PDL="0")
    on, off = _solve(env_on), _solve(env_off)
    for case, a, b in zip(CASES, on, off):
        assert a[0] == b[0], (case, a[0], b[0])
        assert a[1] == b[1], case
