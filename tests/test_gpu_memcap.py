"""Simulated out-of-memory (failure injection on the host side): with
BSM_DEVICE_MEMORY_CAP set, the library's device allocations beyond the cap fail
as on a full device. A multiply that needs more memory reports NOMEM, and the
same context then runs a multiply that fits, with the oracle's result. Runs in
a child process: the cap is read once per process."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, numpy as np, synth, oracle
from paper_1705_10218_gb300 import Context, BsmError
out = {}
ctx = Context(0)
A = synth.water(64, seed=0)      # A 8 MB, C 17 MB: beyond the cap
try:
    dA = ctx.from_blocks(A)
    dC = ctx.empty(A.row_sizes, A.col_sizes)
    ctx.multiply(1.0, dA, dA, 0.0, dC, 1e-10, blocking=True)
    out["big"] = "OK"
except BsmError as e:
    out["big"] = e.name
rng = np.random.default_rng(4)
S = synth.random_blocks(rng, [3, 5, 2, 4] * 5, [3, 5, 2, 4] * 5, 0.3, kind="int")
dS = ctx.from_blocks(S)
dT = ctx.empty(S.row_sizes, S.col_sizes)
ctx.multiply(1.0, dS, dS, 0.0, dT, 0.0, blocking=True)
ref = oracle.multiply(S, S, eps=0.0)
r, c = dT.pattern()
out["small"] = bool(np.array_equal(r, ref.blk_row) and np.array_equal(c, ref.blk_col)
                    and np.array_equal(dT.values(), ref.values))
print(json.dumps(out))
"""


def test_device_memory_cap_gives_nomem(bsm_lib):
    env = dict(os.environ, BSM_DEVICE_MEMORY_CAP=str(12 << 20))
    p = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    out = json.loads(p.stdout.strip().splitlines()[-1])
    assert out["big"] == "NOMEM"
    assert out["small"] is True
