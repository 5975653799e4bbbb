"""The bounded device-side wait of the split-precision kernels (an mbarrier
wait with an iteration limit): a barrier that nothing completes makes the wait
give up within its limit, the host sees BSM_ERR_TIMEOUT, and the context stays
usable (a multiply right after it is exact). No fault, no hang: the wait only
runs out."""
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_wait_completes(gpu_ctx):
    gpu_ctx.selftest_wait(False)


def test_wait_gives_up_and_context_survives(gpu_ctx, bsm_lib, oracle_mod):
    t0 = time.perf_counter()
    with pytest.raises(bsm_lib.BsmError) as e:
        gpu_ctx.selftest_wait(True)
    assert e.value.name == "TIMEOUT"
    assert time.perf_counter() - t0 < 30.0
    rng = np.random.default_rng(3)
    A = synth.random_blocks(rng, [3, 5, 2], [4, 1, 6], 0.8, kind="int")
    B = synth.random_blocks(rng, [4, 1, 6], [2, 7], 0.8, kind="int")
    ref = oracle_mod.multiply(A, B, eps=0.0)
    dA, dB = gpu_ctx.from_blocks(A), gpu_ctx.from_blocks(B)
    dC = gpu_ctx.empty(A.row_sizes, B.col_sizes)
    gpu_ctx.multiply(1.0, dA, dB, 0.0, dC, 0.0, precision=1)
    r, c = dC.pattern()
    assert np.array_equal(r, ref.blk_row) and np.array_equal(c, ref.blk_col)
    assert np.array_equal(dC.values(), ref.values)
    for m in (dA, dB, dC):
        m.destroy()
