"""Launch modes on the GPU: one persistent launch over all shape classes vs one
launch per (m, n) class ("stack"), CUDA-graph replay, and the autotuner. Every
mode must give the oracle's pattern bit for bit and its values to 1e-12."""
import os

import numpy as np
import pytest

import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def amorph():
    return synth.amorphous(160, seed=5, density=0.05, cutoff=7.0)


def _check(ctx, oracle_mod, A, reps=1, **kw):
    ref = oracle_mod.multiply(A, A, eps=1e-8)
    dA = ctx.from_blocks(A)
    dC = ctx.empty(A.row_sizes, A.col_sizes)
    for _ in range(reps):
        ctx.multiply(1.0, dA, dA, 0.0, dC, 1e-8, **kw)
    r, c = dC.pattern()
    v = dC.values()
    dA.destroy()
    dC.destroy()
    assert np.array_equal(r, ref.blk_row) and np.array_equal(c, ref.blk_col)
    assert H.rel_frobenius(v, ref.values) <= TOL
    return v


@pytest.mark.parametrize("launch", [0, 1])
@pytest.mark.parametrize("graph", [False, True])
def test_modes_fp64(gpu_ctx, oracle_mod, amorph, launch, graph):
    _check(gpu_ctx, oracle_mod, amorph, reps=3, launch=launch, graph=graph)


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("launch", [0, 1])
def test_modes_split_pattern(gpu_ctx, oracle_mod, amorph, prec, launch):
    ref = oracle_mod.multiply(amorph, amorph, eps=1e-8)
    dA = gpu_ctx.from_blocks(amorph)
    dC = gpu_ctx.empty(amorph.row_sizes, amorph.col_sizes)
    for _ in range(2):
        gpu_ctx.multiply(1.0, dA, dA, 0.0, dC, 1e-8, precision=prec, launch=launch, graph=True)
    r, c = dC.pattern()
    assert np.array_equal(r, ref.blk_row) and np.array_equal(c, ref.blk_col)
    assert H.rel_frobenius(dC.values(), ref.values) <= 2e-5
    dA.destroy()
    dC.destroy()


def test_autotune_and_cache(bsm_lib, oracle_mod, amorph, tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("BSM_AUTOTUNE_CACHE", str(cache))
    ctx = bsm_lib.Context(0)
    try:
        for launch in (1, 0):
            _check(ctx, oracle_mod, amorph, reps=2, launch=launch, autotune=True)
            _check(ctx, oracle_mod, amorph, reps=2, launch=launch, autotune=True, graph=True)
    finally:
        ctx.close()
    lines = [ln.split() for ln in cache.read_text().splitlines()]
    keys = {ln[0] for ln in lines}
    assert any(k.startswith("fp64/class/") for k in keys)
    assert any(k.startswith("fp64/all/") for k in keys)
    # a new context reads the table back and tunes nothing more
    n_before = len(lines)
    ctx = bsm_lib.Context(0)
    try:
        _check(ctx, oracle_mod, amorph, launch=1, autotune=True)
    finally:
        ctx.close()
    assert len(cache.read_text().splitlines()) == n_before


def test_graph_replay_counts_launches(gpu_ctx, oracle_mod):
    A = synth.water(16, seed=2)
    dA = gpu_ctx.from_blocks(A)
    dC = gpu_ctx.empty(A.row_sizes, A.col_sizes)
    gpu_ctx.multiply(1.0, dA, dA, 0.0, dC, 1e-10, blocking=True)
    gpu_ctx.multiply(1.0, dA, dA, 0.0, dC, 1e-10, blocking=True)
    gpu_ctx.profile(True)
    for _ in range(4):
        gpu_ctx.multiply(1.0, dA, dA, 0.0, dC, 1e-10, graph=True)
    p = gpu_ctx.profile_read()
    gpu_ctx.profile(False)
    assert p.launches == 4 * 5  # norms, count, scan, fill, numeric per multiply
    ref = oracle_mod.multiply(A, A, eps=1e-10)
    assert H.rel_frobenius(dC.values(), ref.values) <= TOL
    dA.destroy()
    dC.destroy()
