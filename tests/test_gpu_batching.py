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


def _formula_shape(te, slots=12, maxg=8):
    """The packed kernel's built-in slot shape (nT, G) for a tile of te
    elements: the most useful lanes te*G/(32 nT), the fewest passes among equals."""
    bt, bg = (te + 31) // 32, 1
    for t in range(1, slots + 1):
        g = min((32 * t) // te, maxg)
        if g >= 1 and g * bt > bg * t:
            bt, bg = t, g
    return bt, bg


@pytest.mark.parametrize("slots", [12, 16])
def test_forced_slot_shapes_parity(bsm_lib, oracle_mod, amorph, tmp_path, monkeypatch, slots):
    """Every tile shape of a packed kernel (12 or 16 slots per lane) set,
    through the cache file, to a shape the formula would not pick (another
    number of k-groups): the persistent launch reads the table on the device,
    so the values change in their last bits and still match the oracle."""
    lines = []
    for tm in range(1, 17):
        for tn in range(1, 17):
            te = tm * tn
            nt, g = _formula_shape(te, slots)
            g2 = g - 1 if g > 1 else 2
            nt2 = (te * g2 + 31) // 32
            if nt2 > slots:
                g2, nt2 = 1, (te + 31) // 32
            assert te * g2 <= 32 * nt2 <= 32 * slots
            lines.append(f"pk{slots}tile:{tm}x{tn} {nt2 << 8 | g2} 0.0")
    cache = tmp_path / "forced.txt"
    cache.write_text("\n".join(lines) + "\n# a note line is ignored\n")
    kw = dict(launch=0, fp64_kernel=bsm_lib.BSM_FP64_PK12 if slots == 12 else bsm_lib.BSM_FP64_PK16)
    with bsm_lib.Context(0) as ctx:
        v_formula = _check(ctx, oracle_mod, amorph, **kw)
    monkeypatch.setenv("BSM_AUTOTUNE_CACHE", str(cache))
    with bsm_lib.Context(0) as ctx:
        v_forced = _check(ctx, oracle_mod, amorph, **kw)
    assert not np.array_equal(v_forced, v_formula)


def test_slot_shape_tuning(bsm_lib, oracle_mod, tmp_path, monkeypatch):
    """The persistent launch with the autotuner times every candidate slot
    shape of each one-tile class with enough C blocks (water: 5x5, 5x13, 13x5,
    13x13), keeps the fastest in the table (cache entries and notes with the
    formula's time beside the tuned one), and its result matches the oracle;
    a new context reads the entries back and tunes nothing more."""
    cache = tmp_path / "tune.txt"
    # the whole-launch choice fixed to the 12-slot packed kernel, so that only
    # the slot shapes are tuned
    cache.write_text(f"fp64/all/5,13,|5,13,|5,13, {bsm_lib.BSM_FP64_PK12} 0.0\n")
    monkeypatch.setenv("BSM_AUTOTUNE_CACHE", str(cache))
    A = synth.water(64, seed=3)
    ref = oracle_mod.multiply(A, A, eps=1e-10)
    for _ in range(2):
        with bsm_lib.Context(0) as ctx:
            dA = ctx.from_blocks(A)
            dC = ctx.empty(A.row_sizes, A.col_sizes)
            ctx.multiply(1.0, dA, dA, 0.0, dC, 1e-10, launch=0, autotune=True)
            r, c = dC.pattern()
            v = dC.values()
            dA.destroy()
            dC.destroy()
        assert np.array_equal(r, ref.blk_row) and np.array_equal(c, ref.blk_col)
        assert H.rel_frobenius(v, ref.values) <= TOL
        text = cache.read_text()
        tiles = {ln.split()[0]: int(ln.split()[1]) for ln in text.splitlines()
                 if ln.startswith("pk12tile:")}
        notes = [ln for ln in text.splitlines() if ln.startswith("# pk12tile:")]
        assert set(tiles) == {"pk12tile:5x5", "pk12tile:5x13", "pk12tile:13x5", "pk12tile:13x13"}
        assert len(notes) == 4
        for key, val in tiles.items():
            m, n = map(int, key.split(":")[1].split("x"))
            assert 1 <= val >> 8 <= 12 and 1 <= (val & 0xFF) <= 8
            assert m * n * (val & 0xFF) <= 32 * (val >> 8)
