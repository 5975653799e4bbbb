"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (persistent launch, default kernel): the GPU computes the whole C; the
oracle computes sampled ranges of C block rows (start, middle, end), which must
match bit for bit in pattern and within 1e-12 relative in values (FP64), or
within the stated per-element bound (split precisions). The same with the
filter active, and for the mixed-size system in both launch modes."""
import numpy as np
import pytest

import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu
ROWS = 96


def row_ranges(nbr):
    return [(0, ROWS), (nbr // 2 - ROWS // 2, nbr // 2 + ROWS // 2), (nbr - ROWS, nbr)]


def gpu_rows(r, v, lens, a, b):
    """The blocks of C block rows [a, b) from the full GPU result, and their values."""
    lo, hi = np.searchsorted(r, a), np.searchsorted(r, b)
    off = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    return lo, hi, v[off[lo]:off[hi]]


def check_sampled(ctx, oracle_mod, A, eps, tol=1e-12, split=None, **kw):
    """split: (precision name, kernel name, stated relative Frobenius bound):
    every sampled element within the kernel's per-element bound instead of
    the FP64 tolerance."""
    dA = ctx.from_blocks(A)
    dC = ctx.empty(A.row_sizes, A.col_sizes)
    st = ctx.multiply(1.0, dA, dA, 0.0, dC, eps, stats=True, **kw)
    r, c = dC.pattern()
    v = dC.values()
    lens = A.row_sizes.astype(np.int64)[r] * A.col_sizes.astype(np.int64)[c]
    absA = synth.BlockMatrix(A.row_sizes, A.col_sizes, A.blk_row, A.blk_col, np.abs(A.values))
    for a, b in row_ranges(A.nbr):
        ref = oracle_mod.multiply(A, A, eps=eps, rows=(a, b), nthreads=oracle_mod.max_threads())
        lo, hi, vg = gpu_rows(r, v, lens, a, b)
        assert np.array_equal(r[lo:hi], ref.blk_row) and np.array_equal(c[lo:hi], ref.blk_col)
        if split is None:
            assert H.rel_frobenius(vg, ref.values) <= tol
        else:
            prec, kernel, rel_f = split
            absref = oracle_mod.multiply(absA, absA, eps=eps, rows=(a, b),
                                         nthreads=oracle_mod.max_threads())
            bound = H.split_elem_bound(A, A, prec, kernel, ref.blk_row, ref.blk_col, absref.values,
                                       rows=(a, b))
            assert np.all(np.abs(vg - ref.values) <= bound)
            assert H.rel_frobenius(vg, ref.values) <= rel_f
    dA.destroy()
    dC.destroy()
    return st


@pytest.fixture(scope="module")
def water2048():
    return synth.water(2048, seed=1)


def test_water2048_default(gpu_ctx, oracle_mod, water2048):
    st = check_sampled(gpu_ctx, oracle_mod, water2048, 1e-10)
    assert st.c_blocks == 3391476 and st.kept == 55255630


def test_water2048_filter_active(gpu_ctx, oracle_mod, water2048):
    A = water2048
    nA = oracle_mod.norms(A)
    rng = np.random.default_rng(0)
    a = rng.integers(0, A.nblk, 200000)
    b = rng.integers(0, A.nblk, 200000)
    eps = float(np.percentile(nA[a] * nA[b], 30))
    st = check_sampled(gpu_ctx, oracle_mod, A, eps)
    assert 0 < st.dropped < st.candidates


@pytest.mark.parametrize("kernel,sk", [("blocks", 1), ("panel", 0), ("chunks", 2)])
@pytest.mark.parametrize("prec,name,bound",
                         [(1, "bf16x3", {"blocks": 2e-6, "panel": 1e-5, "chunks": 2e-6}),
                          (2, "tf32x2", {"blocks": 1e-5, "panel": 2e-5, "chunks": 1e-5})])
def test_water2048_split(gpu_ctx, oracle_mod, water2048, prec, name, bound, kernel, sk):
    check_sampled(gpu_ctx, oracle_mod, water2048, 1e-10, split=(name, kernel, bound[kernel]),
                  precision=prec, split_kernel=sk)


@pytest.mark.parametrize("launch", [0, 1])
def test_amorphous4096(gpu_ctx, oracle_mod, launch):
    A = synth.amorphous(4096, seed=2)
    check_sampled(gpu_ctx, oracle_mod, A, 1e-8, launch=launch)
