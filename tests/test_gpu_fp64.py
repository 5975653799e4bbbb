"""GPU parity of the FP64 path against the CPU oracle, through the C ABI.

The C pattern must match bit for bit (sorted (row, col) lists and the filter
counters); values must match within 1e-12 relative Frobenius error over the
whole of C (exactly, for small-integer inputs with eps = 0, where every sum is
an exact integer)."""
import math

import numpy as np
import pytest

import synth
from synth import BlockMatrix
from tests import helpers as H

pytestmark = pytest.mark.gpu
TOL = 1e-12


def run_gpu(ctx, A, B, alpha=1.0, beta=0.0, C=None, eps=0.0, **kw):
    dA = ctx.from_blocks(A)
    dB = dA if B is A else ctx.from_blocks(B)
    dC = ctx.from_blocks(C) if C is not None else ctx.empty(A.row_sizes, B.col_sizes)
    st = ctx.multiply(alpha, dA, dB, beta, dC, eps, stats=True, **kw)
    r, c = dC.pattern()
    v = dC.values()
    for m in {id(dA): dA, id(dB): dB, id(dC): dC}.values():
        m.destroy()
    return r, c, v, st


def check(ctx, oracle_mod, A, B, alpha=1.0, beta=0.0, C=None, eps=0.0, exact=False, **kw):
    ref = oracle_mod.multiply(A, B, alpha=alpha, beta=beta, C=C, eps=eps)
    r, c, v, st = run_gpu(ctx, A, B, alpha, beta, C, eps, **kw)
    assert np.array_equal(r, ref.blk_row), "pattern rows differ"
    assert np.array_equal(c, ref.blk_col), "pattern cols differ"
    assert st.candidates == ref.candidates and st.kept == ref.kept and st.dropped == ref.dropped
    assert st.c_blocks == len(ref.blk_row) and st.c_nnz == ref.nnz
    assert st.flops == ref.flops
    if exact:
        assert np.array_equal(v, ref.values)
    else:
        assert H.rel_frobenius(v, ref.values) <= TOL
    return ref, v, st


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (2.0, 1.0), (-1.0, -0.5)])
def test_integer_exact(gpu_ctx, oracle_mod, seed, alpha, beta):
    rng = np.random.default_rng(500 + seed)
    sizes = (1, 2, 3, 5, 13)
    rs, ks, cs = rng.choice(sizes, 9), rng.choice(sizes, 11), rng.choice(sizes, 10)
    A = synth.random_blocks(rng, rs, ks, 0.4, kind="int", shuffle=True)
    B = synth.random_blocks(rng, ks, cs, 0.4, kind="int", shuffle=True)
    C = synth.random_blocks(rng, rs, cs, 0.3, kind="int", shuffle=True)
    check(gpu_ctx, oracle_mod, A, B, alpha, beta, C, eps=0.0, exact=True)


def test_water64_config(gpu_ctx, oracle_mod):
    """64 water molecules, eps 1e-10 (the small water configuration)."""
    A = synth.water(64, seed=0)
    ref, v, st = check(gpu_ctx, oracle_mod, A, A, eps=1e-10)
    assert st.c_blocks == A.nbr * A.nbc  # C is fully dense at this size


def test_filter_active(gpu_ctx, oracle_mod):
    """eps at the 30th percentile of the candidate norm products: the same
    products must be dropped on both sides (bit-exact pattern and counters)."""
    A = synth.water(24, seed=7, cutoff=5.0)
    nA = oracle_mod.norms(A)
    prods = []
    for a in range(A.nblk):
        sel = A.blk_row == A.blk_col[a]
        prods.append(nA[a] * nA[sel])
    eps = float(np.percentile(np.concatenate(prods), 30))
    ref, _, st = check(gpu_ctx, oracle_mod, A, A, eps=eps)
    assert 0 < st.dropped < st.candidates


def test_filter_ties_and_nan(gpu_ctx, oracle_mod):
    def single(v):
        return BlockMatrix(np.array([1], np.int32), np.array([1], np.int32), np.array([0], np.int32),
                           np.array([0], np.int32), np.array([v], np.float64))
    A, B = single(2.0 ** -10), single(2.0 ** -20)
    _, _, v, st = run_gpu(gpu_ctx, A, B, eps=2.0 ** -30)
    assert st.kept == 1 and v[0] == 2.0 ** -30
    r, _, _, st = run_gpu(gpu_ctx, A, B, eps=math.nextafter(2.0 ** -30, math.inf))
    assert st.kept == 0 and len(r) == 0
    _, _, v, st = run_gpu(gpu_ctx, single(np.nan), B, eps=1e300)
    assert st.kept == 1 and np.isnan(v[0])


def test_large_and_odd_blocks(gpu_ctx, oracle_mod):
    """Block sizes above the 32 x 32 register tile and odd shapes."""
    rng = np.random.default_rng(12)
    sizes = (1, 7, 33, 40, 64, 65)
    rs, ks, cs = rng.choice(sizes, 5), rng.choice(sizes, 6), rng.choice(sizes, 4)
    A = synth.random_blocks(rng, rs, ks, 0.6, kind="normal")
    B = synth.random_blocks(rng, ks, cs, 0.6, kind="normal")
    C = synth.random_blocks(rng, rs, cs, 0.5, kind="normal")
    check(gpu_ctx, oracle_mod, A, B, 0.75, 1.5, C, eps=0.0)


def test_beta_zero_ignores_nan_c(gpu_ctx, oracle_mod):
    rng = np.random.default_rng(4)
    rs = rng.choice([2, 3, 13], 8)
    A = synth.random_blocks(rng, rs, rs, 0.25, kind="normal")
    C = synth.random_blocks(rng, rs, rs, 0.9, kind="normal")
    C.values[:] = np.nan
    ref, v, _ = check(gpu_ctx, oracle_mod, A, A, 1.0, 0.0, C, eps=0.0)
    assert not np.isnan(v).any()


def test_empty_and_degenerate(gpu_ctx, oracle_mod):
    rs = np.array([2, 3, 5], np.int32)
    E = BlockMatrix(rs, rs, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0))
    C = synth.random_blocks(np.random.default_rng(0), rs, rs, 0.7, kind="int")
    r, c, v, st = run_gpu(gpu_ctx, E, E)
    assert len(r) == 0 and st.candidates == 0
    check(gpu_ctx, oracle_mod, E, E, 1.0, 2.0, C, exact=True)
    A = synth.random_blocks(np.random.default_rng(1), rs, rs, 0.7, kind="int")
    check(gpu_ctx, oracle_mod, A, A, 0.0, -0.5, C, exact=True)  # alpha = 0
    # a single block row / column
    one = np.array([4], np.int32)
    A1 = synth.random_blocks(np.random.default_rng(2), one, rs, 1.0, kind="int")
    B1 = synth.random_blocks(np.random.default_rng(3), rs, one, 1.0, kind="int")
    check(gpu_ctx, oracle_mod, A1, B1, exact=True)


def test_ragged_many_rows(gpu_ctx, oracle_mod):
    """Many block rows (several grid strides of the row-parallel passes) with
    a ragged mix of sizes and empty rows."""
    rng = np.random.default_rng(33)
    n = 2500
    rs = rng.choice([1, 5, 9, 13], n)
    A = synth.random_blocks(rng, rs, rs, 0.004, kind="normal")
    check(gpu_ctx, oracle_mod, A, A, eps=0.0)


def test_chain_and_reuse(gpu_ctx, oracle_mod):
    """C1 = A.A, then C2 = C1.A (a computed matrix as input), then the same C
    handle reused for results of different sizes, asynchronously."""
    A = synth.water(16, seed=9)
    ctx = gpu_ctx
    dA = ctx.from_blocks(A)
    C1 = ctx.empty(A.row_sizes, A.col_sizes)
    C2 = ctx.empty(A.row_sizes, A.col_sizes)
    ctx.multiply(1.0, dA, dA, 0.0, C1, 1e-10)
    ctx.multiply(1.0, C1, dA, 0.0, C2, 1e-10)
    r1 = oracle_mod.multiply(A, A, eps=1e-10)
    M1 = H.result_matrix(r1, A.row_sizes, A.col_sizes)
    r2 = oracle_mod.multiply(M1, A, eps=1e-10)
    r, c = C2.pattern()
    assert np.array_equal(r, r2.blk_row) and np.array_equal(c, r2.blk_col)
    assert H.rel_frobenius(C2.values(), r2.values) <= TOL
    # reuse C2 for a smaller and then a larger result, then beta accumulation
    S = synth.random_blocks(np.random.default_rng(5), A.row_sizes, A.col_sizes, 0.05, kind="normal")
    dS = ctx.from_blocks(S)
    ctx.multiply(1.0, dS, dS, 0.0, C2, 0.0)
    ctx.multiply(1.0, dA, dA, 0.0, C2, 0.0)
    ctx.multiply(2.0, dS, dA, 0.5, C2, 0.0)
    ref_a = oracle_mod.multiply(A, A, eps=0.0)
    ref = oracle_mod.multiply(S, A, alpha=2.0, beta=0.5, C=H.result_matrix(ref_a, A.row_sizes, A.col_sizes))
    r, c = C2.pattern()
    assert np.array_equal(r, ref.blk_row) and np.array_equal(c, ref.blk_col)
    assert H.rel_frobenius(C2.values(), ref.values) <= TOL
    for m in (dA, C1, C2, dS):
        m.destroy()


def test_errors(gpu_ctx, bsm_lib):
    ctx = gpu_ctx
    rs = np.array([2, 3], np.int32)
    with pytest.raises(bsm_lib.BsmError) as e:
        ctx.matrix(rs, rs, [0, 0], [1, 1], np.zeros(12))
    assert e.value.name == "DUPLICATE_BLOCK"
    with pytest.raises(bsm_lib.BsmError) as e:
        ctx.matrix(rs, rs, [0], [2], np.zeros(6))
    assert e.value.name == "OUT_OF_RANGE"
    with pytest.raises(bsm_lib.BsmError) as e:
        ctx.matrix(np.array([0, 3], np.int32), rs, [], [])
    assert e.value.name == "INVALID_ARG"
    A = ctx.matrix(rs, rs, [0, 1], [0, 1], np.ones(13))
    B = ctx.matrix(np.array([3, 2], np.int32), rs, [0], [0], np.ones(6))
    C = ctx.empty(rs, rs)
    with pytest.raises(bsm_lib.BsmError) as e:
        ctx.multiply(1.0, A, B, 0.0, C)
    assert e.value.name == "DIM_MISMATCH"
    with pytest.raises(bsm_lib.BsmError) as e:
        ctx.multiply(1.0, A, A, 0.0, A)
    assert e.value.name == "ALIAS"
    with pytest.raises(bsm_lib.BsmError) as e:
        ctx.multiply(1.0, A, A, 0.0, C, precision=7)
    assert e.value.name in ("UNSUPPORTED", "INVALID_ARG")
    for m in (A, B, C):
        m.destroy()


def test_torch_stream(gpu_ctx, oracle_mod):
    """Work enqueued on a caller's stream (a torch stream) gives the same result."""
    import torch

    A = synth.water(20, seed=3)
    s = torch.cuda.Stream()
    ref, v, _ = check(gpu_ctx, oracle_mod, A, A, eps=1e-10, stream=s)


FP64_KERNELS = range(6)  # BSM_FP64_T16_B2 .. BSM_FP64_G8


@pytest.mark.parametrize("kern", FP64_KERNELS)
def test_each_fp64_kernel(gpu_ctx, oracle_mod, kern):
    """Every FP64 kernel, forced for the whole multiply: integer inputs (exact
    for any summation order) over tile edges 1..33, water blocks with C blocks
    of more than 32 products, alpha/beta with C_in, both launch modes."""
    rng = np.random.default_rng(900 + kern)
    sizes = (1, 2, 5, 6, 9, 13, 16, 17, 23, 32, 33)
    rs, ks, cs = rng.choice(sizes, 12), rng.choice(sizes, 14), rng.choice(sizes, 11)
    A = synth.random_blocks(rng, rs, ks, 0.5, kind="int", shuffle=True)
    B = synth.random_blocks(rng, ks, cs, 0.5, kind="int", shuffle=True)
    C = synth.random_blocks(rng, rs, cs, 0.4, kind="int", shuffle=True)
    for launch in (0, 1):
        check(gpu_ctx, oracle_mod, A, B, 2.0, -1.0, C, eps=0.0, exact=True, fp64_kernel=kern,
              launch=launch)
    W = synth.water(40, seed=11)
    ref, _, st = check(gpu_ctx, oracle_mod, W, W, eps=1e-10, fp64_kernel=kern)
    assert st.kept > 32 * st.c_blocks // 2  # most C blocks span several product batches
    CW = synth.random_blocks(np.random.default_rng(3), W.row_sizes, W.col_sizes, 0.3, kind="normal")
    for launch in (0, 1):
        check(gpu_ctx, oracle_mod, W, W, -0.5, 2.0, CW, eps=1e-6, fp64_kernel=kern, launch=launch)


@pytest.mark.parametrize("kern", FP64_KERNELS)
def test_each_fp64_kernel_nan_and_single(gpu_ctx, oracle_mod, kern):
    def single(v):
        return BlockMatrix(np.array([1], np.int32), np.array([1], np.int32), np.array([0], np.int32),
                           np.array([0], np.int32), np.array([v], np.float64))
    _, _, v, st = run_gpu(gpu_ctx, single(np.nan), single(3.0), eps=1e300, fp64_kernel=kern)
    assert st.kept == 1 and np.isnan(v[0])
    _, _, v, _ = run_gpu(gpu_ctx, single(1.5), single(-2.0), fp64_kernel=kern)
    assert v[0] == -3.0


def test_fp64_kernel_out_of_range(gpu_ctx, bsm_lib):
    rs = np.array([2, 3], np.int32)
    A = gpu_ctx.matrix(rs, rs, [0, 1], [0, 1], np.ones(13))
    C = gpu_ctx.empty(rs, rs)
    for bad in (6, -2):
        with pytest.raises(bsm_lib.BsmError) as e:
            gpu_ctx.multiply(1.0, A, A, 0.0, C, fp64_kernel=bad)
        assert e.value.name == "INVALID_ARG"
    A.destroy()
    C.destroy()


def test_default_fp64_kernel(bsm_lib, oracle_mod):
    """Without a forced or tuned kernel: the packed kernel where C blocks have
    many products (water), g8 where they have about one and at most 8 rows and
    columns (a sparse random pattern of 6-wide blocks), t16 where they have
    about one but are larger (13-wide); all results equal the oracle's. Fresh
    contexts: the product count hint is kept per context."""
    W = synth.water(16, seed=2)
    S = synth.sparse_random(3000, 6, 5e-4, seed=1)
    S13 = synth.sparse_random(1500, 13, 5e-4, seed=2)
    for M, want in ((W, bsm_lib.BSM_FP64_PK12), (S, bsm_lib.BSM_FP64_G8),
                    (S13, bsm_lib.BSM_FP64_T16_B2)):
        ctx = bsm_lib.Context(0)
        try:
            ctx.profile(True)
            ref, _, st = check(ctx, oracle_mod, M, M, eps=1e-10)
            assert ctx.profile_read().last_fp64_kernel == want
            assert (st.kept >= 4 * st.c_blocks) == (want == bsm_lib.BSM_FP64_PK12)
        finally:
            ctx.close()


def _pinned(n, fill=0.0):
    import torch

    a = torch.empty(max(n, 1), dtype=torch.float64, pin_memory=True).numpy()
    a[:] = fill
    return a


@pytest.mark.parametrize("kw", [dict(), dict(fp64_kernel=0), dict(launch=1), dict(precision=1),
                                dict(graph=True)])
def test_host_values(gpu_ctx, oracle_mod, kw):
    """opts.host_values: the device stores the result's values in page-locked
    host memory while the multiply runs (packed kernel epilogue) or right after
    (copy kernel); they equal bsm_mat_get_values bit for bit."""
    A = synth.water(20, seed=6)
    ref = oracle_mod.multiply(A, A, eps=1e-10)
    dA = gpu_ctx.from_blocks(A)
    dC = gpu_ctx.empty(A.row_sizes, A.col_sizes)
    host = _pinned(ref.nnz + 7, np.nan)
    for _ in range(3 if kw.get("graph") else 1):  # graph: capture, then replays
        host[:] = np.nan
        gpu_ctx.multiply(1.0, dA, dA, 0.0, dC, 1e-10, host_out=host, **kw)
        v = dC.values()
        assert len(v) == ref.nnz
        assert np.array_equal(host[:ref.nnz], v)
        assert np.isnan(host[ref.nnz:]).all()
    tol = 2e-6 if kw.get("precision") else TOL
    assert H.rel_frobenius(v, ref.values) <= tol
    dA.destroy()
    dC.destroy()


@pytest.mark.parametrize("prec", [1, 2])
def test_host_values_split_large_blocks(gpu_ctx, oracle_mod, prec):
    """opts.host_values with the split precisions on blocks up to 32 wide: both
    pipelined instances (small and large C blocks) store their C blocks into
    host memory from their epilogues."""
    A = synth.amorphous(60, seed=9, density=0.05, cutoff=6.0)
    ref = oracle_mod.multiply(A, A, eps=1e-8)
    dA = gpu_ctx.from_blocks(A)
    dC = gpu_ctx.empty(A.row_sizes, A.col_sizes)
    host = _pinned(ref.nnz + 3, np.nan)
    gpu_ctx.multiply(1.0, dA, dA, 0.0, dC, 1e-8, host_out=host, precision=prec, blocking=True)
    v = dC.values()
    assert len(v) == ref.nnz and np.array_equal(host[:ref.nnz], v)
    assert np.isnan(host[ref.nnz:]).all()
    assert H.rel_frobenius(v, ref.values) <= 2e-5
    dA.destroy()
    dC.destroy()


def test_host_values_small_or_pageable(gpu_ctx, bsm_lib, oracle_mod):
    A = synth.water(8, seed=1)
    ref = oracle_mod.multiply(A, A, eps=1e-10)
    dA = gpu_ctx.from_blocks(A)
    dC = gpu_ctx.empty(A.row_sizes, A.col_sizes)
    small = _pinned(ref.nnz - 1, -7.0)
    gpu_ctx.multiply(1.0, dA, dA, 0.0, dC, 1e-10, host_out=small, blocking=True)
    assert (small == -7.0).all()  # the result does not fit: nothing written
    assert H.rel_frobenius(dC.values(), ref.values) <= TOL
    with pytest.raises(bsm_lib.BsmError) as e:
        gpu_ctx.multiply(1.0, dA, dA, 0.0, dC, 1e-10, host_out=np.zeros(ref.nnz))
    assert e.value.name == "INVALID_ARG"
    dA.destroy()
    dC.destroy()


def test_assign_reuses_matrix(gpu_ctx, bsm_lib, oracle_mod):
    """bsm_mat_assign: a new block list (smaller, then larger than the buffers)
    in the same handle; multiplies (also graph replays) see the new contents;
    a bad block list leaves the handle unchanged."""
    rng = np.random.default_rng(77)
    rs = rng.choice([1, 5, 13], 30)
    big = synth.random_blocks(rng, rs, rs, 0.5, kind="int")
    small = synth.random_blocks(rng, rs, rs, 0.1, kind="int")
    mid = synth.random_blocks(rng, rs, rs, 0.3, kind="normal", shuffle=True)
    dA = gpu_ctx.from_blocks(mid)
    dC = gpu_ctx.empty(rs, rs)
    for M, graph in ((small, False), (big, True), (mid, True), (small, True)):
        dA.assign(M.blk_row, M.blk_col, M.values)
        for _ in range(2):
            gpu_ctx.multiply(1.0, dA, dA, 0.0, dC, 0.0, graph=graph)
            ref = oracle_mod.multiply(M, M)
            r, c = dC.pattern()
            assert np.array_equal(r, ref.blk_row) and np.array_equal(c, ref.blk_col)
            assert H.rel_frobenius(dC.values(), ref.values) <= TOL
    with pytest.raises(bsm_lib.BsmError) as e:
        dA.assign([0, 0], [1, 1], np.zeros(2 * int(rs[0]) * int(rs[1])))
    assert e.value.name == "DUPLICATE_BLOCK"
    with pytest.raises(bsm_lib.BsmError) as e:
        dA.assign([len(rs)], [0], np.zeros(int(rs[0])))
    assert e.value.name == "OUT_OF_RANGE"
    r, c = dA.pattern()  # still `small`
    assert np.array_equal(r, small.blk_row) and np.array_equal(c, small.blk_col)
    assert np.array_equal(dA.values(), small.values)
    dA.destroy()
    dC.destroy()


def test_assign_beside_queued_multiply(gpu_ctx, bsm_lib, oracle_mod):
    """Uploads run on a stream of their own: an input assigned into one handle
    while a multiply of another is queued, and an input assigned into a handle
    that a queued multiply still reads (that multiply finishes first), leave
    every result equal to the oracle's. 1200 block rows: the row order is
    computed again for each new pattern."""
    eps = 1e-10
    A, B = synth.water(400, seed=51), synth.water(400, seed=52)
    refs = {id(M): oracle_mod.multiply(M, M, eps=eps) for M in (A, B)}
    d = [gpu_ctx.from_blocks(A), gpu_ctx.from_blocks(A)]
    dC = [gpu_ctx.empty(A.row_sizes, A.col_sizes) for _ in range(2)]

    def same(C, M):
        ref = refs[id(M)]
        r, c = C.pattern()
        assert np.array_equal(r, ref.blk_row) and np.array_equal(c, ref.blk_col)
        assert H.rel_frobenius(C.values(), ref.values) <= TOL

    gpu_ctx.multiply(1.0, d[0], d[0], 0.0, dC[0], eps)  # queued: reads d[0] = A
    d[1].assign(B.blk_row, B.blk_col, B.values)          # another handle: no wait
    gpu_ctx.multiply(1.0, d[1], d[1], 0.0, dC[1], eps)  # queued: reads d[1] = B
    d[0].assign(B.blk_row, B.blk_col, B.values)          # waits for the first multiply
    same(dC[0], A)
    same(dC[1], B)
    for k in range(3):  # alternating handles, as a pipelined loop does
        gpu_ctx.multiply(1.0, d[k % 2], d[k % 2], 0.0, dC[0], eps)
        d[(k + 1) % 2].assign(A.blk_row, A.blk_col, A.values)
        same(dC[0], B if k == 0 else A)
        d[k % 2].assign(A.blk_row, A.blk_col, A.values)
    for M in d + dC:
        M.destroy()


@pytest.mark.parametrize("top", [4, 6, 8])
def test_g8_tiny_blocks(gpu_ctx, oracle_mod, bsm_lib, top):
    """The g8 kernel at each of its register-row and lane-group sizes (blocks up
    to 4, 6 and 8 wide pick MR = GS = 4, 6, 8): integer inputs, so the result
    equals the oracle bit for bit; with C_in, alpha and beta; and the default
    choice on such a matrix with about one product per C block."""
    rng = np.random.default_rng(1000 + top)
    sizes = np.arange(1, top + 1)
    rs, ks, cs = rng.choice(sizes, 60), rng.choice(sizes, 50), rng.choice(sizes, 40)
    A = synth.random_blocks(rng, rs, ks, 0.15, kind="int", shuffle=True)
    B = synth.random_blocks(rng, ks, cs, 0.15, kind="int", shuffle=True)
    C = synth.random_blocks(rng, rs, cs, 0.2, kind="int", shuffle=True)
    for launch in (0, 1):
        check(gpu_ctx, oracle_mod, A, B, 2.0, -1.0, C, eps=0.0, exact=True,
              fp64_kernel=bsm_lib.BSM_FP64_G8, launch=launch)
    S = synth.sparse_random(800, top, 2e-3, seed=top)
    ctx = bsm_lib.Context(0)
    try:
        ctx.profile(True)
        _, _, st = check(ctx, oracle_mod, S, S, eps=1e-10)
        assert st.kept < 4 * st.c_blocks
        assert ctx.profile_read().last_fp64_kernel == bsm_lib.BSM_FP64_G8
    finally:
        ctx.close()


def test_long_block_lists(gpu_ctx, bsm_lib):
    """Block lists long enough for the threaded host checks (>= 2^17 blocks):
    a shuffled list gives the same matrix as the sorted one; an index out of
    range in the last chunk is reported and leaves the handle unchanged."""
    n = 600
    rng = np.random.default_rng(12)
    rs = rng.choice([1, 2, 3], n).astype(np.int32)
    mask = rng.random((n, n)) < 0.45
    r, c = np.nonzero(mask)
    r, c = r.astype(np.int32), c.astype(np.int32)
    assert len(r) >= (1 << 17)
    sizes = rs[r].astype(np.int64) * rs[c]
    vals = rng.integers(-4, 5, int(sizes.sum())).astype(np.float64)
    M = gpu_ctx.matrix(rs, rs, r, c, vals)
    r0, c0 = M.pattern()
    v0 = M.values()
    p = rng.permutation(len(r))
    off = np.concatenate([[0], np.cumsum(sizes)])
    pv = np.concatenate([vals[off[b]:off[b + 1]] for b in p])
    M.assign(r[p], c[p], pv)
    r1, c1 = M.pattern()
    assert np.array_equal(r0, r1) and np.array_equal(c0, c1) and np.array_equal(v0, M.values())
    bad = r.copy()
    bad[-1] = n  # out of range, in the last chunk
    with pytest.raises(bsm_lib.BsmError) as e:
        M.assign(bad, c, vals)
    assert e.value.name == "OUT_OF_RANGE"
    r2, c2 = M.pattern()
    assert np.array_equal(r0, r2) and np.array_equal(c0, c2) and np.array_equal(v0, M.values())
    M.destroy()


@pytest.mark.parametrize("kern", ["pk12", "t16b2", "g8"])
def test_row_order_changes_no_result(gpu_ctx, oracle_mod, bsm_lib, kern):
    """A square matrix of at least 1024 block rows carries a breadth-first row
    order, and the persistent launch takes the C blocks in that order. Every
    block is still computed alone: the values equal, bit for bit, those of the
    per-shape-class launch with the same kernel (another order), and the
    oracle's within 1e-12. C = A.A inherits A's order; D = C.A takes its
    blocks in the inherited order. The pattern has several components and is
    not symmetric, so the order covers rows the search reaches late."""
    K = {"pk12": bsm_lib.BSM_FP64_PK12, "t16b2": bsm_lib.BSM_FP64_T16_B2, "g8": bsm_lib.BSM_FP64_G8}[kern]
    rng = np.random.default_rng(41)
    n = 1100
    rs = rng.choice([2, 3, 5, 8], n).astype(np.int32)
    A = synth.random_blocks(rng, rs, rs, 4.0 / n, kind="normal")
    ctx = gpu_ctx
    dA = ctx.from_blocks(A)
    res = {}
    for launch in (bsm_lib.BSM_LAUNCH_PERSISTENT, bsm_lib.BSM_LAUNCH_PER_STACK):
        C = ctx.empty(A.row_sizes, A.col_sizes)
        D = ctx.empty(A.row_sizes, A.col_sizes)
        ctx.multiply(1.0, dA, dA, 0.0, C, 0.0, launch=launch, fp64_kernel=K)
        ctx.multiply(1.0, C, dA, 0.0, D, 0.0, launch=launch, fp64_kernel=K)
        res[launch] = (C.pattern(), C.values(), D.pattern(), D.values())
        C.destroy()
        D.destroy()
    p, q = res[bsm_lib.BSM_LAUNCH_PERSISTENT], res[bsm_lib.BSM_LAUNCH_PER_STACK]
    for a, b in ((p[0], q[0]), (p[2], q[2])):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(p[1], q[1]) and np.array_equal(p[3], q[3])
    ref_c = oracle_mod.multiply(A, A)
    assert np.array_equal(p[0][0], ref_c.blk_row) and np.array_equal(p[0][1], ref_c.blk_col)
    assert H.rel_frobenius(p[1], ref_c.values) <= TOL
    ref_d = oracle_mod.multiply(H.result_matrix(ref_c, A.row_sizes, A.col_sizes), A)
    assert np.array_equal(p[2][0], ref_d.blk_row) and np.array_equal(p[2][1], ref_d.blk_col)
    assert H.rel_frobenius(p[3], ref_d.values) <= TOL
    dA.destroy()


@pytest.mark.parametrize("slices", [2, 7, 64])
def test_numeric_slices(gpu_ctx, oracle_mod, bsm_lib, slices):
    """The FP64 numeric phase in several launches over consecutive ranges of
    the C blocks: every block is still computed alone, so the values equal
    the single launch's bit for bit and the oracle's within 1e-12; a slice
    count out of range is refused."""
    A = synth.water(40, seed=12)
    ref = oracle_mod.multiply(A, A, eps=1e-10)
    r1, c1, v1, _ = run_gpu(gpu_ctx, A, A, eps=1e-10)
    r, c, v, st = run_gpu(gpu_ctx, A, A, eps=1e-10, numeric_slices=slices)
    assert np.array_equal(r, r1) and np.array_equal(c, c1) and np.array_equal(v, v1)
    assert np.array_equal(r, ref.blk_row) and np.array_equal(c, ref.blk_col)
    assert H.rel_frobenius(v, ref.values) <= TOL
    dA = gpu_ctx.from_blocks(A)
    dC = gpu_ctx.empty(A.row_sizes, A.col_sizes)
    with pytest.raises(bsm_lib.BsmError) as e:
        gpu_ctx.multiply(1.0, dA, dA, 0.0, dC, 1e-10, numeric_slices=65)
    assert e.value.name == "INVALID_ARG"
    dA.destroy()
    dC.destroy()
