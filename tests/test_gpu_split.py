"""GPU parity of the split-precision paths (BF16x3, TF32x2) against the CPU
oracle, through the C ABI, for the three split-precision kernels (the per-block
and the chunked mma.sync kernels, the tcgen05 row-panel kernel).

* Small integers (|a| <= 4): every slice after the first is zero, every slice
  product is exact and all FP32 partial sums stay far below 2^24, so the result
  must equal the oracle bit for bit.
* General values: the pattern is bit-exact (same symbolic phase) and every
  element obeys the bound derived from the kernel's own accumulation
  (tests/helpers.py: split_elem_bound): the slices' truncation error u_s plus
  the FP32 error of each accumulator between exact folds, all relative to
  (|A| |B|) of that element.
"""
import numpy as np
import pytest

import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu
PRECS = {"bf16x3": 1, "tf32x2": 2}
KERNELS = {"blocks": 1, "panel": 0, "chunks": 2}  # BSM_SPLIT_BLOCKS, _PANEL, _CHUNKS
# stated relative Frobenius bounds on water (measured: blocks 6.4e-7 / 8.4e-7,
# panel 2.2e-6 / 4.4e-6 on water2048)
REL_F = {("blocks", "bf16x3"): 2e-6, ("blocks", "tf32x2"): 1e-5,
         ("chunks", "bf16x3"): 2e-6, ("chunks", "tf32x2"): 1e-5,
         ("panel", "bf16x3"): 1e-5, ("panel", "tf32x2"): 2e-5}


def gpu_mult(ctx, A, B, prec, kernel, alpha=1.0, beta=0.0, C=None, eps=0.0):
    dA = ctx.from_blocks(A)
    dB = dA if B is A else ctx.from_blocks(B)
    dC = ctx.from_blocks(C) if C is not None else ctx.empty(A.row_sizes, B.col_sizes)
    st = ctx.multiply(alpha, dA, dB, beta, dC, eps, precision=PRECS[prec], stats=True,
                      split_kernel=KERNELS[kernel])
    r, c = dC.pattern()
    v = dC.values()
    for m in {id(dA): dA, id(dB): dB, id(dC): dC}.values():
        m.destroy()
    return r, c, v, st


# block size sets: rows of A / inner k / columns of B. "mixed" has C blocks
# beyond 16 (per-block kernel: two launches; panel kernel: NR = 32); "small"
# keeps everything within 16 (the half k steps of k <= 8 (BF16) and k <= 4
# (TF32)); "wide_k" has C blocks within 16 but k up to 32.
SIZE_SETS = {"mixed": ((1, 2, 5, 9, 13, 23, 32),) * 3,
             "small": ((1, 2, 3, 4, 5, 7, 8, 13, 16),) * 3,
             "wide_k": ((1, 3, 5, 13, 16), (4, 9, 17, 24, 31, 32), (2, 5, 8, 13, 16))}


@pytest.mark.parametrize("kernel", sorted(KERNELS))
@pytest.mark.parametrize("prec", sorted(PRECS))
@pytest.mark.parametrize("sizes", sorted(SIZE_SETS))
@pytest.mark.parametrize("seed", range(3))
def test_split_integer_exact(gpu_ctx, oracle_mod, kernel, prec, sizes, seed):
    rng = np.random.default_rng(700 + seed)
    rsz, ksz, csz = SIZE_SETS[sizes]
    rs, ks, cs = rng.choice(rsz, 7), rng.choice(ksz, 8), rng.choice(csz, 6)
    A = synth.random_blocks(rng, rs, ks, 0.5, kind="int", shuffle=True)
    B = synth.random_blocks(rng, ks, cs, 0.5, kind="int", shuffle=True)
    ref = oracle_mod.multiply(A, B, eps=0.0)
    r, c, v, st = gpu_mult(gpu_ctx, A, B, prec, kernel)
    assert np.array_equal(r, ref.blk_row) and np.array_equal(c, ref.blk_col)
    assert st.kept == ref.kept and st.flops == ref.flops
    assert np.array_equal(v, ref.values)


def _abs(M):
    return synth.BlockMatrix(M.row_sizes, M.col_sizes, M.blk_row, M.blk_col, np.abs(M.values))


@pytest.mark.parametrize("kernel", sorted(KERNELS))
@pytest.mark.parametrize("prec", sorted(PRECS))
def test_split_water_bound(gpu_ctx, oracle_mod, kernel, prec):
    A = synth.water(64, seed=0)
    eps = 1e-10
    ref = oracle_mod.multiply(A, A, eps=eps)
    absref = oracle_mod.multiply(_abs(A), _abs(A), eps=eps)  # same filter: norms ignore signs
    r, c, v, st = gpu_mult(gpu_ctx, A, A, prec, kernel, eps=eps)
    assert np.array_equal(r, ref.blk_row) and np.array_equal(c, ref.blk_col)
    bound = H.split_elem_bound(A, A, prec, kernel, r, c, absref.values)
    assert np.all(np.abs(v - ref.values) <= bound)
    rel = H.rel_frobenius(v, ref.values)
    assert rel <= REL_F[(kernel, prec)], rel
    # the largest error, relative to the largest element
    assert np.max(np.abs(v - ref.values)) <= REL_F[(kernel, prec)] * np.max(np.abs(ref.values))


@pytest.mark.parametrize("kernel", sorted(KERNELS))
@pytest.mark.parametrize("prec", sorted(PRECS))
@pytest.mark.parametrize("sizes", sorted(SIZE_SETS))
def test_split_general_values(gpu_ctx, oracle_mod, kernel, prec, sizes):
    """Normal values on each size set: every slice plane takes part, so a
    misplaced plane, row or k piece shows as an error far above the bound."""
    rng = np.random.default_rng(800)
    rsz, ksz, csz = SIZE_SETS[sizes]
    rs, ks, cs = rng.choice(rsz, 12), rng.choice(ksz, 14), rng.choice(csz, 10)
    A = synth.random_blocks(rng, rs, ks, 0.5, kind="normal", shuffle=True)
    B = synth.random_blocks(rng, ks, cs, 0.5, kind="normal", shuffle=True)
    ref = oracle_mod.multiply(A, B, eps=0.0)
    absref = oracle_mod.multiply(_abs(A), _abs(B), eps=0.0)
    r, c, v, st = gpu_mult(gpu_ctx, A, B, prec, kernel)
    assert np.array_equal(r, ref.blk_row) and np.array_equal(c, ref.blk_col)
    bound = H.split_elem_bound(A, B, prec, kernel, r, c, absref.values)
    assert np.all(np.abs(v - ref.values) <= bound)
    assert H.rel_frobenius(v, ref.values) <= REL_F[(kernel, prec)]


@pytest.mark.parametrize("kernel", sorted(KERNELS))
@pytest.mark.parametrize("prec", sorted(PRECS))
def test_split_mixed_sizes_alpha_beta(gpu_ctx, oracle_mod, kernel, prec):
    """Amorphous-style sizes {5,9,13,23,32}, alpha/beta != (1, 0), filter active."""
    A = synth.amorphous(80, seed=4, density=0.05, cutoff=6.0)
    rng = np.random.default_rng(1)
    C = synth.random_blocks(rng, A.row_sizes, A.col_sizes, 0.2, kind="normal")
    nA = oracle_mod.norms(A)
    eps = float(np.percentile(np.outer(nA[:50], nA[:50]), 20))
    ref = oracle_mod.multiply(A, A, alpha=0.75, beta=-1.25, C=C, eps=eps)
    absref = oracle_mod.multiply(_abs(A), _abs(A), eps=eps)
    r, c, v, st = gpu_mult(gpu_ctx, A, A, prec, kernel, alpha=0.75, beta=-1.25, C=C, eps=eps)
    assert np.array_equal(r, ref.blk_row) and np.array_equal(c, ref.blk_col)
    assert st.dropped == ref.dropped and st.dropped > 0
    # the product part on the absref pattern: bound on |alpha| |A||B|
    Rg = H.to_dense(H.result_matrix(type("R", (), dict(blk_row=r, blk_col=c, values=v))(), A.row_sizes, A.col_sizes))
    Rr = H.to_dense(H.result_matrix(ref, A.row_sizes, A.col_sizes))
    Ab = H.to_dense(H.result_matrix(type("R", (), dict(
        blk_row=absref.blk_row, blk_col=absref.blk_col,
        values=H.split_elem_bound(A, A, prec, kernel, absref.blk_row, absref.blk_col, absref.values)))(),
        A.row_sizes, A.col_sizes))
    bound = 0.75 * Ab + 1e-12 * np.abs(Rr) + 1e-300
    assert np.all(np.abs(Rg - Rr) <= bound)


@pytest.mark.parametrize("kernel", sorted(KERNELS))
def test_split_empty_rows_and_cin_only_blocks(gpu_ctx, oracle_mod, kernel):
    """Rows of A without blocks and C blocks that come only from C_in
    (beta != 0): blocks with no products (empty chunks, an empty product
    stream) give exactly beta * C_in."""
    rng = np.random.default_rng(9)
    rs = np.array([5, 13, 5, 13, 7, 3], np.int32)
    A = synth.random_blocks(rng, rs, rs, 0.4, kind="int")
    keep = A.blk_row != 2  # block row 2 of A empty
    A = H.select_blocks(A, keep)
    C = synth.random_blocks(rng, rs, rs, 0.5, kind="int")
    for prec in PRECS:
        ref = oracle_mod.multiply(A, A, alpha=1.0, beta=2.0, C=C, eps=0.0)
        r, c, v, st = gpu_mult(gpu_ctx, A, A, prec, kernel, alpha=1.0, beta=2.0, C=C)
        assert np.array_equal(r, ref.blk_row) and np.array_equal(c, ref.blk_col)
        assert np.array_equal(v, ref.values)


@pytest.mark.parametrize("kernel", sorted(KERNELS))
def test_split_rejects_large_blocks(gpu_ctx, bsm_lib, kernel):
    rs = np.array([40, 3], np.int32)
    A = gpu_ctx.matrix(rs, rs, [0], [0], np.ones(1600))
    C = gpu_ctx.empty(rs, rs)
    with pytest.raises(bsm_lib.BsmError) as e:
        gpu_ctx.multiply(1.0, A, A, 0.0, C, precision=1, split_kernel=KERNELS[kernel])
    assert e.value.name == "UNSUPPORTED"
    A.destroy()
    C.destroy()
