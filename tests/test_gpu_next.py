"""GPU parity of the post-multiplication filter, the block-sparse add and the
sign iteration (Eq. 3) against the oracle and a dense eigendecomposition."""
import math

import numpy as np
import pytest

import synth
from synth import BlockMatrix
from tests import helpers as H

pytestmark = pytest.mark.gpu


def test_post_filter_parity(gpu_ctx, oracle_mod):
    A = synth.water(24, seed=8, cutoff=5.0)
    ref_c = oracle_mod.multiply(A, A, eps=1e-10)
    Cm = H.result_matrix(ref_c, A.row_sizes, A.col_sizes)
    nrm = oracle_mod.norms(Cm)
    eps = float(np.percentile(nrm, 40))
    ref = oracle_mod.post_filter(Cm, eps)
    dA = gpu_ctx.from_blocks(A)
    dC = gpu_ctx.empty(A.row_sizes, A.col_sizes)
    gpu_ctx.multiply(1.0, dA, dA, 0.0, dC, 1e-10)
    dC.filter(eps)
    r, c = dC.pattern()
    v = dC.values()
    # the canonical norms of C's blocks may differ in the last bits between the
    # GPU result and the oracle's: blocks within 1e-12 of eps may differ
    near = {(int(Cm.blk_row[b]), int(Cm.blk_col[b])) for b in range(Cm.nblk)
            if abs(nrm[b] / eps - 1.0) < 1e-12}
    got = set(zip(r.tolist(), c.tolist()))
    exp = set(zip(ref.blk_row.tolist(), ref.blk_col.tolist()))
    assert got ^ exp <= near
    if not near:
        assert np.array_equal(r, ref.blk_row) and np.array_equal(c, ref.blk_col)
        assert H.rel_frobenius(v, ref.values) <= 1e-12
    # exact tie on the device: a one-entry block 2^-10 at eps = 2^-10 stays
    one = BlockMatrix(np.array([1], np.int32), np.array([1], np.int32), np.array([0], np.int32),
                      np.array([0], np.int32), np.array([2.0 ** -10]))
    d1 = gpu_ctx.from_blocks(one)
    d1.filter(2.0 ** -10)
    assert d1.nblocks()[0] == 1
    d1.filter(math.nextafter(2.0 ** -10, math.inf))
    assert d1.nblocks()[0] == 0
    for m in (dA, dC, d1):
        m.destroy()


@pytest.mark.parametrize("alpha,beta", [(1.0, 1.0), (-2.0, 0.5), (3.0, 0.0)])
def test_add_parity(gpu_ctx, oracle_mod, alpha, beta):
    rng = np.random.default_rng(21)
    rs, cs = rng.choice([1, 2, 5, 13], 40), rng.choice([1, 5, 13], 30)
    A = synth.random_blocks(rng, rs, cs, 0.3, kind="int", shuffle=True)
    C = synth.random_blocks(rng, rs, cs, 0.3, kind="int", shuffle=True)
    ref = oracle_mod.add(alpha, A, beta, C)
    dA, dC = gpu_ctx.from_blocks(A), gpu_ctx.from_blocks(C)
    gpu_ctx.add(alpha, dA, beta, dC)
    r, c = dC.pattern()
    assert np.array_equal(r, ref.blk_row) and np.array_equal(c, ref.blk_col)
    assert np.array_equal(dC.values(), ref.values)
    dA.destroy()
    dC.destroy()


def test_sign_iteration_gpu(gpu_ctx, oracle_mod):
    from paper_1705_10218_gb300.sign import block_identity, sign_iteration

    A = synth.water(4, seed=3)
    D = H.to_dense(A)
    mu = float(np.median(np.linalg.eigvalsh(D))) + 0.37
    sizes = A.row_sizes
    shifted = gpu_ctx.from_blocks(A)
    gpu_ctx.add(-mu, block_identity(gpu_ctx, sizes), 1.0, shifted)  # A - mu I
    Ds = D - mu * np.eye(len(D))
    scale = np.linalg.norm(Ds)
    X0 = gpu_ctx.empty(sizes, sizes)
    gpu_ctx.add(1.0 / scale, shifted, 0.0, X0)
    w, V = np.linalg.eigh(Ds / scale)
    sign = (V * np.sign(w)) @ V.T
    X = sign_iteration(gpu_ctx, X0, sizes, 40)
    r, c = X.pattern()
    Xd = H.to_dense(BlockMatrix(sizes, sizes, r, c, X.values()))
    assert np.linalg.norm(Xd - sign) / np.linalg.norm(sign) < 1e-9
    assert np.allclose(np.abs(np.linalg.eigvalsh(Xd)), 1.0, atol=1e-9)
    # with filtering the iterate keeps converging (eigenvalues near +-1)
    Xf = sign_iteration(gpu_ctx, X0, sizes, 40, eps=1e-12, filter_eps=1e-10)
    r, c = Xf.pattern()
    Xfd = H.to_dense(BlockMatrix(sizes, sizes, r, c, Xf.values()))
    assert np.linalg.norm(Xfd - sign) / np.linalg.norm(sign) < 1e-6
    for m in (shifted, X0, X, Xf):
        m.destroy()


def test_partial_panels_on_device(gpu_ctx, oracle_mod):
    """The partial C panels of Algorithm 2 (products over 3 disjoint k ranges)
    summed on the device with the block-sparse add, and the tick-by-tick
    accumulation C = C + A_k B_k of Algorithm 1 (beta = 1), both with the
    filter active: the pattern equals the oracle's full product bit for bit,
    values within 1e-12."""
    A = synth.water(24, seed=5, cutoff=5.0)
    nA = oracle_mod.norms(A)
    eps = float(np.percentile(np.outer(nA[:200], nA[:200]), 30))
    grp = np.arange(A.nbc) % 3
    ref = oracle_mod.multiply(A, A, eps=eps)
    acc = gpu_ctx.empty(A.row_sizes, A.col_sizes)
    tick = gpu_ctx.empty(A.row_sizes, A.col_sizes)
    owned = [acc, tick]
    for g in range(3):
        dAg = gpu_ctx.from_blocks(H.select_blocks(A, grp[A.blk_col] == g))
        dBg = gpu_ctx.from_blocks(H.select_blocks(A, grp[A.blk_row] == g))
        P = gpu_ctx.empty(A.row_sizes, A.col_sizes)
        gpu_ctx.multiply(1.0, dAg, dBg, 0.0, P, eps)
        gpu_ctx.add(1.0, P, 1.0, acc)
        gpu_ctx.multiply(1.0, dAg, dBg, 1.0 if g else 0.0, tick, eps)
        owned += [dAg, dBg, P]
    for M in (acc, tick):
        r, c = M.pattern()
        assert np.array_equal(r, ref.blk_row) and np.array_equal(c, ref.blk_col)
        assert H.rel_frobenius(M.values(), ref.values) <= 1e-12
    for m in owned:
        m.destroy()


@pytest.mark.parametrize("alpha,beta", [(1.0, 1.0), (-0.3, 0.7), (1.7, 0.0)])
def test_add_parity_float_bit_exact(gpu_ctx, oracle_mod, alpha, beta):
    """The device add rounds beta*C and alpha*A separately and then their sum,
    as the oracle does: bit-identical values on normal data, including
    many-block rows that span several 32-block copy steps."""
    rng = np.random.default_rng(23)
    rs, cs = rng.choice([1, 5, 13, 32], 60), rng.choice([1, 5, 13], 200)
    A = synth.random_blocks(rng, rs, cs, 0.4, kind="normal", shuffle=True)
    C = synth.random_blocks(rng, rs, cs, 0.4, kind="normal", shuffle=True)
    ref = oracle_mod.add(alpha, A, beta, C)
    dA, dC = gpu_ctx.from_blocks(A), gpu_ctx.from_blocks(C)
    gpu_ctx.add(alpha, dA, beta, dC)
    r, c = dC.pattern()
    assert np.array_equal(r, ref.blk_row) and np.array_equal(c, ref.blk_col)
    assert np.array_equal(dC.values(), ref.values)
    dA.destroy()
    dC.destroy()
