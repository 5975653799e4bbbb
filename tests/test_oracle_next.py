"""Pins of the oracle's post-multiplication filter, block-sparse add, and of the
sign-function iteration built on the oracle multiply (CPU only)."""
import math

import numpy as np
import pytest

import synth
from synth import BlockMatrix
from tests import helpers as H


def _blocks(sizes, entries, vals):
    sizes = np.asarray(sizes, np.int32)
    rows = np.array([e[0] for e in entries], np.int32)
    cols = np.array([e[1] for e in entries], np.int32)
    return BlockMatrix(sizes, sizes, rows, cols, np.concatenate(vals))


def test_post_filter_closed_forms(oracle_mod):
    """Blocks of ones have norm sqrt(r*c) exactly; a one-entry block 2^-10 has
    norm 2^-10: eps decides by 'not below' (a tie is kept)."""
    sizes = [2, 3, 1]
    M = _blocks(sizes, [(0, 0), (1, 2), (2, 1), (2, 2)],
                [np.ones(4), np.ones(3) * 2.0, np.ones(3), np.array([2.0 ** -10])])
    # norms: sqrt(4)=2, sqrt(3*4)=sqrt(12), sqrt(3), 2^-10
    r = oracle_mod.post_filter(M, 2.0)
    assert list(zip(r.blk_row, r.blk_col)) == [(0, 0), (1, 2)]
    r = oracle_mod.post_filter(M, 2.0 ** -10)
    assert len(r.blk_row) == 4
    r = oracle_mod.post_filter(M, math.nextafter(2.0 ** -10, math.inf))
    assert (2, 2) not in set(zip(r.blk_row.tolist(), r.blk_col.tolist()))
    assert len(oracle_mod.post_filter(M, 0.0).blk_row) == 4
    assert len(oracle_mod.post_filter(M, -1.0).blk_row) == 4
    # values of kept blocks are untouched, in (row, col) order
    r = oracle_mod.post_filter(M, math.sqrt(3.0))
    assert np.array_equal(r.values, np.concatenate([np.ones(4), np.ones(3) * 2.0, np.ones(3)]))
    N = _blocks([1], [(0, 0)], [np.array([np.nan])])
    assert len(oracle_mod.post_filter(N, 1e300).blk_row) == 1


def test_post_filter_vs_numpy_norms(oracle_mod):
    rng = np.random.default_rng(3)
    M = synth.random_blocks(rng, rng.choice([2, 5, 13], 12), rng.choice([2, 5, 13], 12), 0.5,
                            kind="normal", shuffle=True)
    nrm = H.numpy_block_norms(M)
    eps = float(np.median(nrm)) * (1 + 1e-9)
    assert np.min(np.abs(nrm / eps - 1)) > 1e-12
    r = oracle_mod.post_filter(M, eps)
    keep = {(int(M.blk_row[b]), int(M.blk_col[b])) for b in range(M.nblk) if nrm[b] >= eps}
    assert set(zip(r.blk_row.tolist(), r.blk_col.tolist())) == keep


@pytest.mark.parametrize("alpha,beta", [(1.0, 1.0), (-2.0, 0.5), (3.0, 0.0), (0.0, -1.0)])
def test_add_dense_integer(oracle_mod, alpha, beta):
    rng = np.random.default_rng(11)
    rs, cs = rng.choice([1, 2, 3, 5], 8), rng.choice([1, 2, 3, 5], 7)
    A = synth.random_blocks(rng, rs, cs, 0.4, kind="int", shuffle=True)
    C = synth.random_blocks(rng, rs, cs, 0.4, kind="int", shuffle=True)
    r = oracle_mod.add(alpha, A, beta, C)
    P = H.presence(A) | (H.presence(C) if beta != 0 else False)
    assert np.array_equal(np.stack(np.nonzero(P)), np.stack([r.blk_row, r.blk_col]))
    D = alpha * H.to_dense(A) + (beta * H.to_dense(C) if beta != 0 else 0)
    assert np.array_equal(H.to_dense(H.result_matrix(r, rs, cs)), D)


def sign_iteration_oracle(oracle_mod, X, eps, iters):
    """X_{n+1} = 1/2 X_n (3I - X_n^2) (Eq. 3) with the oracle multiply."""
    sizes = X.row_sizes
    n = len(sizes)
    I3 = BlockMatrix(sizes, sizes, np.arange(n, dtype=np.int32), np.arange(n, dtype=np.int32),
                     np.concatenate([3.0 * np.eye(s).T.reshape(-1) for s in sizes]))
    for _ in range(iters):
        T = oracle_mod.multiply(X, X, alpha=-1.0, beta=1.0, C=I3, eps=eps)
        T = H.result_matrix(T, sizes, sizes)
        Xn = oracle_mod.multiply(X, T, alpha=0.5, eps=eps)
        X = H.result_matrix(Xn, sizes, sizes)
    return X


def test_sign_iteration_converges_to_sign(oracle_mod):
    """Eq. 3: X converges to sign(X_0) (eigenvalues -1 / +1) when X_0 is scaled
    so that its spectrum lies in (-1, 1); checked against a dense eigen
    decomposition."""
    A = synth.water(4, seed=3)
    D = H.to_dense(A)
    mu = float(np.median(np.linalg.eigvalsh(D))) + 0.37
    sizes = A.row_sizes
    shift = BlockMatrix(sizes, sizes, np.arange(len(sizes), dtype=np.int32),
                        np.arange(len(sizes), dtype=np.int32),
                        np.concatenate([-mu * np.eye(s).reshape(-1) for s in sizes]))
    S = H.result_matrix(oracle_mod.add(1.0, A, 1.0, shift), sizes, sizes)
    Ds = H.to_dense(S)
    scale = np.linalg.norm(Ds)
    X0 = BlockMatrix(S.row_sizes, S.col_sizes, S.blk_row, S.blk_col, S.values / scale)
    w, V = np.linalg.eigh(Ds / scale)
    assert np.min(np.abs(w)) > 1e-3
    sign = (V * np.sign(w)) @ V.T
    X = sign_iteration_oracle(oracle_mod, X0, 0.0, 40)
    assert np.linalg.norm(H.to_dense(X) - sign) / np.linalg.norm(sign) < 1e-9
    ev = np.linalg.eigvalsh(H.to_dense(X))
    assert np.allclose(np.abs(ev), 1.0, atol=1e-9)


def test_partial_panels_sum_to_full_product(oracle_mod):
    """Algorithms 1 and 2: the products over L disjoint k ranges (the partial C
    panels of one process), summed with the block-sparse add, or accumulated
    tick by tick with beta = 1, give the full product: same pattern, and, for
    integer inputs, the same values exactly (dense integer product)."""
    rng = np.random.default_rng(31)
    rs, ks, cs = rng.choice([1, 2, 3, 5], 10), rng.choice([1, 2, 3, 5], 12), rng.choice([1, 2, 3, 5], 9)
    A = synth.random_blocks(rng, rs, ks, 0.5, kind="int", shuffle=True)
    B = synth.random_blocks(rng, ks, cs, 0.5, kind="int", shuffle=True)
    grp = rng.integers(0, 3, len(ks))
    acc = tick = None
    for g in range(3):
        Ag = H.select_blocks(A, grp[A.blk_col] == g)
        Bg = H.select_blocks(B, grp[B.blk_row] == g)
        P = H.result_matrix(oracle_mod.multiply(Ag, Bg), rs, cs)
        acc = P if acc is None else H.result_matrix(oracle_mod.add(1.0, P, 1.0, acc), rs, cs)
        T = oracle_mod.multiply(Ag, Bg, beta=1.0 if tick is not None else 0.0, C=tick)
        tick = H.result_matrix(T, rs, cs)
    full = oracle_mod.multiply(A, B)
    D = H.to_dense(A) @ H.to_dense(B)
    for M in (acc, tick):
        assert np.array_equal(M.blk_row, full.blk_row) and np.array_equal(M.blk_col, full.blk_col)
        assert np.array_equal(H.to_dense(M), D)
