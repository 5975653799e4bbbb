"""Pins of the CPU oracle against facts that do not come from the oracle itself:
dense integer products, identities, closed forms, exact ties, the filter error
bound, the FLOP convention of Table 1. CPU only."""
import math
import os

import numpy as np
import pytest

import synth
from synth import BlockMatrix
from tests import helpers as H

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- norms

def test_norm_closed_forms(oracle_mod):
    o = oracle_mod
    assert o.block_norm(np.array([3.0, 4.0]), 2, 1) == 5.0
    for r, c in [(1, 1), (5, 5), (13, 13), (13, 5), (32, 32)]:
        # r*c ones: every partial sum is an exact integer
        assert o.block_norm(np.ones(r * c), r, c) == math.sqrt(r * c)
    assert o.block_norm(np.zeros(25), 5, 5) == 0.0
    assert o.block_norm(np.array([-2.0 ** -10]), 1, 1) == 2.0 ** -10


def test_norm_is_column_major_sequential(oracle_mod):
    """With x = 2^27 (x^2 = 2^54, ulp 4) a run of ones is lost if it is added
    after x and kept if added before: 6 ones then x gives 2^54 + 8, and
    later ones round back to it (ties to even), so nrm = nextafter(2^27, inf).
    The big entry sits at (0,2) of a 3x3 block: position 6 in column-major
    order but position 2 in row-major order, so the two orders differ."""
    o = oracle_mod
    blk = np.ones((3, 3))
    blk[0, 2] = 2.0 ** 27
    # column-major order: (0,0)..(2,1) are 6 ones, then x, then 2 ones
    # -> 6 + 2^54 = 2^54 + 8 after rounding (6 is a tie between 4 and 8: even -> 8)
    colmaj = blk.T.reshape(-1)
    got = o.block_norm(colmaj, 3, 3)
    assert got == math.nextafter(2.0 ** 27, math.inf)
    # a 1 x 9 row with x first: every one is lost -> exactly 2^27
    row_first = np.concatenate([[2.0 ** 27], np.ones(8)])
    assert o.block_norm(row_first, 1, 9) == 2.0 ** 27


# ---------------------------------------------------------------- brute force

def _int_case(rng, nbr, nbk, nbc, dens=0.5, sizes=(1, 2, 3, 5)):
    rs = rng.choice(sizes, nbr)
    ks = rng.choice(sizes, nbk)
    cs = rng.choice(sizes, nbc)
    A = synth.random_blocks(rng, rs, ks, dens, kind="int", shuffle=True)
    B = synth.random_blocks(rng, ks, cs, dens, kind="int", shuffle=True)
    C = synth.random_blocks(rng, rs, cs, dens * 0.6, kind="int", shuffle=True)
    return A, B, C


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (2.0, 1.0), (-1.0, -0.5), (0.5, 3.0)])
def test_bruteforce_dense_integer(oracle_mod, seed, alpha, beta):
    """eps = 0 and small integers: every partial sum is an exact integer, so the
    result equals the dense triple-loop product bit for bit, in any order."""
    rng = np.random.default_rng(100 + seed)
    A, B, C = _int_case(rng, 7, 6, 8)
    res = oracle_mod.multiply(A, B, alpha=alpha, beta=beta, C=C, eps=0.0)
    # pattern: (i,j) with some k where A_ik and B_kj exist, plus C_in when beta != 0
    P = (H.presence(A).astype(int) @ H.presence(B).astype(int)) > 0
    if beta != 0:
        P |= H.presence(C)
    exp_r, exp_c = np.nonzero(P)
    assert np.array_equal(res.blk_row, exp_r) and np.array_equal(res.blk_col, exp_c)
    Dexp = alpha * (H.to_dense(A) @ H.to_dense(B))
    if beta != 0:
        Dexp = Dexp + beta * H.to_dense(C)
    got = H.to_dense(H.result_matrix(res, A.row_sizes, B.col_sizes))
    assert np.array_equal(got, Dexp)
    assert res.kept == res.candidates and res.dropped == 0
    # candidates: sum over (i,k) in A of the number of blocks in B's row k
    nB = H.presence(B).sum(axis=1)
    assert res.candidates == int(nB[A.blk_col].sum())


def test_flops_convention_table1(oracle_mod):
    """Table 1: Dense = 10 multiplies of a 60000^2 matrix with 32x32 blocks and
    4.320e15 FLOPs, i.e. 2*n^3 per multiply; the oracle counts 2*m*n*k per kept
    block product, which on a full dense block matrix is 2*n^3."""
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "table1_flops.txt")) if ln.strip() and not ln.startswith("#")]
    dense = [r for r in rows if r[0] == "Dense"][0]
    blk, dim, nmul, pflop = int(dense[1]), int(dense[2]), int(dense[3]), float(dense[4])
    assert nmul * 2 * dim ** 3 == pytest.approx(pflop * 1e15, rel=1e-12)
    assert dim % blk == 0
    rng = np.random.default_rng(7)
    nb = 4
    A = synth.random_blocks(rng, [blk] * nb, [blk] * nb, 1.0, kind="normal")
    res = oracle_mod.multiply(A, A, pattern_only=True)
    n = blk * nb
    assert res.flops == 2.0 * n ** 3
    assert res.kept == nb ** 3


# ---------------------------------------------------------------- identities

def _block_identity(sizes):
    sizes = np.asarray(sizes, np.int32)
    n = len(sizes)
    vals = np.concatenate([np.eye(s).reshape(-1) for s in sizes])
    return BlockMatrix(sizes, sizes, np.arange(n, dtype=np.int32), np.arange(n, dtype=np.int32), vals)


def test_block_identity(oracle_mod):
    rng = np.random.default_rng(3)
    rs = rng.choice([2, 3, 5, 13], 9)
    cs = rng.choice([1, 4, 5], 7)
    A = synth.random_blocks(rng, rs, cs, 0.4, kind="normal", shuffle=True)
    nA = H.numpy_block_norms(A)
    eps = 0.5 * nA.min()  # identity blocks have norm sqrt(s) >= 1
    AI = oracle_mod.multiply(A, _block_identity(cs), eps=eps)
    IA = oracle_mod.multiply(_block_identity(rs), A, eps=eps)
    order = np.lexsort((A.blk_col, A.blk_row))
    Asorted = BlockMatrix(A.row_sizes, A.col_sizes, A.blk_row[order], A.blk_col[order],
                          np.concatenate([H.block_of(A, b).T.reshape(-1) for b in order]))
    for R in (AI, IA):
        assert np.array_equal(R.blk_row, Asorted.blk_row) and np.array_equal(R.blk_col, Asorted.blk_col)
        assert np.array_equal(R.values, Asorted.values)


def test_transpose_identity(oracle_mod):
    """(A.B)^T = B^T.A^T with non-square blocks; same pattern, values to 1e-12."""
    rng = np.random.default_rng(11)
    rs, ks, cs = rng.choice([2, 3, 5], 8), rng.choice([1, 4, 7], 9), rng.choice([3, 6], 6)
    A = synth.random_blocks(rng, rs, ks, 0.35, kind="normal")
    B = synth.random_blocks(rng, ks, cs, 0.35, kind="normal")
    AB = oracle_mod.multiply(A, B, eps=0.0)
    BtAt = oracle_mod.multiply(H.transpose(B), H.transpose(A), eps=0.0)
    T = H.transpose(H.result_matrix(AB, rs, cs))
    assert set(zip(T.blk_row.tolist(), T.blk_col.tolist())) == set(zip(BtAt.blk_row.tolist(), BtAt.blk_col.tolist()))
    D1 = H.to_dense(T)
    D2 = H.to_dense(H.result_matrix(BtAt, cs, rs))
    assert H.rel_frobenius(D2, D1) < 1e-12
    assert H.rel_frobenius(D1, (H.to_dense(A) @ H.to_dense(B)).T) < 1e-12


def test_symmetry_of_square(oracle_mod):
    """A symmetric -> A.A symmetric: C_ij = C_ji^T within 1e-12."""
    A = synth.water(12, seed=5)
    D = H.to_dense(A)
    assert np.array_equal(D, D.T)
    C = oracle_mod.multiply(A, A, eps=1e-10)
    Dc = H.to_dense(H.result_matrix(C, A.row_sizes, A.col_sizes))
    assert H.rel_frobenius(Dc, Dc.T) < 1e-12
    assert H.rel_frobenius(Dc, D @ D) < 1e-12


def test_power_of_two_scaling(oracle_mod):
    rng = np.random.default_rng(21)
    rs = rng.choice([3, 5], 6)
    A = synth.random_blocks(rng, rs, rs, 0.5, kind="normal")
    C = synth.random_blocks(rng, rs, rs, 0.5, kind="normal")
    r1 = oracle_mod.multiply(A, A, alpha=1.0, beta=0.0)
    r2 = oracle_mod.multiply(A, A, alpha=2.0, beta=0.0)
    assert np.array_equal(r2.values, 2.0 * r1.values)
    # beta*C_in with a power-of-two beta and alpha = 0: exactly beta * C_in on C_in's pattern
    r3 = oracle_mod.multiply(A, A, alpha=0.0, beta=-0.5, C=C)
    D3 = H.to_dense(H.result_matrix(r3, rs, rs))
    assert np.array_equal(D3, -0.5 * H.to_dense(C))


def test_beta_zero_ignores_c_in(oracle_mod):
    rng = np.random.default_rng(4)
    rs = rng.choice([2, 3], 6)
    A = synth.random_blocks(rng, rs, rs, 0.2, kind="int")
    C = synth.random_blocks(rng, rs, rs, 0.9, kind="int")
    C.values[:] = np.nan
    r = oracle_mod.multiply(A, A, beta=0.0, C=C)
    P = (H.presence(A).astype(int) @ H.presence(A).astype(int)) > 0
    assert np.array_equal(np.stack(np.nonzero(P)), np.stack([r.blk_row, r.blk_col]))
    assert not np.isnan(r.values).any()


def test_empty_operands(oracle_mod):
    rs = np.array([2, 3], np.int32)
    E = BlockMatrix(rs, rs, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0))
    C = synth.random_blocks(np.random.default_rng(0), rs, rs, 1.0, kind="int")
    r = oracle_mod.multiply(E, E)
    assert r.blk_row.size == 0 and r.candidates == 0
    r = oracle_mod.multiply(E, E, beta=2.0, C=C)
    assert np.array_equal(H.to_dense(H.result_matrix(r, rs, rs)), 2.0 * H.to_dense(C))


# ---------------------------------------------------------------- the filter

def _single(v, r=1, c=1):
    return BlockMatrix(np.array([r], np.int32), np.array([c], np.int32), np.array([0], np.int32),
                       np.array([0], np.int32), np.array(v, np.float64))


def test_filter_tie_is_kept(oracle_mod):
    """nrm(A)=2^-10, nrm(B)=2^-20: the norm product is exactly 2^-30. At
    eps = 2^-30 it is kept (only products strictly below eps are dropped);
    at the next double above 2^-30 it is dropped."""
    A, B = _single([2.0 ** -10]), _single([2.0 ** -20])
    r = oracle_mod.multiply(A, B, eps=2.0 ** -30)
    assert r.kept == 1 and r.dropped == 0 and list(r.values) == [2.0 ** -30]
    r = oracle_mod.multiply(A, B, eps=math.nextafter(2.0 ** -30, math.inf))
    assert r.kept == 0 and r.dropped == 1 and r.blk_row.size == 0
    # a zero block is dropped by any positive eps, kept by eps = 0
    Z = _single([0.0])
    assert oracle_mod.multiply(A, Z, eps=1e-300).kept == 0
    assert oracle_mod.multiply(A, Z, eps=0.0).kept == 1
    # eps <= 0 drops nothing; NaN norms are kept
    assert oracle_mod.multiply(A, B, eps=-1.0).kept == 1
    rn = oracle_mod.multiply(_single([np.nan]), B, eps=1e300)
    assert rn.kept == 1 and np.isnan(rn.values[0])


def test_filter_per_product_and_bound(oracle_mod):
    """The filter acts per block product (i,k,j) on nrm(A_ik)*nrm(B_kj) (Sec. 2).
    Independently of the oracle's own norms: numpy norms decide which products
    are below eps (eps sits between well-separated products), and
    ||C_eps - C_0||_F <= |alpha| * sum_dropped nrm(A_ik) nrm(B_kj)."""
    rng = np.random.default_rng(9)
    rs, ks, cs = rng.choice([2, 5], 10), rng.choice([3, 4], 12), rng.choice([2, 5], 9)
    A = synth.random_blocks(rng, rs, ks, 0.5, kind="normal")
    B = synth.random_blocks(rng, ks, cs, 0.5, kind="normal")
    # spread the block norms over many orders of magnitude
    for M in (A, B):
        bo = H.block_list_offsets(M)
        sc = 10.0 ** rng.uniform(-4, 1, len(M.blk_row))
        for b in range(len(M.blk_row)):
            M.values[bo[b]:bo[b + 1]] *= sc[b]
    nA, nB = H.numpy_block_norms(A), H.numpy_block_norms(B)
    prods = []
    for a in range(len(A.blk_row)):
        for b in np.nonzero(B.blk_row == A.blk_col[a])[0]:
            prods.append((A.blk_row[a], B.blk_col[b], nA[a] * nB[b]))
    pv = np.sort(np.array([p[2] for p in prods]))
    gaps = np.diff(pv) / pv[1:]
    t = int(np.argmax(gaps[len(pv) // 4: 3 * len(pv) // 4])) + len(pv) // 4
    eps = math.sqrt(pv[t] * pv[t + 1])  # well inside a relative gap
    assert gaps[t] > 1e-6
    alpha = -1.5
    r0 = oracle_mod.multiply(A, B, alpha=alpha, eps=0.0)
    re = oracle_mod.multiply(A, B, alpha=alpha, eps=eps)
    dropped = [p for p in prods if p[2] < eps]
    assert re.dropped == len(dropped) and re.kept == len(prods) - len(dropped)
    assert re.candidates == r0.candidates == len(prods)
    kept_pairs = {(int(i), int(j)) for i, j, v in prods if v >= eps}
    assert kept_pairs == set(zip(re.blk_row.tolist(), re.blk_col.tolist()))
    D0 = H.to_dense(H.result_matrix(r0, rs, cs))
    De = H.to_dense(H.result_matrix(re, rs, cs))
    bound = abs(alpha) * sum(p[2] for p in dropped)
    assert np.linalg.norm(De - D0) <= bound * (1 + 1e-12) + 1e-300
    assert np.linalg.norm(De - D0) > 0
    # FLOPs count only kept products
    fl = 0.0
    for a in range(len(A.blk_row)):
        for b in np.nonzero(B.blk_row == A.blk_col[a])[0]:
            if nA[a] * nB[b] >= eps:
                fl += 2.0 * rs[A.blk_row[a]] * ks[A.blk_col[a]] * cs[B.blk_col[b]]
    assert re.flops == fl


def test_alpha_does_not_enter_filter(oracle_mod):
    A, B = _single([2.0 ** -10]), _single([2.0 ** -20])
    r = oracle_mod.multiply(A, B, alpha=1e10, eps=2.0 ** -29)
    assert r.kept == 0


# ---------------------------------------------------------------- plumbing

def test_rows_and_threads_do_not_change_results(oracle_mod):
    A = synth.water(10, seed=2)
    full = oracle_mod.multiply(A, A, eps=1e-10)
    part = [oracle_mod.multiply(A, A, eps=1e-10, rows=(s, min(s + 7, A.nbr)), nthreads=3)
            for s in range(0, A.nbr, 7)]
    assert np.array_equal(np.concatenate([p.blk_row for p in part]), full.blk_row)
    assert np.array_equal(np.concatenate([p.blk_col for p in part]), full.blk_col)
    assert np.array_equal(np.concatenate([p.values for p in part]), full.values)
    mt = oracle_mod.multiply(A, A, eps=1e-10, nthreads=4)
    assert np.array_equal(mt.values, full.values) and mt.flops == full.flops


@pytest.mark.parametrize("bad", ["dup", "range", "zero_size", "dims"])
def test_errors(oracle_mod, bad):
    rs = np.array([2, 3], np.int32)
    A = synth.random_blocks(np.random.default_rng(0), rs, rs, 1.0, kind="int")
    B = A
    if bad == "dup":
        A = BlockMatrix(rs, rs, np.array([0, 0], np.int32), np.array([1, 1], np.int32), np.zeros(12))
        code = -3
    elif bad == "range":
        A = BlockMatrix(rs, rs, np.array([0], np.int32), np.array([2], np.int32), np.zeros(6))
        code = -4
    elif bad == "zero_size":
        A = BlockMatrix(np.array([0, 3], np.int32), rs, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0))
        code = -1
    else:
        B = synth.random_blocks(np.random.default_rng(0), np.array([3, 2], np.int32), rs, 1.0, kind="int")
        code = -2
    with pytest.raises(oracle_mod.OracleError) as ei:
        oracle_mod.multiply(A, B)
    assert ei.value.code == code
