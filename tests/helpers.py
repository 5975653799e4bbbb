"""Test-side helpers: dense expansion of block lists and transposition.

These are plain numpy and belong to the tests only; neither the oracle nor the
GPU path imports them.
"""
import numpy as np

from synth import BlockMatrix


def offsets(sizes):
    o = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(np.asarray(sizes, dtype=np.int64), out=o[1:])
    return o


def block_list_offsets(M):
    lens = np.asarray(M.row_sizes, np.int64)[M.blk_row] * np.asarray(M.col_sizes, np.int64)[M.blk_col]
    return offsets(lens)


def to_dense(M, dtype=np.float64):
    ro, co = offsets(M.row_sizes), offsets(M.col_sizes)
    D = np.zeros((ro[-1], co[-1]), dtype=dtype)
    bo = block_list_offsets(M)
    for b in range(len(M.blk_row)):
        i, j = int(M.blk_row[b]), int(M.blk_col[b])
        r, c = int(M.row_sizes[i]), int(M.col_sizes[j])
        D[ro[i]:ro[i] + r, co[j]:co[j] + c] = np.asarray(M.values[bo[b]:bo[b] + r * c]).reshape(c, r).T
    return D


def presence(M):
    P = np.zeros((len(M.row_sizes), len(M.col_sizes)), dtype=bool)
    P[M.blk_row, M.blk_col] = True
    return P


def transpose(M):
    """Block-list transpose: block (i,j) becomes (j,i) with its values transposed."""
    bo = block_list_offsets(M)
    vals = []
    for b in range(len(M.blk_row)):
        r = int(M.row_sizes[M.blk_row[b]])
        c = int(M.col_sizes[M.blk_col[b]])
        blk = np.asarray(M.values[bo[b]:bo[b] + r * c]).reshape(c, r)  # [col][row]
        vals.append(blk.T.reshape(-1))  # column-major of the c x r transpose
    v = np.concatenate(vals) if vals else np.zeros(0)
    return BlockMatrix(np.asarray(M.col_sizes, np.int32).copy(), np.asarray(M.row_sizes, np.int32).copy(),
                       np.asarray(M.blk_col, np.int32).copy(), np.asarray(M.blk_row, np.int32).copy(), v)


def result_matrix(res, row_sizes, col_sizes):
    return BlockMatrix(np.asarray(row_sizes, np.int32), np.asarray(col_sizes, np.int32),
                       res.blk_row, res.blk_col, res.values)


def block_of(M, b):
    bo = block_list_offsets(M)
    r = int(M.row_sizes[M.blk_row[b]])
    c = int(M.col_sizes[M.blk_col[b]])
    return np.asarray(M.values[bo[b]:bo[b] + r * c]).reshape(c, r).T


def numpy_block_norms(M):
    """Frobenius norms by numpy (not in the canonical order; for checks away from ties)."""
    bo = block_list_offsets(M)
    return np.array([np.linalg.norm(M.values[bo[b]:bo[b + 1]]) for b in range(len(M.blk_row))])


def rel_frobenius(x, y):
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    den = np.linalg.norm(y)
    return float(np.linalg.norm(x - y) / (den if den > 0 else 1.0))


def select_blocks(M, keep):
    """The blocks of M where the boolean array keep (one entry per block) is set,
    in their list order, with their values."""
    keep = np.asarray(keep, bool)
    bo = block_list_offsets(M)
    parts = [np.asarray(M.values[bo[b]:bo[b + 1]]) for b in np.nonzero(keep)[0]]
    v = np.concatenate(parts) if parts else np.zeros(0)
    return BlockMatrix(np.asarray(M.row_sizes, np.int32), np.asarray(M.col_sizes, np.int32),
                       np.asarray(M.blk_row, np.int32)[keep].copy(),
                       np.asarray(M.blk_col, np.int32)[keep].copy(), v)


# ---------------------------------------------------------------------------
# Per-element error bound of the split-precision paths.
#
# A product a.b of FP64 values is replaced by sum over the kept slice pairs of
# a_p.b_q. Slices are cut by truncation: BF16x3 leaves a remainder below
# 2^-23 |a| after three slices and drops pairs (2,3), (3,2), (3,3) whose sum
# is below 2^-21 |a||b|, together u_s = 3 * 2^-22; TF32x2 leaves 2^-21 |a| per
# operand and drops a2.b2 (below 2^-20), u_s = 2^-19. Every slice product is
# exact in FP32; the tensor cores add them in FP32. One MMA with kmma products
# per output adds at most eta = (kmma + 2) * 2^-23 of |accumulator| + sum of
# |terms| (a conservative model that also covers truncating adders); an MMA
# whose terms are all zero adds nothing. |accumulator| never exceeds the sum of
# |terms| added since it last started from zero, and the slices of a value sum
# to at most (1 + 2^-7) times its magnitude, so an accumulator that takes W
# MMAs before it is folded exactly (TwoSum) or read out contributes at most
# W * eta * (1 + 2^-6) * (|A| |B|)_element.
#   per-block kernel: folds every 4 products: W = 4 * pairs * k steps of the
#     largest k block (BF16: 6 pairs, k steps of 16; TF32: 3 pairs, of 8);
#   panel kernel: one FP32 accumulator per element over the row's K steps;
#     only steps that hold a product of the element's C block count: a block
#     of np 16-byte pieces (8 BF16 / 4 TF32 values) spans at most
#     (np + 2) // 2 steps of 2 pieces, and each step adds the slices' MMAs
#     (3 for BF16, 2 for TF32) into the element's group.
# The groups are then combined with one FP32 rounding below 2^-24 of a group
# 2^-8 smaller than the result and an exact TwoSum, and C is formed in FP64.
# ---------------------------------------------------------------------------
def split_block_factors(A, B, prec, kernel, rows=None):
    """Bound factor per C block of the candidate pattern of A.B (a dict
    (i, j) -> factor is not needed: returns a function of block row / column
    arrays). prec: "bf16x3" / "tf32x2"; kernel: "blocks" / "chunks" / "panel"."""
    import scipy.sparse as sp

    bf = prec == "bf16x3"
    u_s = 3 * 2.0 ** -22 if bf else 2.0 ** -19
    kmma = 16 if bf else 8
    eta = (kmma + 2) * 2.0 ** -23
    ks = np.asarray(A.col_sizes, np.int64)
    if kernel in ("blocks", "chunks"):
        # per-block kernel: 4 products between folds, each ceil(k / kmma) k steps
        # of every slice pair into one FP32 accumulator
        w = 4 * (6 if bf else 3) * int(-(-ks.max() // kmma))
        if kernel == "chunks":
            # chunks of 8 pieces of k (two per k step): 4 k steps of every slice
            # pair between folds; C blocks beyond 16 x 16 take the per-block kernel
            w = max(w, 4 * (6 if bf else 3))
        const = u_s + w * eta * (1 + 2.0 ** -6)
        return lambda bi, bj: np.full(len(bi), const)
    piece = 8 if bf else 4
    nsl = 3 if bf else 2
    steps = ((-(-ks // piece)) + 2) // 2
    PA = sp.csr_matrix((np.ones(len(A.blk_row)), (A.blk_row, A.blk_col)), shape=(len(A.row_sizes), len(ks)))
    PB = sp.csr_matrix((np.ones(len(B.blk_row)), (B.blk_row, B.blk_col)), shape=(len(ks), len(B.col_sizes)))
    if rows is not None:
        PA = PA[rows[0]:rows[1]]
    S = (PA @ sp.diags(steps.astype(np.float64)) @ PB).tocsr()
    r0 = rows[0] if rows is not None else 0

    def f(bi, bj):
        n = np.asarray(S[np.asarray(bi) - r0, np.asarray(bj)]).ravel()
        return u_s + nsl * n * eta * (1 + 2.0 ** -6)

    return f


def split_elem_bound(A, B, prec, kernel, blk_row, blk_col, absvals, rows=None):
    """Per-element bound (the layout of a result's values) for the pattern
    (blk_row, blk_col) with |A||B| values absvals."""
    fac = split_block_factors(A, B, prec, kernel, rows)(blk_row, blk_col)
    lens = np.asarray(A.row_sizes, np.int64)[blk_row] * np.asarray(B.col_sizes, np.int64)[blk_col]
    return np.repeat(fac, lens) * np.asarray(absvals) + 1e-300
