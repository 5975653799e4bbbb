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
