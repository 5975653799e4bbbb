"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module only builds input matrices. It holds none of the multiply's
arithmetic: no norms, no filter, no block products.

A matrix is a :class:`BlockMatrix` in "block list" form: block row sizes,
block column sizes, the (row, col) of every stored block, and the values of
every block concatenated in list order, each block column-major.

Workloads (the paper's benchmarks use CP2K matrices that are not available, so
these stand in for them with the same block structure):

* :func:`water` -- liquid water, atoms O (13x13 blocks) and H (5x5 blocks),
  DZVP-like sizes; block (i,j) present when the minimum-image distance is under
  the cutoff; entries N(0,1)*exp(-decay*r); symmetric with +5 on the diagonal
  of diagonal blocks. Like H2O-DFT-LS of Table 1 (water, medium occupancy).
* :func:`amorphous` -- uniform random atoms with block sizes drawn from
  {5, 9, 13, 23, 32}; the mixed-size batching case.
* :func:`random_blocks` -- small random block-sparse matrices for edge cases.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class BlockMatrix:
    row_sizes: np.ndarray  # int32[nbr]
    col_sizes: np.ndarray  # int32[nbc]
    blk_row: np.ndarray  # int32[nblk]
    blk_col: np.ndarray  # int32[nblk]
    values: np.ndarray  # float64[nnz], blocks in list order, column-major

    @property
    def nbr(self) -> int:
        return len(self.row_sizes)

    @property
    def nbc(self) -> int:
        return len(self.col_sizes)

    @property
    def nblk(self) -> int:
        return len(self.blk_row)


# Water geometry (Sec. 4 benchmark family H2O-DFT-LS): O-H 0.96 A, H-O-H 104.5 deg,
# liquid density: 64 molecules in a 12.4 A periodic cube.
WATER_OH = 0.96
WATER_HOH_DEG = 104.5
WATER_BOX_64 = 12.4
SIZE_O, SIZE_H = 13, 5


def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """n uniformly distributed rotation matrices from random unit quaternions
    (Shoemake's subgroup algorithm)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a = np.sqrt(1.0 - u1)
    b = np.sqrt(u1)
    w = a * np.sin(2 * np.pi * u2)
    x = a * np.cos(2 * np.pi * u2)
    y = b * np.sin(2 * np.pi * u3)
    z = b * np.cos(2 * np.pi * u3)
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def water_positions(nmol: int, seed: int):
    """Atom positions (O, H, H per molecule), block sizes and box side."""
    rng = np.random.default_rng(seed)
    box = (nmol * WATER_BOX_64 ** 3 / 64.0) ** (1.0 / 3.0)
    O = rng.random((nmol, 3)) * box
    half = np.deg2rad(WATER_HOH_DEG) / 2.0
    body = np.array([[np.sin(half), np.cos(half), 0.0], [-np.sin(half), np.cos(half), 0.0]]) * WATER_OH
    R = _random_rotations(rng, nmol)
    H = O[:, None, :] + np.einsum("nij,hj->nhi", R, body)
    pos = np.empty((nmol, 3, 3))
    pos[:, 0] = O
    pos[:, 1:] = H
    pos = np.mod(pos.reshape(-1, 3), box)
    sizes = np.tile(np.array([SIZE_O, SIZE_H, SIZE_H], dtype=np.int32), nmol)
    return pos, sizes, box, rng


def _pairs_within(pos: np.ndarray, box: float, cutoff: float):
    """All (i, j), i <= j, with minimum-image distance < cutoff, and r_ij
    (periodic k-d tree search, then the distances by the minimum image)."""
    from scipy.spatial import cKDTree

    n = len(pos)
    pos = np.where(pos >= box, pos - box, pos)
    pos = np.where(pos < 0, pos + box, pos)
    tree = cKDTree(pos, boxsize=box)
    pr = tree.query_pairs(cutoff * (1 + 1e-9), output_type="ndarray")
    ii = np.concatenate([pr[:, 0], np.arange(n)]).astype(np.int64)
    jj = np.concatenate([pr[:, 1], np.arange(n)]).astype(np.int64)
    lo, hi = np.minimum(ii, jj), np.maximum(ii, jj)
    d = pos[lo] - pos[hi]
    d -= box * np.round(d / box)
    r = np.sqrt(np.einsum("ak,ak->a", d, d))
    keep = r < cutoff
    lo, hi, r = lo[keep], hi[keep], r[keep]
    order = np.lexsort((hi, lo))
    return lo[order], hi[order], r[order]


def _symmetric_matrix(sizes: np.ndarray, I: np.ndarray, J: np.ndarray, R: np.ndarray,
                      decay: float, diag_shift: float, rng: np.random.Generator) -> BlockMatrix:
    """Symmetric block matrix on the upper pattern (I <= J): off-diagonal blocks
    N(0,1)*exp(-decay*r), mirrored; diagonal blocks symmetric N(0,1) + diag_shift*I.
    Blocks are listed in (row, col) order."""
    sizes = np.asarray(sizes, dtype=np.int32)
    up = I < J
    rows = np.concatenate([I, J[up]]).astype(np.int32)
    cols = np.concatenate([J, I[up]]).astype(np.int32)
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    # src[b]: index into the upper list; tr[b]: block is the mirror of an upper block
    src_all = np.concatenate([np.arange(len(I)), np.nonzero(up)[0]])[order]
    tr_all = np.concatenate([np.zeros(len(I), bool), np.ones(int(up.sum()), bool)])[order]
    lens = sizes[rows].astype(np.int64) * sizes[cols].astype(np.int64)
    off = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    values = np.empty(int(off[-1]), dtype=np.float64)
    # position of each upper block in the final list, and of its mirror
    pos_up = np.empty(len(I), dtype=np.int64)
    pos_up[src_all[~tr_all]] = np.nonzero(~tr_all)[0]
    pos_lo = np.full(len(I), -1, dtype=np.int64)
    pos_lo[src_all[tr_all]] = np.nonzero(tr_all)[0]
    si, sj = sizes[I], sizes[J]
    for a in np.unique(si):
        for b in np.unique(sj):
            sel = np.nonzero((si == a) & (sj == b))[0]
            if len(sel) == 0:
                continue
            # X[p, c, r] = element (r, c) of upper block p (column-major order)
            X = rng.standard_normal((len(sel), b, a))
            diag = I[sel] == J[sel]
            if diag.any():
                D = X[diag]
                iu = np.triu_indices(a)
                # symmetric: mirror the upper triangle (r <= c), then shift the diagonal
                full = np.zeros((len(D), a, a))
                full[:, iu[1], iu[0]] = D[:, iu[1], iu[0]]
                full[:, iu[0], iu[1]] = D[:, iu[1], iu[0]]
                full[:, np.arange(a), np.arange(a)] += diag_shift
                X[diag] = full
            scale = np.exp(-decay * R[sel])
            scale[diag] = 1.0
            X *= scale[:, None, None]
            ln = a * b
            idx = off[pos_up[sel]][:, None] + np.arange(ln)[None, :]
            values[idx] = X.reshape(len(sel), ln)
            lo = pos_lo[sel]
            m = lo >= 0
            if m.any():
                # mirror block (j,i) is b x a; its column-major layout is X[p].T flattened
                idx = off[lo[m]][:, None] + np.arange(ln)[None, :]
                values[idx] = np.transpose(X[m], (0, 2, 1)).reshape(int(m.sum()), ln)
    return BlockMatrix(sizes.copy(), sizes.copy(), rows, cols, values)


def water(nmol: int, seed: int, cutoff: float = 6.0, decay: float = 0.5,
          diag_shift: float = 5.0) -> BlockMatrix:
    """Water-like symmetric block-sparse matrix (dimension 23*nmol)."""
    pos, sizes, box, rng = water_positions(nmol, seed)
    I, J, R = _pairs_within(pos, box, cutoff)
    return _symmetric_matrix(sizes, I, J, R, decay, diag_shift, rng)


AMORPHOUS_SIZES = np.array([5, 9, 13, 23, 32], dtype=np.int32)
AMORPHOUS_PROBS = np.array([0.4, 0.2, 0.2, 0.1, 0.1])


def amorphous(natoms: int, seed: int, density: float = 0.1, cutoff: float = 7.0,
              decay: float = 0.4, diag_shift: float = 5.0) -> BlockMatrix:
    """Amorphous system: uniform random atoms at the given density (atoms/A^3),
    block size per atom drawn from {5, 9, 13, 23, 32} w.p. {.4, .2, .2, .1, .1}."""
    rng = np.random.default_rng(seed)
    box = (natoms / density) ** (1.0 / 3.0)
    pos = rng.random((natoms, 3)) * box
    sizes = rng.choice(AMORPHOUS_SIZES, size=natoms, p=AMORPHOUS_PROBS).astype(np.int32)
    I, J, R = _pairs_within(pos, box, cutoff)
    return _symmetric_matrix(sizes, I, J, R, decay, diag_shift, rng)


def random_blocks(rng: np.random.Generator, row_sizes, col_sizes, density: float,
                  kind: str = "normal", lo: int = -4, hi: int = 4, shuffle: bool = False) -> BlockMatrix:
    """Random block-sparse matrix: each block present with probability density.
    kind="int": integer entries in [lo, hi]; "normal": N(0,1). With shuffle the
    block list comes in random order (the API accepts any order)."""
    row_sizes = np.asarray(row_sizes, dtype=np.int32)
    col_sizes = np.asarray(col_sizes, dtype=np.int32)
    mask = rng.random((len(row_sizes), len(col_sizes))) < density
    rows, cols = np.nonzero(mask)
    rows = rows.astype(np.int32)
    cols = cols.astype(np.int32)
    if shuffle and len(rows):
        p = rng.permutation(len(rows))
        rows, cols = rows[p], cols[p]
    n = int((row_sizes[rows].astype(np.int64) * col_sizes[cols]).sum()) if len(rows) else 0
    if kind == "int":
        values = rng.integers(lo, hi + 1, size=n).astype(np.float64)
    else:
        values = rng.standard_normal(n)
    return BlockMatrix(row_sizes, col_sizes, rows, cols, values)


def paper_workload(name: str) -> BlockMatrix:
    """The synthetic stand-ins by name."""
    if name == "water64":
        return water(64, seed=0)
    if name == "water2048":
        return water(2048, seed=1)
    if name == "amorphous4096":
        return amorphous(4096, seed=2)
    raise KeyError(name)


def dense_blocks(nb: int, bs: int, seed: int) -> BlockMatrix:
    """Fully occupied symmetric matrix of nb x nb blocks of bs x bs (the Dense
    benchmark of Table 1, block 32, scaled to one GPU)."""
    rng = np.random.default_rng(seed)
    n = nb * bs
    X = rng.standard_normal((n, n))
    D = (X + X.T) / np.sqrt(2.0 * n) + 5.0 * np.eye(n) / np.sqrt(n)
    rows, cols = np.divmod(np.arange(nb * nb, dtype=np.int64), nb)
    blocks = D.reshape(nb, bs, nb, bs).transpose(0, 2, 3, 1)  # [i, j, col, row]: column-major
    sizes = np.full(nb, bs, np.int32)
    return BlockMatrix(sizes, sizes.copy(), rows.astype(np.int32), cols.astype(np.int32),
                       np.ascontiguousarray(blocks).reshape(-1))


def sparse_random(nb: int, bs: int, occupancy: float, seed: int) -> BlockMatrix:
    """Symmetric random block pattern with the given block occupancy (off
    diagonal) plus the diagonal, blocks bs x bs (the S-E benchmark of Table 1:
    block 6, occupancy about 0.05%, scaled to one GPU). Entries N(0,1)*0.3,
    diagonal blocks symmetric with +5 on the diagonal."""
    rng = np.random.default_rng(seed)
    npairs = int(round(occupancy * nb * (nb - 1) / 2))
    I = rng.integers(0, nb, 2 * npairs + 16)
    J = rng.integers(0, nb, 2 * npairs + 16)
    keep = I < J
    key = np.unique(I[keep].astype(np.int64) * nb + J[keep])[:npairs]
    I, J = np.divmod(key, nb)
    I = np.concatenate([I, np.arange(nb)])
    J = np.concatenate([J, np.arange(nb)])
    order = np.lexsort((J, I))
    I, J = I[order], J[order]
    R = np.full(len(I), -np.log(0.3) / 0.5)  # entries scaled by exp(-0.5 r) = 0.3
    return _symmetric_matrix(np.full(nb, bs, np.int32), I, J, R, 0.5, 5.0, rng)
