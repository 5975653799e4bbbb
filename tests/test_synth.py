"""The synthetic inputs follow their stated recipe (CPU): water geometry (box
side, O-H length, H-O-H angle, atom order and block sizes), the cutoff rule by
brute-force minimum-image distances, symmetry, the diagonal shift and the
distance decay of the entries, the amorphous size mix and the sparse
occupancy. These fix the workloads the parity tests and the benchmark use."""
import numpy as np

import synth


def _min_image(d, box):
    return d - box * np.round(d / box)


def test_rotations_are_proper():
    R = synth._random_rotations(np.random.default_rng(0), 500)
    eye = np.einsum("nij,nkj->nik", R, R)
    assert np.allclose(eye, np.eye(3), atol=1e-12)
    assert np.allclose(np.linalg.det(R), 1.0, atol=1e-12)


def test_water_geometry():
    # liquid density: 64 molecules in a 12.4 A box; 2048 in 12.4 * 32^(1/3) = 39.37 A
    for nmol, side in ((64, 12.4), (2048, 12.4 * 32.0 ** (1.0 / 3.0))):
        pos, sizes, box, _ = synth.water_positions(nmol, seed=1)
        assert abs(box - side) < 1e-9 * side
        assert pos.shape == (3 * nmol, 3) and (pos >= 0).all() and (pos < box).all()
        assert (sizes[0::3] == 13).all() and (sizes[1::3] == 5).all() and (sizes[2::3] == 5).all()
        assert sizes.sum() == 23 * nmol
        o = pos[0::3]
        h1 = _min_image(pos[1::3] - o, box)
        h2 = _min_image(pos[2::3] - o, box)
        assert np.allclose(np.linalg.norm(h1, axis=1), 0.96, atol=1e-9)
        assert np.allclose(np.linalg.norm(h2, axis=1), 0.96, atol=1e-9)
        cos = np.einsum("ak,ak->a", h1, h2) / 0.96 ** 2
        assert np.allclose(np.degrees(np.arccos(cos)), 104.5, atol=1e-6)


def test_water_pattern_is_the_cutoff_rule():
    nmol, cutoff = 8, 6.0
    pos, sizes, box, _ = synth.water_positions(nmol, seed=3)
    A = synth.water(nmol, seed=3, cutoff=cutoff)
    n = len(pos)
    d = _min_image(pos[:, None, :] - pos[None, :, :], box)
    r = np.linalg.norm(d, axis=2)
    want = {(i, j) for i in range(n) for j in range(n) if r[i, j] < cutoff}
    got = set(zip(A.blk_row.tolist(), A.blk_col.tolist()))
    assert got == want
    # blocks listed in (row, col) order
    key = A.blk_row.astype(np.int64) * n + A.blk_col
    assert (np.diff(key) > 0).all()


def _blocks(A):
    off = np.concatenate([[0], np.cumsum(A.row_sizes[A.blk_row].astype(np.int64) *
                                         A.col_sizes[A.blk_col])])
    out = {}
    for b, (i, j) in enumerate(zip(A.blk_row.tolist(), A.blk_col.tolist())):
        m, n = A.row_sizes[i], A.col_sizes[j]
        out[(i, j)] = A.values[off[b]:off[b + 1]].reshape(n, m).T  # column-major
    return out


def test_water_values_symmetry_shift_and_decay():
    nmol = 24
    pos, _, box, _ = synth.water_positions(nmol, seed=5)
    A = synth.water(nmol, seed=5)
    B = _blocks(A)
    ratios, diag = [], []
    for (i, j), X in B.items():
        assert np.array_equal(X, B[(j, i)].T)  # A_ji = A_ij^T exactly
        if i == j:
            assert np.array_equal(X, X.T)
            diag.append(np.diag(X))
        elif i < j:
            r = np.linalg.norm(_min_image(pos[i] - pos[j], box))
            ratios.append((X / np.exp(-0.5 * r)).ravel())
    z = np.concatenate(ratios)  # N(0,1) after removing the decay
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1.0) < 0.02
    dg = np.concatenate(diag)  # N(0,1) + 5
    assert abs(dg.mean() - 5.0) < 0.1 and abs(dg.std() - 1.0) < 0.1


def test_amorphous_sizes_and_box():
    natoms = 4096
    A = synth.amorphous(natoms, seed=2)
    counts = np.array([(A.row_sizes == s).sum() for s in (5, 9, 13, 23, 32)])
    p = np.array([0.4, 0.2, 0.2, 0.1, 0.1])
    sigma = np.sqrt(natoms * p * (1 - p))
    assert (np.abs(counts - natoms * p) < 4 * sigma).all() and counts.sum() == natoms
    occupancy = len(A.blk_row) / natoms ** 2
    # cutoff 7 A at 0.1 atoms/A^3: about 4/3 pi 7^3 * 0.1 = 144 neighbours per atom
    assert 0.03 < occupancy < 0.04


def test_sparse_random_occupancy():
    nb, occ = 4000, 5e-4
    S = synth.sparse_random(nb, 6, occ, seed=1)
    off = (S.blk_row != S.blk_col).sum()
    assert abs(off / (nb * (nb - 1)) - occ) < 0.1 * occ
    assert ((S.blk_row == S.blk_col).sum()) == nb
    assert (S.row_sizes == 6).all()
