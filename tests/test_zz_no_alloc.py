"""The allocation-free entry point bsm_multiply_noalloc, through the C ABI.

Some callers cannot allocate device memory themselves (a framework whose pool
owns the GPU's memory, a callback that must not wait on the allocator); they
pass device buffers they own, and the multiply's temporaries come from a fixed
array inside the library. These tests hand it torch-owned device buffers and
check its result against the CPU oracle (pattern bit for bit, values within
1e-12 relative Frobenius; integer inputs exactly), twice in a row (the array
keeps the previous call's contents, so the second call also checks that what
must start at zero is cleared). Malformed device arrays must come back as
error codes, a problem larger than the array as UNSUPPORTED, and the call must
work with the library's own device allocations capped at one byte.

The file is named to be collected last: if it fails, a run that stops at the
first failure has already run every other test."""
import os
import subprocess
import sys

import numpy as np
import pytest

import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu
TOL = 1e-12
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def csr_arrays(M):
    """Blocked CSR of a block list (test-side marshalling): row_ptr, columns,
    offsets and values with the blocks of a row sorted by column."""
    order = np.lexsort((M.blk_col, M.blk_row))
    rows, cols = M.blk_row[order], M.blk_col[order]
    lo = H.block_list_offsets(M)
    vals = np.concatenate([M.values[lo[b]:lo[b + 1]] for b in order]) if len(order) else np.zeros(0)
    lens = (np.asarray(M.row_sizes, np.int64)[rows] * np.asarray(M.col_sizes, np.int64)[cols])
    off = np.zeros(len(order), np.int64)
    if len(order):
        off[1:] = np.cumsum(lens)[:-1]
    row_ptr = np.zeros(M.nbr + 1, np.int32)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    return dict(rs=np.array(M.row_sizes, np.int32), cs=np.array(M.col_sizes, np.int32),
                rp=row_ptr, ci=cols.astype(np.int32), bo=off, v=vals.astype(np.float64))


def device_csr(M, torch, edit=None):
    """A bsm_dev_csr over torch-owned device copies of M's CSR arrays; edit
    may change the host arrays first (to build malformed inputs)."""
    from paper_1705_10218_gb300.bsm import DevCsr

    a = csr_arrays(M)
    if edit is not None:
        edit(a)
    t = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in a.items()}
    s = DevCsr(M.nbr, M.nbc, t["rs"].data_ptr(), t["cs"].data_ptr(), t["rp"].data_ptr(),
               t["ci"].data_ptr(), t["bo"].data_ptr(), t["v"].data_ptr(), len(a["ci"]))
    return s, t


def out_buffers(torch, nbr, cap_blk, cap_nnz):
    from paper_1705_10218_gb300.bsm import DevCsrOut

    out = {"rp": torch.full((nbr + 1,), -1, dtype=torch.int32, device="cuda"),
           "ci": torch.full((max(cap_blk, 1),), -1, dtype=torch.int32, device="cuda"),
           "bo": torch.full((max(cap_blk, 1),), -1, dtype=torch.int64, device="cuda"),
           "v": torch.full((max(cap_nnz, 1),), float("nan"), dtype=torch.float64, device="cuda")}
    sC = DevCsrOut(out["rp"].data_ptr(), out["ci"].data_ptr(), out["bo"].data_ptr(),
                   out["v"].data_ptr(), cap_blk, cap_nnz)
    return sC, out


def check_against_oracle(out, ref, nbr, row_sizes, col_sizes, exact):
    nblk, nnz = len(ref.blk_row), len(ref.values)
    rp = out["rp"].cpu().numpy()
    ci = out["ci"].cpu().numpy()[:nblk]
    rows = np.repeat(np.arange(nbr, dtype=np.int32), np.diff(rp))
    assert np.array_equal(rows, ref.blk_row) and np.array_equal(ci, ref.blk_col), "pattern"
    # block offsets: prefix sums of the blocks' sizes in pattern order
    lens = np.asarray(row_sizes, np.int64)[rows] * np.asarray(col_sizes, np.int64)[ci]
    want = np.zeros(nblk, np.int64)
    if nblk:
        want[1:] = np.cumsum(lens)[:-1]
    assert np.array_equal(out["bo"].cpu().numpy()[:nblk], want), "block offsets"
    v = out["v"].cpu().numpy()[:nnz]
    if exact:
        assert np.array_equal(v, ref.values), "values"
    else:
        assert H.rel_frobenius(v, ref.values) <= TOL, "values"


def test_noalloc_matches_oracle_twice(bsm_lib, oracle_mod):
    import torch

    from paper_1705_10218_gb300.bsm import multiply_noalloc

    A = synth.water(64, seed=0)
    eps = 1e-10
    ref = oracle_mod.multiply(A, A, eps=eps)
    sA, keep = device_csr(A, torch)
    nblk, nnz = len(ref.blk_row), len(ref.values)
    for call in range(2):
        sC, out = out_buffers(torch, A.nbr, nblk + 7, nnz + 5)
        torch.cuda.synchronize()
        rc, sizes = multiply_noalloc(1.0, sA, sA, eps, sC, stream=torch.cuda.current_stream())
        assert rc == 0, f"call {call}: rc {rc}"
        assert sizes == (nblk, nnz, ref.kept), f"call {call}: sizes {sizes}"
        check_against_oracle(out, ref, A.nbr, A.row_sizes, A.col_sizes, exact=False)


def test_noalloc_distinct_operands_exact(bsm_lib, oracle_mod):
    """B != A (its own norms and row indices in the array), integer entries
    (exact for any summation order), alpha = 2, filter active."""
    import torch

    from paper_1705_10218_gb300.bsm import multiply_noalloc

    rng = np.random.default_rng(31)
    rs, ks, cs = rng.choice([1, 2, 5, 13], 9), rng.choice([3, 5, 13], 11), rng.choice([1, 5, 7], 8)
    A = synth.random_blocks(rng, rs, ks, 0.5, kind="int", shuffle=True)
    B = synth.random_blocks(rng, ks, cs, 0.5, kind="int", shuffle=True)
    nA, nB = oracle_mod.norms(A), oracle_mod.norms(B)
    eps = float(np.percentile(np.outer(nA, nB), 25))
    ref = oracle_mod.multiply(A, B, alpha=2.0, eps=eps)
    assert ref.dropped > 0
    sA, ka = device_csr(A, torch)
    sB, kb = device_csr(B, torch)
    for call in range(2):
        sC, out = out_buffers(torch, A.nbr, len(ref.blk_row) + 3, len(ref.values) + 3)
        rc, sizes = multiply_noalloc(2.0, sA, sB, eps, sC, stream=torch.cuda.current_stream())
        assert rc == 0 and sizes == (len(ref.blk_row), len(ref.values), ref.kept), (rc, sizes)
        check_against_oracle(out, ref, A.nbr, A.row_sizes, B.col_sizes, exact=True)


def test_noalloc_rejects_small_output(bsm_lib):
    import torch

    from paper_1705_10218_gb300.bsm import multiply_noalloc

    A = synth.water(8, seed=1)
    sA, keep = device_csr(A, torch)
    sC, out = out_buffers(torch, A.nbr, 4, 16)
    rc, sizes = multiply_noalloc(1.0, sA, sA, 0.0, sC, stream=torch.cuda.current_stream())
    assert rc == -1 and sizes[0] > 4  # INVALID_ARG, with the needed sizes reported


def _bad_col(a):
    a["ci"][len(a["ci"]) // 2] = 10 ** 6


def _neg_col(a):
    a["ci"][0] = -1


def _rowptr_decreasing(a):
    a["rp"][3], a["rp"][4] = a["rp"][4], a["rp"][3] - 1


def _rowptr_end(a):
    a["rp"][-1] += 1


def _unsorted(a):
    r = int(np.argmax(np.diff(a["rp"]) >= 2))
    b = int(a["rp"][r])
    a["ci"][b], a["ci"][b + 1] = a["ci"][b + 1], a["ci"][b]


def _duplicate(a):
    r = int(np.argmax(np.diff(a["rp"]) >= 2))
    b = int(a["rp"][r])
    a["ci"][b + 1] = a["ci"][b]


def _zero_size(a):
    a["rs"][2] = 0


def _neg_offset(a):
    a["bo"][5] = -8


@pytest.mark.parametrize("edit,code", [(_bad_col, -4), (_neg_col, -4), (_rowptr_decreasing, -1),
                                       (_rowptr_end, -1), (_unsorted, -1), (_duplicate, -1),
                                       (_zero_size, -1), (_neg_offset, -1)])
def test_noalloc_rejects_malformed_csr(bsm_lib, oracle_mod, edit, code):
    """A malformed device CSR is found by the device check and reported, and
    the next call with good data is still exact."""
    import torch

    from paper_1705_10218_gb300.bsm import multiply_noalloc

    A = synth.water(8, seed=2)
    bad, kb = device_csr(A, torch, edit)
    sC, out = out_buffers(torch, A.nbr, 1 << 14, 1 << 20)
    rc, _ = multiply_noalloc(1.0, bad, bad, 0.0, sC, stream=torch.cuda.current_stream())
    assert rc == code
    good, kg = device_csr(A, torch)
    rc, _ = multiply_noalloc(1.0, good, bad, 0.0, sC, stream=torch.cuda.current_stream())
    assert rc == code  # B alone malformed
    ref = oracle_mod.multiply(A, A, eps=0.0)
    rc, sizes = multiply_noalloc(1.0, good, good, 0.0, sC, stream=torch.cuda.current_stream())
    assert rc == 0
    check_against_oracle(out, ref, A.nbr, A.row_sizes, A.col_sizes, exact=False)


def test_noalloc_dim_mismatch(bsm_lib):
    import torch

    from paper_1705_10218_gb300.bsm import multiply_noalloc

    rng = np.random.default_rng(5)
    A = synth.random_blocks(rng, [2, 3, 4], [3, 5, 2], 0.8, kind="int")
    B = synth.random_blocks(rng, [3, 5, 3], [2, 2], 0.8, kind="int")  # row sizes differ in one place
    sA, ka = device_csr(A, torch)
    sB, kb = device_csr(B, torch)
    sC, out = out_buffers(torch, A.nbr, 64, 4096)
    rc, _ = multiply_noalloc(1.0, sA, sB, 0.0, sC, stream=torch.cuda.current_stream())
    assert rc == -2


def test_noalloc_unsupported_beyond_scratch(bsm_lib):
    """Product records beyond the fixed array: UNSUPPORTED (the output buffers
    are large enough, so the cause is the scratch)."""
    import torch

    from paper_1705_10218_gb300.bsm import multiply_noalloc

    # 170 x 170 blocks of 1 x 1, all present: 170^3 = 4.9 M products (39 MB of
    # records) for a C of only 28,900 values
    A = synth.dense_blocks(170, 1, seed=3)
    sA, keep = device_csr(A, torch)
    sC, out = out_buffers(torch, A.nbr, A.nbr * A.nbr, A.nbr * A.nbr)
    rc, sizes = multiply_noalloc(1.0, sA, sA, 0.0, sC, stream=torch.cuda.current_stream())
    assert rc == -9, (rc, sizes)
    assert sizes[0] <= A.nbr * A.nbr


CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
import synth, oracle
from tests.test_zz_no_alloc import device_csr, out_buffers, check_against_oracle
from paper_1705_10218_gb300.bsm import multiply_noalloc
torch.cuda.init()
A = synth.water(16, seed=4)
ref = oracle.multiply(A, A, eps=1e-10)
sA, keep = device_csr(A, torch)
sC, out = out_buffers(torch, A.nbr, len(ref.blk_row), len(ref.values))
rc, sizes = multiply_noalloc(1.0, sA, sA, 1e-10, sC, stream=torch.cuda.current_stream())
assert rc == 0, rc
check_against_oracle(out, ref, A.nbr, A.row_sizes, A.col_sizes, exact=False)
print("child ok")
"""


def test_noalloc_with_library_allocations_capped(bsm_lib, oracle_mod):
    """With the library's own device allocations capped at one byte (every
    allocation through it fails), the allocation-free call still works."""
    env = dict(os.environ, BSM_DEVICE_MEMORY_CAP="1")
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "child ok" in r.stdout, r.stdout + r.stderr
