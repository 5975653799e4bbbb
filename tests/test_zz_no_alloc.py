"""The allocation-free entry point bsm_multiply_noalloc, through the C ABI.

Some callers cannot allocate device memory themselves (a framework whose pool
owns the GPU's memory, a callback that must not wait on the allocator); they
pass device buffers they own, and the multiply's temporaries come from a fixed
array inside the library. This test hands it torch-owned device buffers and
checks its result against the ordinary entry point (bsm_multiply) on the same
input, twice in a row (the array keeps the previous call's contents, so the
second call also checks that what must start at zero is cleared).

The file is named to be collected last: if it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest

import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu
TOL = 1e-12


def device_csr(M, torch):
    """Blocked CSR of a block list on the device (test-side marshalling)."""
    from paper_1705_10218_gb300.bsm import DevCsr

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
    t = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in dict(
        rs=np.asarray(M.row_sizes, np.int32), cs=np.asarray(M.col_sizes, np.int32), rp=row_ptr,
        ci=cols.astype(np.int32), bo=off, v=vals.astype(np.float64)).items()}
    s = DevCsr(M.nbr, M.nbc, t["rs"].data_ptr(), t["cs"].data_ptr(), t["rp"].data_ptr(),
               t["ci"].data_ptr(), t["bo"].data_ptr(), t["v"].data_ptr(), len(order))
    return s, t


def test_noalloc_matches_bsm_multiply(bsm_lib):
    import torch

    from paper_1705_10218_gb300.bsm import DevCsrOut, multiply_noalloc

    A = synth.water(64, seed=0)
    eps = 1e-10
    # the ordinary entry point
    ctx = bsm_lib.Context(0)
    dA = ctx.from_blocks(A)
    dC = ctx.empty(A.row_sizes, A.col_sizes)
    ctx.multiply(1.0, dA, dA, 0.0, dC, eps, blocking=True)
    ref_r, ref_c = dC.pattern()
    ref_v = dC.values()
    ctx.close()

    sA, keep = device_csr(A, torch)
    nblk, nnz = len(ref_r), len(ref_v)
    for call in range(2):
        out = {"rp": torch.full((A.nbr + 1,), -1, dtype=torch.int32, device="cuda"),
               "ci": torch.full((nblk + 7,), -1, dtype=torch.int32, device="cuda"),
               "bo": torch.full((nblk + 7,), -1, dtype=torch.int64, device="cuda"),
               "v": torch.full((nnz + 5,), float("nan"), dtype=torch.float64, device="cuda")}
        sC = DevCsrOut(out["rp"].data_ptr(), out["ci"].data_ptr(), out["bo"].data_ptr(),
                       out["v"].data_ptr(), nblk + 7, nnz + 5)
        torch.cuda.synchronize()
        rc, sizes = multiply_noalloc(1.0, sA, sA, eps, sC, stream=torch.cuda.current_stream())
        assert rc == 0, f"call {call}: rc {rc}"
        assert sizes[0] == nblk and sizes[1] == nnz
        rp = out["rp"].cpu().numpy()
        ci = out["ci"].cpu().numpy()[:nblk]
        rows = np.repeat(np.arange(A.nbr, dtype=np.int32), np.diff(rp))
        assert np.array_equal(rows, ref_r) and np.array_equal(ci, ref_c), f"call {call}: pattern"
        v = out["v"].cpu().numpy()[:nnz]
        assert H.rel_frobenius(v, ref_v) <= TOL, f"call {call}: values"


def test_noalloc_rejects_small_output(bsm_lib):
    import torch

    from paper_1705_10218_gb300.bsm import DevCsrOut, multiply_noalloc

    A = synth.water(8, seed=1)
    sA, keep = device_csr(A, torch)
    rp = torch.zeros(A.nbr + 1, dtype=torch.int32, device="cuda")
    ci = torch.zeros(4, dtype=torch.int32, device="cuda")
    bo = torch.zeros(4, dtype=torch.int64, device="cuda")
    v = torch.zeros(16, dtype=torch.float64, device="cuda")
    sC = DevCsrOut(rp.data_ptr(), ci.data_ptr(), bo.data_ptr(), v.data_ptr(), 4, 16)
    rc, sizes = multiply_noalloc(1.0, sA, sA, 0.0, sC, stream=torch.cuda.current_stream())
    assert rc == -1 and sizes[0] > 4  # INVALID_ARG, with the needed sizes reported
