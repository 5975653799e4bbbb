"""ctypes binding of libbsm (include/bsm.h). Argument marshalling only.

The library must have been built (``paper_1705_10218_gb300/build.py`` or
``__graft_entry__.build()``); there is no fallback of any kind: without the
library, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
lib_path = os.path.join(_HERE, "libbsm.so")

BSM_OK = 0
ERRORS = {
    -1: "INVALID_ARG", -2: "DIM_MISMATCH", -3: "DUPLICATE_BLOCK", -4: "OUT_OF_RANGE",
    -5: "ALIAS", -6: "NOMEM", -7: "CUDA", -8: "TIMEOUT", -9: "UNSUPPORTED",
}
BSM_PREC_FP64 = 0
BSM_PREC_SPLIT_BF16X3 = 1
BSM_PREC_SPLIT_TF32X2 = 2
BSM_LAUNCH_PERSISTENT = 0
BSM_LAUNCH_PER_STACK = 1
BSM_FP64_T16_B2 = 0
BSM_FP64_T16_B3 = 1
BSM_FP64_T32 = 2
BSM_FP64_PK12 = 3
BSM_FP64_PK16 = 4
BSM_FP64_G8 = 5
BSM_FP64_NUM_KERNELS = 6
BSM_SPLIT_PANEL = 0
BSM_SPLIT_BLOCKS = 1
BSM_SPLIT_CHUNKS = 2


class BsmError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        name = ERRORS.get(code, str(code))
        detail = ""
        if code == -7 and _lib is not None:
            detail = ": " + _lib.bsm_last_cuda_error().decode()
        super().__init__(f"{where}: BSM_ERR_{name}{detail}")
        self.code = code
        self.name = name


class _Opts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("launch", ctypes.c_int32),
        ("blocking", ctypes.c_int32),
        ("autotune", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
        ("graph", ctypes.c_int32),
        ("fp64_kernel", ctypes.c_int32),
        ("host_values", ctypes.c_void_p),
        ("host_cap", ctypes.c_int64),
        ("split_kernel", ctypes.c_int32),
        ("numeric_slices", ctypes.c_int32),
    ]


class _Stats(ctypes.Structure):
    _fields_ = [
        ("candidates", ctypes.c_int64),
        ("kept", ctypes.c_int64),
        ("dropped", ctypes.c_int64),
        ("c_blocks", ctypes.c_int64),
        ("c_nnz", ctypes.c_int64),
        ("flops", ctypes.c_double),
        ("ms_total", ctypes.c_float),
        ("retries", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class _Profile(ctypes.Structure):
    _fields_ = [
        ("ms_norms", ctypes.c_double),
        ("ms_symbolic", ctypes.c_double),
        ("ms_numeric", ctypes.c_double),
        ("ms_total", ctypes.c_double),
        ("multiplies", ctypes.c_int64),
        ("launches", ctypes.c_int64),
        ("last_fp64_kernel", ctypes.c_int32),
        ("last_split_kernel", ctypes.c_int32),
    ]


@dataclass
class Profile:
    ms_norms: float
    ms_symbolic: float
    ms_numeric: float
    ms_total: float
    multiplies: int
    launches: int
    last_fp64_kernel: int  # BSM_FP64_* of the last FP64 numeric launch, -1 if none
    last_split_kernel: int = -1  # BSM_SPLIT_* of the last split-precision numeric launch


@dataclass
class Stats:
    candidates: int
    kept: int
    dropped: int
    c_blocks: int
    c_nnz: int
    flops: float
    ms_total: float
    retries: int


_lib = None

_P = ctypes.c_void_p
_I32, _I64, _D = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_SIGS = {
    "bsm_ctx_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_P)]),
    "bsm_ctx_destroy": (ctypes.c_int, [_P]),
    "bsm_mat_create": (ctypes.c_int, [_P, _I32, _P, _I32, _P, _I64, _P, _P, _P, ctypes.POINTER(_P)]),
    "bsm_mat_destroy": (ctypes.c_int, [_P]),
    "bsm_multiply": (ctypes.c_int, [_P, _D, _P, _P, _D, _P, _D, ctypes.POINTER(_Opts), ctypes.POINTER(_Stats)]),
    "bsm_mat_nblocks": (ctypes.c_int, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "bsm_mat_get_pattern": (ctypes.c_int, [_P, _I64, _P, _P]),
    "bsm_mat_get_values": (ctypes.c_int, [_P, _I64, _P]),
    "bsm_sync": (ctypes.c_int, [_P]),
    "bsm_selftest_wait": (ctypes.c_int, [_P, ctypes.c_int]),
    "bsm_ctx_profile": (ctypes.c_int, [_P, ctypes.c_int]),
    "bsm_mat_filter": (ctypes.c_int, [_P, _D]),
    "bsm_mat_assign": (ctypes.c_int, [_P, _I64, _P, _P, _P]),
    "bsm_mat_add": (ctypes.c_int, [_P, _D, _P, _D, _P]),
    "bsm_ctx_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(_Profile)]),
    "bsm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "bsm_last_cuda_error": (ctypes.c_char_p, []),
}


def lib():
    """The loaded libbsm (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(lib_path):
            raise RuntimeError(f"libbsm.so is not built ({lib_path}); run __graft_entry__.build()")
        L = ctypes.CDLL(lib_path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != BSM_OK:
        raise BsmError(rc, where)


def _vp(a: np.ndarray | None):
    return None if a is None or a.size == 0 else a.ctypes.data_as(ctypes.c_void_p)


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream"))


class Context:
    """A libbsm context: one device, one stream, one workspace."""

    def __init__(self, device: int = 0):
        h = _P()
        _check(lib().bsm_ctx_create(int(device), ctypes.byref(h)), "bsm_ctx_create")
        self._h = h
        self.device = device
        self._mats: list[Matrix] = []

    @property
    def handle(self):
        return self._h

    def matrix(self, row_sizes, col_sizes, blk_row, blk_col, values=None) -> "Matrix":
        rs = np.ascontiguousarray(row_sizes, dtype=np.int32)
        cs = np.ascontiguousarray(col_sizes, dtype=np.int32)
        br = np.ascontiguousarray(blk_row, dtype=np.int32)
        bc = np.ascontiguousarray(blk_col, dtype=np.int32)
        if br.shape != bc.shape:
            raise BsmError(-1, "bsm_mat_create")
        v = None if values is None else np.ascontiguousarray(values, dtype=np.float64)
        h = _P()
        rc = lib().bsm_mat_create(self._h, len(rs), _vp(rs), len(cs), _vp(cs), len(br), _vp(br),
                                  _vp(bc), _vp(v), ctypes.byref(h))
        _check(rc, "bsm_mat_create")
        m = Matrix(self, h, len(rs), len(cs))
        self._mats.append(m)
        return m

    def from_blocks(self, M) -> "Matrix":
        """From any object with row_sizes, col_sizes, blk_row, blk_col, values."""
        return self.matrix(M.row_sizes, M.col_sizes, M.blk_row, M.blk_col, M.values)

    def empty(self, row_sizes, col_sizes) -> "Matrix":
        return self.matrix(row_sizes, col_sizes, np.zeros(0, np.int32), np.zeros(0, np.int32))

    def multiply(self, alpha, A: "Matrix", B: "Matrix", beta, C: "Matrix", eps: float = 0.0, *,
                 precision: int = BSM_PREC_FP64, launch: int = BSM_LAUNCH_PERSISTENT,
                 blocking: bool = False, autotune: bool = False, stream=None,
                 graph: bool = False, stats: bool = False, fp64_kernel: int | None = None,
                 host_out: np.ndarray | None = None, split_kernel: int | None = None,
                 numeric_slices: int = 0) -> Stats | None:
        """fp64_kernel: one of BSM_FP64_* to force that FP64 kernel, None for the
        library's choice. split_kernel: one of BSM_SPLIT_* likewise for the
        split precisions. host_out: a float64 array in page-locked host memory
        that also receives C's values (bsm_mat_get_values order) while the
        multiply runs, when they fit; valid once the result is complete."""
        hv, hcap = None, 0
        if host_out is not None:
            if host_out.dtype != np.float64 or not host_out.flags.c_contiguous:
                raise ValueError("host_out must be a contiguous float64 array")
            hv, hcap = host_out.ctypes.data, host_out.size
        o = _Opts(int(precision), int(launch), int(bool(blocking)), int(bool(autotune)),
                  _stream_ptr(stream), int(bool(graph)),
                  0 if fp64_kernel is None else int(fp64_kernel) + 1, hv, hcap,
                  0 if split_kernel is None else int(split_kernel) + 1, int(numeric_slices))
        st = _Stats() if stats else None
        rc = lib().bsm_multiply(self._h, float(alpha), A._h, B._h, float(beta), C._h, float(eps),
                                ctypes.byref(o), ctypes.byref(st) if st is not None else None)
        _check(rc, "bsm_multiply")
        if st is None:
            return None
        return Stats(st.candidates, st.kept, st.dropped, st.c_blocks, st.c_nnz, st.flops,
                     st.ms_total, st.retries)

    def sync(self):
        _check(lib().bsm_sync(self._h), "bsm_sync")

    def selftest_wait(self, never_complete: bool):
        """The split kernels' bounded device-side barrier wait on its own
        (bsm_selftest_wait): raises BsmError TIMEOUT when it gives up."""
        _check(lib().bsm_selftest_wait(self._h, int(bool(never_complete))), "bsm_selftest_wait")

    def add(self, alpha, A: "Matrix", beta, C: "Matrix"):
        """C = beta*C + alpha*A on the union of the patterns."""
        _check(lib().bsm_mat_add(self._h, float(alpha), A._h, float(beta), C._h), "bsm_mat_add")

    def profile(self, enable: bool = True):
        _check(lib().bsm_ctx_profile(self._h, int(bool(enable))), "bsm_ctx_profile")

    def profile_read(self) -> Profile:
        p = _Profile()
        _check(lib().bsm_ctx_profile_read(self._h, ctypes.byref(p)), "bsm_ctx_profile_read")
        return Profile(p.ms_norms, p.ms_symbolic, p.ms_numeric, p.ms_total, p.multiplies, p.launches,
                       p.last_fp64_kernel, p.last_split_kernel)

    def close(self):
        if self._h:
            for m in self._mats:
                m._h = None
            lib().bsm_ctx_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Matrix:
    def __init__(self, ctx: Context, h, nbr: int, nbc: int):
        self.ctx = ctx
        self._h = h
        self.nbr = nbr
        self.nbc = nbc

    def nblocks(self) -> tuple[int, int]:
        nb, nz = _I64(), _I64()
        _check(lib().bsm_mat_nblocks(self._h, ctypes.byref(nb), ctypes.byref(nz)), "bsm_mat_nblocks")
        return int(nb.value), int(nz.value)

    def pattern(self) -> tuple[np.ndarray, np.ndarray]:
        nb, _ = self.nblocks()
        r = np.empty(nb, np.int32)
        c = np.empty(nb, np.int32)
        _check(lib().bsm_mat_get_pattern(self._h, nb, _vp(r), _vp(c)), "bsm_mat_get_pattern")
        return r, c

    def values(self, out: np.ndarray | None = None) -> np.ndarray:
        _, nz = self.nblocks()
        if out is None:
            out = np.empty(nz, np.float64)
        if out.dtype != np.float64 or not out.flags.c_contiguous or out.size < nz:
            raise BsmError(-1, "bsm_mat_get_values")
        _check(lib().bsm_mat_get_values(self._h, out.size, _vp(out)), "bsm_mat_get_values")
        return out[:nz]

    def filter(self, eps: float):
        """Drop the blocks whose canonical norm is below eps."""
        _check(lib().bsm_mat_filter(self._h, float(eps)), "bsm_mat_filter")

    def assign(self, blk_row, blk_col, values=None):
        """Replace the block list and values (same block sizes), reusing the
        device buffers."""
        br = np.ascontiguousarray(blk_row, dtype=np.int32)
        bc = np.ascontiguousarray(blk_col, dtype=np.int32)
        if br.shape != bc.shape:
            raise BsmError(-1, "bsm_mat_assign")
        v = None if values is None else np.ascontiguousarray(values, dtype=np.float64)
        _check(lib().bsm_mat_assign(self._h, len(br), _vp(br), _vp(bc), _vp(v)), "bsm_mat_assign")

    def destroy(self):
        if self._h:
            lib().bsm_mat_destroy(self._h)
            self._h = None
            if self in self.ctx._mats:
                self.ctx._mats.remove(self)


# ---------------------------------------------------------------------------
# Allocation-free multiply (bsm_multiply_noalloc): for callers that cannot
# allocate device memory. Every pointer here is a device address the caller
# owns (e.g. torch tensors' data_ptr()); the library adds no allocation.
# ---------------------------------------------------------------------------
class DevCsr(ctypes.Structure):
    _fields_ = [
        ("nbr", ctypes.c_int32), ("nbc", ctypes.c_int32),
        ("row_sizes", ctypes.c_void_p), ("col_sizes", ctypes.c_void_p),
        ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p),
        ("blk_off", ctypes.c_void_p), ("values", ctypes.c_void_p),
        ("nblk", ctypes.c_int64),
    ]


class DevCsrOut(ctypes.Structure):
    _fields_ = [
        ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p),
        ("blk_off", ctypes.c_void_p), ("values", ctypes.c_void_p),
        ("cap_blk", ctypes.c_int64), ("cap_nnz", ctypes.c_int64),
    ]


_SIGS["bsm_multiply_noalloc"] = (ctypes.c_int, [ctypes.c_double, ctypes.POINTER(DevCsr), ctypes.POINTER(DevCsr),
                                                ctypes.c_double, ctypes.POINTER(DevCsrOut),
                                                ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p])


def multiply_noalloc(alpha: float, A: DevCsr, B: DevCsr, eps: float, C: DevCsrOut, stream=None):
    """Calls bsm_multiply_noalloc; returns (rc, (C blocks, C values, kept products))."""
    sizes = (ctypes.c_int64 * 3)()
    rc = lib().bsm_multiply_noalloc(float(alpha), ctypes.byref(A), ctypes.byref(B), float(eps),
                                    ctypes.byref(C), sizes, _stream_ptr(stream))
    return int(rc), (int(sizes[0]), int(sizes[1]), int(sizes[2]))


# ---------------------------------------------------------------------------
# Request loop (bsm_server_*): multiplies C = A.A of independent square systems,
# run with continuous batching on several lanes.
# ---------------------------------------------------------------------------
class _ServerOpts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("precision", ctypes.c_int32), ("hbm_budget", ctypes.c_int64)]


class _ServerInfo(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int64), ("running", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_int64), ("bytes_peak", ctypes.c_int64), ("budget", ctypes.c_int64),
                ("batches", ctypes.c_int64)]


_SIGS.update({
    "bsm_server_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_ServerOpts), ctypes.POINTER(_P)]),
    "bsm_server_destroy": (ctypes.c_int, [_P]),
    "bsm_server_submit": (ctypes.c_int, [_P, _I32, _P, _I64, _P, _P, _P, _D, ctypes.POINTER(_I64)]),
    "bsm_server_submit_borrowed": (ctypes.c_int, [_P, _I32, _P, _I64, _P, _P, _P, _D,
                                                  ctypes.POINTER(_I64)]),
    "bsm_server_progress": (ctypes.c_int, [_P, ctypes.POINTER(_I32)]),
    "bsm_server_poll": (ctypes.c_int, [_P, _I64, ctypes.POINTER(_I32), ctypes.POINTER(_D),
                                       ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "bsm_server_timing": (ctypes.c_int, [_P, _I64, ctypes.POINTER(_D), ctypes.POINTER(_D),
                                         ctypes.POINTER(_D)]),
    "bsm_server_take": (ctypes.c_int, [_P, _I64, _I64, _P, _P, _I64, _P]),
    "bsm_server_result": (ctypes.c_int, [_P, _I64, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                         ctypes.POINTER(_P), ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "bsm_server_release": (ctypes.c_int, [_P, _I64]),
    "bsm_server_get_info": (ctypes.c_int, [_P, ctypes.POINTER(_ServerInfo)]),
})

REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3


class Server:
    def __init__(self, device: int = 0, slots: int = 4, precision: int = BSM_PREC_FP64,
                 hbm_budget: int = 8 << 30):
        h = _P()
        o = _ServerOpts(int(slots), int(precision), int(hbm_budget))
        _check(lib().bsm_server_create(int(device), ctypes.byref(o), ctypes.byref(h)), "bsm_server_create")
        self._h = h
        self._borrowed = {}  # request id -> values array the server reads (borrowed submissions)

    def submit(self, M, eps: float, borrow: bool = False) -> int:
        """Queue C = M.M for a square block matrix M (row sizes = column sizes).
        borrow: the values are uploaded from M's array when the request runs
        instead of being copied now (bsm_server_submit_borrowed; the block list
        must be sorted); the array is kept referenced here until the request is
        released or taken."""
        sz = np.ascontiguousarray(M.row_sizes, dtype=np.int32)
        br = np.ascontiguousarray(M.blk_row, dtype=np.int32)
        bc = np.ascontiguousarray(M.blk_col, dtype=np.int32)
        v = np.ascontiguousarray(M.values, dtype=np.float64)
        rid = _I64()
        fn = "bsm_server_submit_borrowed" if borrow else "bsm_server_submit"
        _check(getattr(lib(), fn)(self._h, len(sz), _vp(sz), len(br), _vp(br), _vp(bc), _vp(v),
                                  float(eps), ctypes.byref(rid)), fn)
        if borrow:
            self._borrowed[int(rid.value)] = v
        return int(rid.value)

    def progress(self) -> int:
        n = _I32()
        _check(lib().bsm_server_progress(self._h, ctypes.byref(n)), "bsm_server_progress")
        return int(n.value)

    def poll(self, rid: int):
        st, lat, nb, nz = _I32(), _D(), _I64(), _I64()
        rc = lib().bsm_server_poll(self._h, int(rid), ctypes.byref(st), ctypes.byref(lat),
                                   ctypes.byref(nb), ctypes.byref(nz))
        if rc != BSM_OK and st.value != REQ_FAILED:
            raise BsmError(rc, "bsm_server_poll")
        return int(st.value), float(lat.value), int(nb.value), int(nz.value)

    def timing(self, rid: int):
        """(submit_ms, wait_ms, run_ms) of a finished request: inside submit,
        queued, and from a lane taking its batch to the result in host memory."""
        a, b, c = _D(), _D(), _D()
        _check(lib().bsm_server_timing(self._h, int(rid), ctypes.byref(a), ctypes.byref(b),
                                       ctypes.byref(c)), "bsm_server_timing")
        return float(a.value), float(b.value), float(c.value)

    def take(self, rid: int):
        st, _, nb, nz = self.poll(rid)
        if st != REQ_DONE:
            raise BsmError(-1, "bsm_server_take")
        r = np.empty(nb, np.int32)
        c = np.empty(nb, np.int32)
        v = np.empty(nz, np.float64)
        _check(lib().bsm_server_take(self._h, int(rid), nb, _vp(r), _vp(c), nz, _vp(v)), "bsm_server_take")
        self._borrowed.pop(int(rid), None)
        return r, c, v

    def result(self, rid: int):
        """A finished request's (rows, cols, values) as numpy views of the
        server's page-locked memory, without a copy; valid until release(rid)."""
        pr, pc, pv, nb, nz = _P(), _P(), _P(), _I64(), _I64()
        _check(lib().bsm_server_result(self._h, int(rid), ctypes.byref(pr), ctypes.byref(pc),
                                       ctypes.byref(pv), ctypes.byref(nb), ctypes.byref(nz)),
               "bsm_server_result")

        def view(ptr, n, ctype, dtype):
            if n == 0:
                return np.zeros(0, dtype)
            return np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ctype)), (n,))

        return (view(pr.value, nb.value, ctypes.c_int32, np.int32),
                view(pc.value, nb.value, ctypes.c_int32, np.int32),
                view(pv.value, nz.value, ctypes.c_double, np.float64))

    def release(self, rid: int):
        """Forget a finished request; its result views become invalid."""
        _check(lib().bsm_server_release(self._h, int(rid)), "bsm_server_release")
        self._borrowed.pop(int(rid), None)

    def info(self) -> dict:
        i = _ServerInfo()
        _check(lib().bsm_server_get_info(self._h, ctypes.byref(i)), "bsm_server_get_info")
        return {k: int(getattr(i, k)) for k, _ in _ServerInfo._fields_}

    def close(self):
        if self._h:
            lib().bsm_server_destroy(self._h)
            self._h = None
            self._borrowed.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
