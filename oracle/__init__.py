"""CPU oracle for the filtered block-sparse multiply -- TEST INFRASTRUCTURE ONLY.

The arithmetic lives in ``bsm_oracle.c`` (plain FP64 C, compiled with
``-ffp-contract=off``); this module only builds it and marshals numpy arrays.
It computes, by the definition in Sec. 2 of the paper (blocked CSR, on-the-fly
filtering on the product of block norms) and Algorithm 1 (C = C + A.B),

    C = beta * C_in + alpha * sum_{k kept} A_ik B_kj .

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of
``bench.py`` may import this package. The GPU path never does, and this package
never imports the GPU path.

Matrices are passed as any object with the attributes ``row_sizes``,
``col_sizes``, ``blk_row``, ``blk_col`` and ``values`` (blocks in list order,
each column-major), e.g. ``synth.BlockMatrix``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bsm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

ERRORS = {
    -1: "INVALID_ARG",
    -2: "DIM_MISMATCH",
    -3: "DUPLICATE_BLOCK",
    -4: "OUT_OF_RANGE",
    -6: "NOMEM",
}


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle error {code} ({ERRORS.get(code, '?')})")
        self.code = code


def build(force: bool = False) -> str:
    """Compile bsm_oracle.c into liboracle.so beside it (OpenMP when available)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", _LIB_PATH + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class _Mat(ctypes.Structure):
    _fields_ = [
        ("nbr", ctypes.c_int32),
        ("nbc", ctypes.c_int32),
        ("row_sizes", ctypes.c_void_p),
        ("col_sizes", ctypes.c_void_p),
        ("nblk", ctypes.c_int64),
        ("blk_row", ctypes.c_void_p),
        ("blk_col", ctypes.c_void_p),
        ("values", ctypes.c_void_p),
    ]


class _Res(ctypes.Structure):
    _fields_ = [
        ("nblk", ctypes.c_int64),
        ("nnz", ctypes.c_int64),
        ("blk_row", ctypes.POINTER(ctypes.c_int32)),
        ("blk_col", ctypes.POINTER(ctypes.c_int32)),
        ("blk_off", ctypes.POINTER(ctypes.c_int64)),
        ("values", ctypes.POINTER(ctypes.c_double)),
        ("candidates", ctypes.c_int64),
        ("kept", ctypes.c_int64),
        ("dropped", ctypes.c_int64),
        ("flops", ctypes.c_double),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.bsmo_block_norm.restype = ctypes.c_double
        lib.bsmo_block_norm.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
        lib.bsmo_multiply.restype = ctypes.c_int
        lib.bsmo_multiply.argtypes = [
            ctypes.POINTER(_Mat), ctypes.POINTER(_Mat), ctypes.POINTER(_Mat),
            ctypes.c_double, ctypes.c_double, ctypes.c_double,
            ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
            ctypes.POINTER(_Res),
        ]
        lib.bsmo_free_result.restype = None
        lib.bsmo_free_result.argtypes = [ctypes.POINTER(_Res)]
        lib.bsmo_norms.restype = ctypes.c_int
        lib.bsmo_norms.argtypes = [ctypes.POINTER(_Mat), ctypes.c_void_p]
        lib.bsmo_post_filter.restype = ctypes.c_int
        lib.bsmo_post_filter.argtypes = [ctypes.POINTER(_Mat), ctypes.c_double, ctypes.POINTER(_Res)]
        lib.bsmo_add.restype = ctypes.c_int
        lib.bsmo_add.argtypes = [ctypes.POINTER(_Mat), ctypes.POINTER(_Mat), ctypes.c_double,
                                 ctypes.c_double, ctypes.POINTER(_Res)]
        lib.bsmo_max_threads.restype = ctypes.c_int
        lib.bsmo_max_threads.argtypes = []
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a.size else None


class _Held:
    """Keeps the contiguous numpy copies alive while C reads them."""

    def __init__(self, m):
        self.rs = np.ascontiguousarray(m.row_sizes, dtype=np.int32)
        self.cs = np.ascontiguousarray(m.col_sizes, dtype=np.int32)
        self.br = np.ascontiguousarray(m.blk_row, dtype=np.int32)
        self.bc = np.ascontiguousarray(m.blk_col, dtype=np.int32)
        vals = getattr(m, "values", None)
        self.v = None if vals is None else np.ascontiguousarray(vals, dtype=np.float64)
        self.s = _Mat(
            len(self.rs), len(self.cs), _ptr(self.rs), _ptr(self.cs), len(self.br),
            _ptr(self.br), _ptr(self.bc), None if self.v is None else _ptr(self.v),
        )


@dataclass
class Result:
    blk_row: np.ndarray
    blk_col: np.ndarray
    blk_off: np.ndarray
    values: np.ndarray | None
    nnz: int
    candidates: int
    kept: int
    dropped: int
    flops: float


def max_threads() -> int:
    return int(_load().bsmo_max_threads())


def block_norm(block: np.ndarray, r: int, c: int) -> float:
    """Canonical norm of one r x c block given as its column-major values."""
    x = np.ascontiguousarray(block, dtype=np.float64)
    assert x.size == r * c
    return float(_load().bsmo_block_norm(r, c, _ptr(x)))


def norms(m) -> np.ndarray:
    """Canonical norms of every block of m, in list order."""
    h = _Held(m)
    out = np.empty(len(h.br), dtype=np.float64)
    rc = _load().bsmo_norms(ctypes.byref(h.s), _ptr(out))
    if rc:
        raise OracleError(rc)
    return out


def multiply(A, B, alpha: float = 1.0, beta: float = 0.0, C=None, eps: float = 0.0,
             rows: tuple[int, int] | None = None, pattern_only: bool = False,
             nthreads: int = 1) -> Result:
    """C = beta*C_in + alpha*A.B with the on-the-fly filter, over all C block rows
    (or the half-open range ``rows``). Returns the pattern sorted by (row, col)."""
    lib = _load()
    ha, hb = _Held(A), _Held(B)
    hc = _Held(C) if C is not None else None
    res = _Res()
    r0, r1 = rows if rows is not None else (0, 0)
    rc = lib.bsmo_multiply(
        ctypes.byref(ha.s), ctypes.byref(hb.s), ctypes.byref(hc.s) if hc else None,
        float(alpha), float(beta), float(eps), int(r0), int(r1), int(bool(pattern_only)),
        int(nthreads), ctypes.byref(res),
    )
    if rc:
        raise OracleError(rc)
    try:
        nb, nnz = int(res.nblk), int(res.nnz)
        br = np.ctypeslib.as_array(res.blk_row, (nb,)).copy() if nb else np.zeros(0, np.int32)
        bc = np.ctypeslib.as_array(res.blk_col, (nb,)).copy() if nb else np.zeros(0, np.int32)
        bo = np.ctypeslib.as_array(res.blk_off, (nb,)).copy() if nb else np.zeros(0, np.int64)
        vals = None
        if not pattern_only:
            vals = np.ctypeslib.as_array(res.values, (nnz,)).copy() if nnz else np.zeros(0)
        return Result(br, bc, bo, vals, nnz, int(res.candidates), int(res.kept),
                      int(res.dropped), float(res.flops))
    finally:
        lib.bsmo_free_result(ctypes.byref(res))


def _result(lib, res, pattern_only=False) -> Result:
    try:
        nb, nnz = int(res.nblk), int(res.nnz)
        br = np.ctypeslib.as_array(res.blk_row, (nb,)).copy() if nb else np.zeros(0, np.int32)
        bc = np.ctypeslib.as_array(res.blk_col, (nb,)).copy() if nb else np.zeros(0, np.int32)
        bo = np.ctypeslib.as_array(res.blk_off, (nb,)).copy() if nb else np.zeros(0, np.int64)
        vals = None
        if not pattern_only:
            vals = np.ctypeslib.as_array(res.values, (nnz,)).copy() if nnz else np.zeros(0)
        return Result(br, bc, bo, vals, nnz, int(res.candidates), int(res.kept),
                      int(res.dropped), float(res.flops))
    finally:
        lib.bsmo_free_result(ctypes.byref(res))


def post_filter(M, eps: float) -> Result:
    """Blocks of M whose canonical norm is not below eps (Sec. 1 and 2: the
    filter applied after the multiplication), sorted by (row, col)."""
    lib = _load()
    h = _Held(M)
    res = _Res()
    rc = lib.bsmo_post_filter(ctypes.byref(h.s), float(eps), ctypes.byref(res))
    if rc:
        raise OracleError(rc)
    return _result(lib, res)


def add(alpha: float, A, beta: float = 0.0, C=None) -> Result:
    """C = beta*C_in + alpha*A on the union of the patterns (Algorithm 2's
    accumulation of partial C panels); beta == 0 ignores C_in."""
    lib = _load()
    ha = _Held(A)
    hc = _Held(C) if C is not None else None
    res = _Res()
    rc = lib.bsmo_add(ctypes.byref(ha.s), ctypes.byref(hc.s) if hc else None, float(alpha),
                      float(beta), ctypes.byref(res))
    if rc:
        raise OracleError(rc)
    return _result(lib, res)
