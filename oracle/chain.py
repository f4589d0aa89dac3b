"""ctypes wrapper of the C oracle (test infrastructure).

`evaluate(ohin, query)` returns the canonical CSR (row_ptr int64, col int32, val uint64)
of A_m = M_1 A_1 M_2 ... A_{n-1} M_n (Sec. 2, Problem 1 and the constrained adjacency
after it), computed left to right by the plain single-threaded code in chain.c.
"""
import ctypes as C

import numpy as np

from . import build as _build


class OracleOverflow(ArithmeticError):
    """A count does not fit in uint64."""


class _CSR(C.Structure):
    _fields_ = [("nrows", C.c_int64), ("ncols", C.c_int64),
                ("rp", C.c_void_p), ("ci", C.c_void_p), ("val", C.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        P = C.POINTER
        L.orc_spgemm.argtypes = [P(_CSR), P(_CSR), C.c_void_p, C.c_void_p, C.c_void_p,
                                 P(C.c_void_p), P(C.c_void_p), P(C.c_void_p), P(C.c_int64)]
        L.orc_chain.argtypes = [C.c_int, P(_CSR), P(C.c_void_p), P(C.c_void_p), P(C.c_void_p),
                                P(C.c_void_p), P(C.c_int64)]
        L.orc_rowsum.argtypes = [C.c_int, P(_CSR), P(C.c_void_p), C.c_void_p]
        L.orc_colsum.argtypes = [C.c_int, P(_CSR), P(C.c_void_p), C.c_void_p]
        L.orc_free.argtypes = [C.c_void_p]
        for f in (L.orc_spgemm, L.orc_chain, L.orc_rowsum, L.orc_colsum):
            f.restype = C.c_int
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _csr(f, keep):
    rp, ci, nr, nc = f[:4]
    val = f[4] if len(f) > 4 else None
    rp = np.ascontiguousarray(rp, np.int64)
    ci = np.ascontiguousarray(ci, np.int32)
    val = None if val is None else np.ascontiguousarray(val, np.uint64)
    keep += [rp, ci, val]
    return _CSR(int(nr), int(nc), _ptr(rp), _ptr(ci), _ptr(val))


def _mask(m, keep):
    if m is None:
        return None
    m = np.ascontiguousarray(m, np.uint8)
    keep.append(m)
    return m.ctypes.data


def _take(rp, ci, val, nnz, nrows):
    L = lib()
    try:
        out_rp = np.ctypeslib.as_array((C.c_int64 * (nrows + 1)).from_address(rp.value)).copy()
        if nnz:
            out_ci = np.ctypeslib.as_array((C.c_int32 * nnz).from_address(ci.value)).copy()
            out_val = np.ctypeslib.as_array((C.c_uint64 * nnz).from_address(val.value)).copy()
        else:
            out_ci = np.zeros(0, np.int32)
            out_val = np.zeros(0, np.uint64)
    finally:
        for p in (rp, ci, val):
            if p.value:
                L.orc_free(p)
    return out_rp, out_ci, out_val


def _check(rc):
    if rc == -5:
        raise OracleOverflow("a path count exceeds 2^64-1")
    if rc != 0:
        raise RuntimeError(f"oracle error {rc}")


def spgemm(X, Y, rmask=None, kmask=None, cmask=None):
    """diag(rmask) X diag(kmask) Y diag(cmask); X, Y = (rp, ci, nrows, ncols[, val])."""
    keep = []
    cx, cy = _csr(X, keep), _csr(Y, keep)
    rp, ci, val, nnz = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_int64()
    _check(lib().orc_spgemm(C.byref(cx), C.byref(cy), _mask(rmask, keep), _mask(kmask, keep),
                            _mask(cmask, keep), C.byref(rp), C.byref(ci), C.byref(val), C.byref(nnz)))
    return _take(rp, ci, val, nnz.value, int(X[2]))


def _chain_args(factors, masks, keep):
    arr = (_CSR * len(factors))(*[_csr(f, keep) for f in factors])
    marr = (C.c_void_p * len(masks))(*[_mask(m, keep) for m in masks])
    return arr, marr


def chain(factors, masks):
    """A_m for factors (rp, ci, nrows, ncols) and per-position masks, left to right."""
    assert len(masks) == len(factors) + 1
    keep = []
    arr, marr = _chain_args(factors, masks, keep)
    rp, ci, val, nnz = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_int64()
    _check(lib().orc_chain(len(factors), arr, marr, C.byref(rp), C.byref(ci), C.byref(val),
                           C.byref(nnz)))
    return _take(rp, ci, val, nnz.value, int(factors[0][2]))


def rowsum(factors, masks):
    keep = []
    arr, marr = _chain_args(factors, masks, keep)
    out = np.zeros(int(factors[0][2]), np.uint64)
    _check(lib().orc_rowsum(len(factors), arr, marr, out.ctypes.data))
    return out


def colsum(factors, masks):
    keep = []
    arr, marr = _chain_args(factors, masks, keep)
    out = np.zeros(int(factors[-1][3]), np.uint64)
    _check(lib().orc_colsum(len(factors), arr, marr, out.ctypes.data))
    return out


def evaluate(ohin, query):
    """Canonical CSR of the query's result on an oracle HIN."""
    factors, masks = ohin.query(query)
    return chain(factors, masks)
