"""Oracle (test infrastructure, not product code) for the contraction itself.

Section 1 ("Tensor Notation") defines the operation: in ``C_abc = A_ai B_ibc``
every entry ``C[a,b,c]`` is the sum over ``i`` of ``A[a,i] * B[i,b,c]``.
Indices that appear in both inputs are contracted; indices that appear in one
input (and therefore in C) are free.  Tensors are stored Fortran-style, first
index fastest.  This module restates that definition in FP64:

    C[f] = beta * C[f] + alpha * sum_k A[f_A, k] * B[f_B, k]

by calling the plain nested-loop C code in ``contraction.c`` (built by
``oracle/build.py``).  Operands are flat FP64 numpy arrays addressed through
element strides; ``None`` strides mean Fortran-contiguous.

Conventions shared with the library's public interface (the paper fixes
none of them): the spec string is ``"C=A,B"`` with one letter per index;
``extents`` gives one extent per distinct letter in order of first appearance
in the spec string, left to right; ``strides`` concatenates the element
strides of the C modes, then the A modes, then the B modes.

Only ``tests/``, the smoke check and the benchmark's CPU-baseline leg may
import this module.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        i64p = ctypes.POINTER(ctypes.c_int64)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_contract.argtypes = [
            ctypes.c_int, i64p, i64p, i64p, i64p,
            ctypes.c_int, i64p, i64p, i64p,
            ctypes.c_double, dp, dp, ctypes.c_double, dp,
            ctypes.c_int64, ctypes.c_int64, ctypes.c_int]
        lib.oracle_contract.restype = ctypes.c_int
        lib.oracle_contract_points.argtypes = [
            ctypes.c_int, i64p, i64p,
            ctypes.c_int, i64p, i64p, i64p, dp, dp,
            ctypes.c_int64, i64p, dp, ctypes.c_int]
        lib.oracle_contract_points.restype = ctypes.c_int
        lib.oracle_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def parse_spec(spec):
    """Split ``"abc=ai,ibc"`` into the mode strings of C, A and B."""
    s = spec.replace(" ", "")
    lhs, rhs = s.split("=")
    a, b = rhs.split(",")
    return lhs, a, b


def index_order(spec):
    """Distinct index letters in order of first appearance in the spec."""
    c, a, b = parse_spec(spec)
    seen = []
    for ch in c + a + b:
        if ch not in seen:
            seen.append(ch)
    return seen


def fortran_strides(modes, ext):
    """Section 1 storage: first index fastest, contiguous."""
    out, s = [], 1
    for m in modes:
        out.append(s)
        s *= ext[m]
    return out


def operand_layout(spec, extents, strides=None):
    """Per-operand dict index -> element stride, and the extent dict."""
    c, a, b = parse_spec(spec)
    order = index_order(spec)
    ext = dict(zip(order, [int(e) for e in extents]))
    if strides is None:
        sc = fortran_strides(c, ext)
        sa = fortran_strides(a, ext)
        sb = fortran_strides(b, ext)
    else:
        strides = [int(x) for x in strides]
        sc = strides[:len(c)]
        sa = strides[len(c):len(c) + len(a)]
        sb = strides[len(c) + len(a):len(c) + len(a) + len(b)]
    return ext, dict(zip(c, sc)), dict(zip(a, sa)), dict(zip(b, sb))


def required_length(modes, ext, strides_by_index):
    """Smallest flat buffer length that holds every element of the operand."""
    if not modes:
        return 1
    return 1 + sum((ext[m] - 1) * strides_by_index[m] for m in modes)


def _arrays(spec, extents, strides):
    c, a, b = parse_spec(spec)
    ext, sc, sa, sb = operand_layout(spec, extents, strides)
    contracted = [m for m in a if m in b and m not in c]
    free = list(c) if c else []
    ext_f = [ext[m] for m in free]
    sC_f = [sc[m] for m in free]
    sA_f = [sa.get(m, 0) for m in free]
    sB_f = [sb.get(m, 0) for m in free]
    ext_k = [ext[m] for m in contracted]
    sA_k = [sa[m] for m in contracted]
    sB_k = [sb[m] for m in contracted]
    if not free:  # scalar C: one mode of extent 1
        ext_f, sC_f, sA_f, sB_f = [1], [0], [0], [0]
    return ext_f, sC_f, sA_f, sB_f, ext_k, sA_k, sB_k


def _i64(v):
    arr = np.ascontiguousarray(np.asarray(v, dtype=np.int64))
    return arr, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _dbl(x):
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def contract(spec, extents, A, B, C=None, alpha=1.0, beta=0.0, strides=None,
             threads=1, outer_range=None):
    """Full contraction in FP64.  A, B (and C) are flat float64 arrays.

    Returns the C buffer (a new zero buffer when C is None).  ``outer_range``
    restricts the computation to a slab ``[lo, hi)`` of the last C mode.
    """
    lib = _load()
    c, a, b = parse_spec(spec)
    ext, sc, sa, sb = operand_layout(spec, extents, strides)
    A = np.ascontiguousarray(A, dtype=np.float64).ravel()
    B = np.ascontiguousarray(B, dtype=np.float64).ravel()
    assert A.size >= required_length(a, ext, sa)
    assert B.size >= required_length(b, ext, sb)
    if C is None:
        C = np.zeros(required_length(c, ext, sc), dtype=np.float64)
        beta = 0.0
    else:
        assert C.dtype == np.float64 and C.flags.c_contiguous and C.ndim == 1
        assert C.size >= required_length(c, ext, sc)
    ext_f, sC_f, sA_f, sB_f, ext_k, sA_k, sB_k = _arrays(spec, extents, strides)
    lo, hi = (0, ext_f[-1]) if outer_range is None else outer_range
    keep = [_i64(v) for v in (ext_f, sC_f, sA_f, sB_f, ext_k, sA_k, sB_k)]
    rc = lib.oracle_contract(len(ext_f), keep[0][1], keep[1][1], keep[2][1],
                             keep[3][1], len(ext_k), keep[4][1], keep[5][1],
                             keep[6][1], float(alpha), _dbl(A), _dbl(B),
                             float(beta), _dbl(C), int(lo), int(hi),
                             int(threads))
    if rc != 0:
        raise ValueError("oracle_contract rejected its arguments")
    return C


def contract_points(spec, extents, A, B, points, strides=None, threads=1):
    """The contraction sum at chosen C multi-indices (rows of ``points``)."""
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.float64).ravel()
    B = np.ascontiguousarray(B, dtype=np.float64).ravel()
    ext_f, _, sA_f, sB_f, ext_k, sA_k, sB_k = _arrays(spec, extents, strides)
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.int64))
    nf = len(parse_spec(spec)[0])
    if nf == 0:
        pts = np.zeros((pts.shape[0] if pts.ndim == 2 else 1, 1), np.int64)
        nf = 1
    pts = pts.reshape(-1, nf)
    out = np.zeros(pts.shape[0], dtype=np.float64)
    keep = [_i64(v) for v in (sA_f, sB_f, ext_k, sA_k, sB_k)]
    rc = lib.oracle_contract_points(
        nf, keep[0][1], keep[1][1], len(ext_k), keep[2][1], keep[3][1],
        keep[4][1], _dbl(A), _dbl(B), pts.shape[0],
        pts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dbl(out),
        int(threads))
    if rc != 0:
        raise ValueError("oracle_contract_points rejected its arguments")
    return out


def max_threads():
    return int(_load().oracle_max_threads())


def flops(spec, extents):
    """2 * product of all extents: one multiply and one add per term."""
    n = 2
    for e in extents:
        n *= int(e)
    return n
