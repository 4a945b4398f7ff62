"""Plain CPU oracle for the ray-casting point-in-polygon method (test infrastructure).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference arm are the only code allowed to import this
package.  The product path (``paper_2306_04316_gb300``) never imports it and it
never imports the product: the two share only the seeded input generators.

``oracle.c`` holds the arithmetic (Method section, seven-step algorithm with
Constraint 1, exact 128-bit integer products, half-open vertex reading); this
module compiles it with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (plain gcc, -O2, pthreads)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-shared", "-fPIC",
                               "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def open_library(path: str):
    """Open a compiled copy of ``oracle.c`` and declare its entry points."""
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.oracle_classify.argtypes = [P, ctypes.c_int64, P, P, ctypes.c_int32, P, P, P,
                                    ctypes.c_int]
    lib.oracle_classify.restype = ctypes.c_int
    lib.oracle_classify_rule.argtypes = [P, ctypes.c_int64, P, P, ctypes.c_int32, P, P, ctypes.c_int, P,
                                         ctypes.c_int]
    lib.oracle_classify_rule.restype = ctypes.c_int
    lib.oracle_classify_sample.argtypes = [P, ctypes.c_int64, P, P, ctypes.c_int32, P, P,
                                           P, ctypes.c_int64, P]
    lib.oracle_classify_sample.restype = ctypes.c_int
    lib.oracle_pip_single.argtypes = [ctypes.c_int32, ctypes.c_int32, P, ctypes.c_int64]
    lib.oracle_pip_single.restype = ctypes.c_int
    lib.oracle_bbox_join.argtypes = [P, ctypes.c_int64, P, P, P, ctypes.c_int64, P, P,
                                     ctypes.c_int64]
    lib.oracle_bbox_join.restype = ctypes.c_int64
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = open_library(_LIB)
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _i32(a, shape_tail=None):
    a = np.ascontiguousarray(a, dtype=np.int32)
    if shape_tail is not None:
        a = a.reshape((-1,) + shape_tail)
    return a


def default_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def n_out_words(n_points, n_polys, cand_offsets=None) -> int:
    if cand_offsets is None:
        return n_polys * ((n_points + 31) // 32)
    c = int(cand_offsets[-1]) if n_polys > 0 else 0
    return (c + 31) // 32


def classify(points, poly_offsets, verts, cand_offsets=None, cand_ids=None, threads=None,
             lib=None):
    """Bits of every candidate (CSR) or every (polygon, point) pair (dense).

    Returns a uint32 array laid out exactly like the GPU library's ``out_bits``.
    ``lib`` selects another compiled copy (default: the built ``liboracle.so``).
    """
    lib = lib or _load()
    points = _i32(points, (2,))
    verts = _i32(verts, (2,))
    poly_offsets = _i32(poly_offsets)
    n_polys = len(poly_offsets) - 1
    if cand_offsets is not None:
        cand_offsets = _i32(cand_offsets)
        cand_ids = _i32(cand_ids)
    out = np.zeros(n_out_words(len(points), n_polys, cand_offsets), dtype=np.uint32)
    rc = lib.oracle_classify(_ptr(points), len(points), _ptr(poly_offsets), _ptr(verts), n_polys,
                             _ptr(cand_offsets), _ptr(cand_ids), _ptr(out),
                             int(threads or default_threads()))
    if rc != 0:
        raise ValueError("oracle_classify rejected its arguments")
    return out


def classify_rule(points, poly_offsets, verts, rule, cand_offsets=None, cand_ids=None, threads=None):
    """Like ``classify`` with the paper's printed rule: 1 = Algorithm 1, 2 = Algorithm 2
    (0 = the half-open rule of ``classify``)."""
    lib = _load()
    points = _i32(points, (2,))
    verts = _i32(verts, (2,))
    poly_offsets = _i32(poly_offsets)
    n_polys = len(poly_offsets) - 1
    if cand_offsets is not None:
        cand_offsets = _i32(cand_offsets)
        cand_ids = _i32(cand_ids)
    out = np.zeros(n_out_words(len(points), n_polys, cand_offsets), dtype=np.uint32)
    rc = lib.oracle_classify_rule(_ptr(points), len(points), _ptr(poly_offsets), _ptr(verts), n_polys,
                                  _ptr(cand_offsets), _ptr(cand_ids), int(rule), _ptr(out),
                                  int(threads or default_threads()))
    if rc != 0:
        raise ValueError("oracle_classify_rule rejected its arguments")
    return out


def quantize(values, scale=1e7):
    """float64 -> int32 fixed point by the plain definition: rint(v * scale) with the product
    rounded once in float64 and ties to even; (out, status) with status bit 1 for NaN and bit 2
    for a result outside int32 (those values become 0)."""
    v = np.asarray(values, dtype=np.float64)
    with np.errstate(invalid="ignore", over="ignore"):
        q = np.rint(v * np.float64(scale))
    nan = np.isnan(q)
    out_of_range = ~nan & ((q < -2.0**31) | (q > 2.0**31 - 1))
    out = np.where(nan | out_of_range, 0, np.nan_to_num(q)).astype(np.int64).astype(np.int32)
    status = (1 if nan.any() else 0) | (2 if out_of_range.any() else 0)
    return out, status


def classify_sample(points, poly_offsets, verts, sample, cand_offsets=None, cand_ids=None):
    """0/1 per listed bit index (candidate index, or k*32*W + j in dense mode)."""
    lib = _load()
    points = _i32(points, (2,))
    verts = _i32(verts, (2,))
    poly_offsets = _i32(poly_offsets)
    n_polys = len(poly_offsets) - 1
    if cand_offsets is not None:
        cand_offsets = _i32(cand_offsets)
        cand_ids = _i32(cand_ids)
    sample = np.ascontiguousarray(sample, dtype=np.int64)
    out = np.zeros(len(sample), dtype=np.uint8)
    rc = lib.oracle_classify_sample(_ptr(points), len(points), _ptr(poly_offsets), _ptr(verts),
                                    n_polys, _ptr(cand_offsets), _ptr(cand_ids), _ptr(sample),
                                    len(sample), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_classify_sample: index out of range")
    return out


def pip_single(px: int, py: int, verts) -> int:
    """Inside bit of one point against one polygon (vertices as [(x, y), ...])."""
    lib = _load()
    v = _i32(verts, (2,)) if len(verts) else np.zeros((0, 2), np.int32)
    return int(lib.oracle_pip_single(int(px), int(py), _ptr(v), len(v)))


def bbox_join(points, poly_offsets, verts, polys):
    """Closed-bbox candidate lists (ascending point ids) for the listed polygons."""
    lib = _load()
    points = _i32(points, (2,))
    verts = _i32(verts, (2,))
    poly_offsets = _i32(poly_offsets)
    polys = _i32(polys)
    counts = np.zeros(len(polys), dtype=np.int64)
    total = lib.oracle_bbox_join(_ptr(points), len(points), _ptr(poly_offsets), _ptr(verts),
                                 _ptr(polys), len(polys), _ptr(counts), None, 0)
    ids = np.zeros(max(int(total), 1), dtype=np.int32)
    total2 = lib.oracle_bbox_join(_ptr(points), len(points), _ptr(poly_offsets), _ptr(verts),
                                  _ptr(polys), len(polys), _ptr(counts), _ptr(ids), len(ids))
    if total2 != total:
        raise RuntimeError("oracle_bbox_join: inconsistent sizes")
    return counts, ids[:total]


def unpack_bits(words, n_bits: int) -> np.ndarray:
    """uint32 words (LSB first) -> uint8 array of n_bits 0/1 values."""
    b = np.unpackbits(np.ascontiguousarray(words, dtype="<u4").view(np.uint8), bitorder="little")
    return b[:n_bits]
