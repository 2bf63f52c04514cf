"""CPU oracle for the fixed-radius nearest-neighbour graph build.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only users.  The CUDA library and its Python binding
never import this package, and it imports nothing from them.

The arithmetic lives in ``frnn_oracle.c`` (plain brute force over all pairs,
float32 squared distances summed in dimension order, edge iff d2 <= fl32(r*r),
rows capped at the k smallest (d2, j) pairs).  Paper: Sec. 2 (graph of points
within a constant radius of each other in the embedded space), Sec. 3.4 (the
FRNN problem), Sec. 3.1 (exact kNN followed by a radius cut).  This module
only marshals numpy arrays, builds the row offsets from the degrees and
compiles the C file on first use.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "frnn_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle_frnn.so")
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_f32p = ctypes.POINTER(ctypes.c_float)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                               "-std=c11", "-Wall", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _configure(lib):
    lib.fo_degree.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int, ctypes.c_float, _i64p,
                              ctypes.c_int64, _i64p]
    lib.fo_fill.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_int,
                            _i64p, ctypes.c_int64, _i64p, _i32p, _f32p]
    lib.fo_degree_grid.argtypes = [_i32p, ctypes.c_int64, ctypes.c_int, ctypes.c_int64, _i64p,
                                   ctypes.c_int64, _i64p]
    lib.fo_fill_grid.argtypes = [_i32p, ctypes.c_int64, ctypes.c_int, ctypes.c_int64,
                                 ctypes.c_int, _i64p, ctypes.c_int64, _i64p, _i32p, _i64p]
    lib.fo_num_threads.argtypes = []
    lib.fo_components.argtypes = [_i64p, _i32p, _f32p, ctypes.c_float, ctypes.c_int64, _i32p]
    lib.fo_components.restype = ctypes.c_int
    for f in (lib.fo_degree, lib.fo_fill, lib.fo_degree_grid, lib.fo_fill_grid, lib.fo_num_threads):
        f.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _configure(ctypes.CDLL(build()))
    return _lib


def use_library(path):
    """Point this module at another build of the oracle source (returns the
    previous handle; pass it back to restore).  The mutation tests use this to
    check that the pins reject a deliberately broken copy."""
    global _lib
    prev = _lib
    _lib = path if not isinstance(path, str) else _configure(ctypes.CDLL(path))
    return prev


def _ptr(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _queries(n, queries):
    if queries is None:
        return None, n
    q = np.ascontiguousarray(queries, dtype=np.int64)
    return q, q.shape[0]


def num_threads() -> int:
    """OpenMP threads the oracle runs on (OMP_NUM_THREADS, else all cores)."""
    return int(_load().fo_num_threads())


def degree(x: np.ndarray, r: float, queries=None) -> np.ndarray:
    """|S_i| (uncapped) for each query (all points if queries is None)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    n, d = x.shape
    q, nq = _queries(n, queries)
    deg = np.zeros(nq, dtype=np.int64)
    if nq and _load().fo_degree(_ptr(x, _f32p), n, d, float(r), _ptr(q, _i64p), nq,
                                _ptr(deg, _i64p)) != 0:
        raise ValueError("oracle: bad argument")
    return deg


def radius_graph(x: np.ndarray, r: float, k: int, queries=None, with_d2: bool = False):
    """Rows of the capped FRNN graph, CSR form.

    Returns (row_ptr int64 [nq+1], col int32 [E]) or, with ``with_d2``,
    (row_ptr, col, d2 float32 [E]).  Row qi belongs to point queries[qi]
    (or qi); entries are sorted by (d2, j); k <= 0 means no cap."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    n, d = x.shape
    q, nq = _queries(n, queries)
    deg = degree(x, r, q)
    cnt = np.minimum(deg, k) if k > 0 else deg
    row_ptr = np.zeros(nq + 1, dtype=np.int64)
    np.cumsum(cnt, out=row_ptr[1:])
    e = int(row_ptr[-1])
    col = np.zeros(max(e, 1), dtype=np.int32)
    d2 = np.zeros(max(e, 1), dtype=np.float32) if with_d2 else None
    if nq and _load().fo_fill(_ptr(x, _f32p), n, d, float(r), int(k), _ptr(q, _i64p), nq,
                              _ptr(row_ptr, _i64p), _ptr(col, _i32p), _ptr(d2, _f32p)) != 0:
        raise ValueError("oracle: bad argument")
    if with_d2:
        return row_ptr, col[:e], d2[:e]
    return row_ptr, col[:e]


def knn_graph(x: np.ndarray, k: int, queries=None, with_d2: bool = False):
    """Rows of the exact k-nearest-neighbour graph (no radius cut), CSR form:
    row i holds the min(k, n - 1) points j != i smallest by (d2, j), in that
    order.  This is the radius graph with an unbounded radius: every other
    point is in S_i, and the cap keeps the k nearest.  Paper: Sec. 3.1 (exact
    kNN search over the embedded points, Faiss IndexFlat), here without the
    radius cut that follows it there."""
    if k < 1:
        raise ValueError("k must be >= 1")
    return radius_graph(x, float("inf"), k, queries=queries, with_d2=with_d2)


def grid_threshold(r: float) -> int:
    """floor(r2 * 65536) for r2 = fl32(r * r), in exact rational arithmetic.

    On the 1/256 grid a float32 squared distance equals q / 65536 with q an
    integer, so d2 <= r2 holds exactly when q <= floor(r2 * 65536)."""
    r32 = np.float32(r)
    r2 = np.float32(r32 * r32)
    return math.floor(Fraction(float(r2)) * 65536)


def to_grid_ints(x: np.ndarray) -> np.ndarray:
    """Integer coordinates m = 256 x of on-grid float32 points (checked)."""
    m = np.asarray(x, dtype=np.float64) * 256.0
    mi = np.rint(m)
    if not np.all(mi == m):
        raise ValueError("points are not on the 1/256 grid")
    return np.ascontiguousarray(mi.astype(np.int32))


def radius_graph_grid(m: np.ndarray, thr: int, k: int, queries=None, with_q: bool = False):
    """Integer-grid oracle: edge iff sum (m_i - m_j)^2 <= thr, rows by (q, j)."""
    m = np.ascontiguousarray(m, dtype=np.int32)
    n, d = m.shape
    q, nq = _queries(n, queries)
    deg = np.zeros(nq, dtype=np.int64)
    lib = _load()
    if nq and lib.fo_degree_grid(_ptr(m, _i32p), n, d, int(thr), _ptr(q, _i64p), nq,
                                 _ptr(deg, _i64p)) != 0:
        raise ValueError("oracle: bad argument")
    cnt = np.minimum(deg, k) if k > 0 else deg
    row_ptr = np.zeros(nq + 1, dtype=np.int64)
    np.cumsum(cnt, out=row_ptr[1:])
    e = int(row_ptr[-1])
    col = np.zeros(max(e, 1), dtype=np.int32)
    qv = np.zeros(max(e, 1), dtype=np.int64) if with_q else None
    if nq and lib.fo_fill_grid(_ptr(m, _i32p), n, d, int(thr), int(k), _ptr(q, _i64p), nq,
                               _ptr(row_ptr, _i64p), _ptr(col, _i32p), _ptr(qv, _i64p)) != 0:
        raise ValueError("oracle: bad argument")
    if with_q:
        return row_ptr, col[:e], qv[:e]
    return row_ptr, col[:e]


def components(row_ptr: np.ndarray, col: np.ndarray, w=None, w_max: float = float("inf")) -> np.ndarray:
    """Weakly connected components of a CSR graph (edges with w <= w_max,
    direction ignored): each point's label is the smallest index of its
    component.  Paper: Sec. 2 (track candidates from a score cut and weakly
    connected components), Sec. 3.2."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    c = np.ascontiguousarray(col, dtype=np.int32)
    wt = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
    n = rp.size - 1
    labels = np.zeros(max(n, 1), dtype=np.int32)
    if n and _load().fo_components(_ptr(rp, _i64p), _ptr(c, _i32p), _ptr(wt, _f32p), float(w_max), n,
                                   _ptr(labels, _i32p)) != 0:
        raise ValueError("oracle: bad argument")
    return labels[:n]


def track_labels(x: np.ndarray, r: float, k: int, d2_max: float) -> np.ndarray:
    """Labels of the capped radius graph's edges with d2 <= fl32(d2_max)."""
    rp, col, d2 = radius_graph(x, r, k, with_d2=True)
    return components(rp, col, d2, float(np.float32(d2_max)))
