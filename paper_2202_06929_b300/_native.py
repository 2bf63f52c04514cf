"""ctypes binding of libfrnn (the C ABI in include/frnn.h).

Argument marshalling only: every step of the graph build runs in the CUDA
kernels of libfrnn.so.  PyTorch supplies device memory and streams; results
are exposed as zero-copy torch views of the plan-owned device buffers.
There is no CPU fallback: if the library cannot be loaded this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

FRNN_OK = 0
FRNN_ERR_INVALID_ARG = 1
FRNN_ERR_CUDA = 2
FRNN_ERR_OOM = 3
FRNN_ERR_NONFINITE_INPUT = 4
FRNN_ERR_TIMEOUT = 5
FRNN_ERR_OVERFLOW = 6
FRNN_ERR_CAPACITY = 7
FRNN_ERR_CHECK = 8

FRNN_NO_CAP = 0   # k = FRNN_NO_CAP keeps every row whole (rows over 32 neighbours unsorted)
FRNN_EMIT_D2 = 0x1
FRNN_USE_GRAPH = 0x2
FRNN_AUTOTUNE = 0x4
FRNN_DEBUG = 0x8

# Debug checks of a build's output (frnn_check_last_build), in pipeline order.
CHECKS = ("none", "event_offsets", "cell_table", "scatter", "row_ptr", "column", "radius", "d2", "order",
          "complete")

# Every function the header declares (checked by the tests against the .so).
ABI_FUNCTIONS = (
    "frnn_plan_create", "frnn_plan_destroy", "frnn_plan_set_tuning", "frnn_plan_get_tuning",
    "frnn_build_graph", "frnn_build_graph_batched", "frnn_build_graph_host", "frnn_build_graph_profiled",
    "frnn_get_last_status", "frnn_status_string", "frnn_version", "frnn_build_graph_noalloc",
    "frnn_plan_bytes", "frnn_server_create", "frnn_server_reserved_bytes", "frnn_server_submit",
    "frnn_server_wait", "frnn_server_run_trace", "frnn_server_destroy", "frnn_plan_autotune",
    "frnn_label_components", "frnn_edge_features", "frnn_knn_graph_batched",
    "frnn_plan_test_stall_next_build", "frnn_server_poll", "frnn_server_get_stats", "frnn_plan_tuning_for",
    "frnn_check_last_build", "frnn_get_last_check",
)


class frnn_plan_params(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("d_max", ctypes.c_int), ("n_max", ctypes.c_int64),
                ("events_max", ctypes.c_int), ("k_max_cap", ctypes.c_int),
                ("edge_capacity", ctypes.c_int64), ("cells_per_point", ctypes.c_int),
                ("flags", ctypes.c_uint32), ("hit_capacity", ctypes.c_int64),
                ("mem_budget_bytes", ctypes.c_uint64)]


class frnn_csr(ctypes.Structure):
    _fields_ = [("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("d2", ctypes.c_void_p),
                ("edge_off", ctypes.c_void_p), ("n_edges", ctypes.c_void_p),
                ("n_events", ctypes.c_int), ("n_total", ctypes.c_int64)]


class frnn_tuning(ctypes.Structure):
    _fields_ = [("g_max", ctypes.c_int), ("cell_scale", ctypes.c_float), ("walk", ctypes.c_int)]


FRNN_WALK_AUTO, FRNN_WALK_CANDIDATES, FRNN_WALK_QUERIES = 0, 1, 2


class frnn_server_params(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("d", ctypes.c_int), ("r", ctypes.c_float), ("k", ctypes.c_int),
                ("batch_points", ctypes.c_int64), ("batch_events", ctypes.c_int), ("slots", ctypes.c_int),
                ("edges_per_point", ctypes.c_int), ("mem_budget_bytes", ctypes.c_uint64),
                ("n_devices", ctypes.c_int), ("devices", ctypes.POINTER(ctypes.c_int))]


class frnn_server_stats(ctypes.Structure):
    _fields_ = [("batches", ctypes.c_uint64), ("spill_batches", ctypes.c_uint64), ("readmitted", ctypes.c_uint64),
                ("requests_done", ctypes.c_uint64), ("max_queue", ctypes.c_uint64),
                ("regular_edge_capacity", ctypes.c_uint64), ("spill_edge_capacity", ctypes.c_uint64)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Load libfrnn.so (building it first if the in-tree copy is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    if not os.path.exists(path):
        raise ImportError(f"libfrnn.so not found at {path}")
    lib = ctypes.CDLL(path)
    vp, i64, i32, f32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_float
    P = ctypes.POINTER
    lib.frnn_plan_create.argtypes = [P(vp), P(frnn_plan_params)]
    lib.frnn_plan_destroy.argtypes = [vp]
    lib.frnn_plan_set_tuning.argtypes = [vp, P(frnn_tuning)]
    lib.frnn_plan_get_tuning.argtypes = [vp, P(frnn_tuning)]
    lib.frnn_build_graph.argtypes = [vp, vp, i64, i32, f32, i32, vp, P(frnn_csr)]
    lib.frnn_build_graph_batched.argtypes = [vp, vp, P(ctypes.c_int64), i32, i32, f32, i32, vp, P(frnn_csr)]
    lib.frnn_knn_graph_batched.argtypes = [vp, vp, P(ctypes.c_int64), i32, i32, i32, vp, P(frnn_csr)]
    lib.frnn_build_graph_host.argtypes = [vp, vp, P(ctypes.c_int64), i32, i32, f32, i32, vp, vp, i64,
                                          vp, P(ctypes.c_int64), vp]
    lib.frnn_build_graph_profiled.argtypes = [vp, vp, P(ctypes.c_int64), i32, i32, f32, i32, vp,
                                              P(frnn_csr), P(ctypes.c_float), i32]
    lib.frnn_plan_bytes.argtypes = [P(frnn_plan_params), P(ctypes.c_uint64)]
    lib.frnn_plan_autotune.argtypes = [vp, vp, P(ctypes.c_int64), i32, i32, f32, i32, vp, P(frnn_tuning),
                                       P(ctypes.c_float)]
    lib.frnn_server_create.argtypes = [P(vp), P(frnn_server_params)]
    lib.frnn_server_reserved_bytes.argtypes = [vp, P(ctypes.c_uint64)]
    lib.frnn_server_submit.argtypes = [vp, vp, i64, P(ctypes.c_uint64)]
    lib.frnn_server_wait.argtypes = [vp, ctypes.c_uint64, vp, vp, i64, P(ctypes.c_int64), P(ctypes.c_double)]
    lib.frnn_server_poll.argtypes = [vp, ctypes.c_uint64, P(ctypes.c_int)]
    lib.frnn_plan_tuning_for.argtypes = [vp, P(ctypes.c_int64), i32, i32, f32, i32, P(frnn_tuning), P(ctypes.c_int)]
    lib.frnn_server_get_stats.argtypes = [vp, P(frnn_server_stats)]
    lib.frnn_server_run_trace.argtypes = [vp, vp, P(ctypes.c_int64), P(ctypes.c_int64), P(ctypes.c_double), i32,
                                          P(ctypes.c_double), P(ctypes.c_int64), P(ctypes.c_double)]
    lib.frnn_server_destroy.argtypes = [vp]
    lib.frnn_build_graph_noalloc.argtypes = [vp, i64, i32, f32, i32, vp, vp, i64, vp, vp]
    lib.frnn_label_components.argtypes = [vp, f32, vp, vp]
    lib.frnn_edge_features.argtypes = [vp, vp, i64, i64, vp, vp]
    lib.frnn_get_last_status.argtypes = [vp, vp]
    lib.frnn_plan_test_stall_next_build.argtypes = [vp]
    lib.frnn_check_last_build.argtypes = [vp, vp]
    lib.frnn_get_last_check.argtypes = [vp, vp, P(ctypes.c_int), P(ctypes.c_int64)]
    lib.frnn_status_string.argtypes = [i32]
    lib.frnn_status_string.restype = ctypes.c_char_p
    lib.frnn_version.argtypes = []
    for name in ABI_FUNCTIONS:
        if name != "frnn_status_string":
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


class FrnnError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = int(status)
        msg = load().frnn_status_string(self.status).decode()
        super().__init__(f"{where}: {msg} (status {self.status})" if where else msg)


def _check(rc: int, where: str) -> None:
    if rc != FRNN_OK:
        raise FrnnError(rc, where)


def status_string(status: int) -> str:
    return load().frnn_status_string(int(status)).decode()


def version() -> int:
    return int(load().frnn_version())


def _stream_handle(stream) -> int | None:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) or None


class _DevArray:
    """__cuda_array_interface__ wrapper for a plan-owned device buffer."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {
            "shape": (int(n),), "typestr": typestr, "data": (int(ptr) if n else 0, False),
            "version": 3, "strides": None,
        }


def _view(ptr, n, dtype, device):
    import torch
    if n == 0:
        return torch.zeros(0, dtype=dtype, device=device)
    typestr = {torch.int32: "<i4", torch.float32: "<f4"}[dtype]
    return torch.as_tensor(_DevArray(ptr, n, typestr), device=device)


class Csr:
    """Result of a build: device views into plan-owned buffers.

    Valid until the next build on the same plan (clone to keep)."""

    def __init__(self, c: frnn_csr, device, ev_off: np.ndarray, edge_capacity: int):
        self._c = c
        self.device = device
        self.edge_capacity = int(edge_capacity)
        self.n_events = int(c.n_events)
        self.n_total = int(c.n_total)
        self.ev_off = ev_off
        self.row_ptr = _view(c.row_ptr, self.n_total + 1, _torch().int32, device)
        self.edge_off = _view(c.edge_off, self.n_events + 1, _torch().int32, device)

    def n_edges(self) -> int:
        """Total edges (reads one device word: synchronises the stream's work)."""
        return int(self.edge_off[-1].item())

    def col(self, n_edges: int | None = None):
        """col[0 .. n_edges) (at most the plan's edge capacity: after an
        overflow the edges that did not fit were never written)."""
        n = self.n_edges() if n_edges is None else n_edges
        return _view(self._c.col, min(n, self.edge_capacity), _torch().int32, self.device)

    def d2(self, n_edges: int | None = None):
        if not self._c.d2:
            return None
        n = self.n_edges() if n_edges is None else n_edges
        return _view(self._c.d2, min(n, self.edge_capacity), _torch().float32, self.device)

    def to_host(self) -> dict:
        """Copy the whole CSR to numpy (row_ptr, col, edge_off, and d2 if emitted)."""
        edge_off = self.edge_off.cpu().numpy()
        e = min(int(edge_off[-1]), self.edge_capacity)
        out = dict(row_ptr=self.row_ptr.cpu().numpy(), col=self.col(e).cpu().numpy(),
                   edge_off=edge_off)
        d2 = self.d2(e)
        if d2 is not None:
            out["d2"] = d2.cpu().numpy()
        return out

    def event_rows(self, host: dict, b: int):
        """(row_ptr, col) of event b, local to the event, from a to_host() dict."""
        lo, hi = int(self.ev_off[b]), int(self.ev_off[b + 1])
        e0 = int(host["edge_off"][b])
        rp = host["row_ptr"][lo:hi + 1].astype(np.int64) - e0
        col = host["col"][e0:e0 + int(rp[-1])]
        return rp, col


def _torch():
    import torch
    return torch


class Plan:
    """Owner of all device memory of the graph build (frnn_plan)."""

    def __init__(self, n_max: int, d_max: int, k_max_cap: int, events_max: int = 1,
                 edge_capacity: int = 0, cells_per_point: int = 0, emit_d2: bool = False,
                 use_graph: bool = False, device: int = 0, autotune: bool = False, hit_capacity: int = 0,
                 debug: bool = False, mem_budget_bytes: int = 0):
        lib = load()
        prm = frnn_plan_params(device=device, d_max=d_max, n_max=n_max, events_max=events_max,
                               k_max_cap=k_max_cap, edge_capacity=edge_capacity,
                               cells_per_point=cells_per_point, hit_capacity=hit_capacity,
                               mem_budget_bytes=mem_budget_bytes,
                               flags=((FRNN_EMIT_D2 if emit_d2 else 0) | (FRNN_USE_GRAPH if use_graph else 0)
                                      | (FRNN_AUTOTUNE if autotune else 0) | (FRNN_DEBUG if debug else 0)))
        h = ctypes.c_void_p()
        _check(lib.frnn_plan_create(ctypes.byref(h), ctypes.byref(prm)), "frnn_plan_create")
        self._h = h
        self.device = _torch().device("cuda", device)
        self.params = prm
        self.edge_capacity = int(edge_capacity) if edge_capacity else int(n_max) * int(k_max_cap)
        self._last_n = 0

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            load().frnn_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self) -> int:
        return int(self._h.value or 0)

    def set_tuning(self, g_max: int = 0, cell_scale: float = 0.0, walk: int = FRNN_WALK_AUTO) -> None:
        t = frnn_tuning(g_max=g_max, cell_scale=cell_scale, walk=walk)
        _check(load().frnn_plan_set_tuning(self._h, ctypes.byref(t)), "frnn_plan_set_tuning")

    def get_tuning(self) -> tuple[int, float, int]:
        """(g_max, cell_scale, walk) used by the next builds."""
        t = frnn_tuning()
        _check(load().frnn_plan_get_tuning(self._h, ctypes.byref(t)), "frnn_plan_get_tuning")
        return int(t.g_max), float(t.cell_scale), int(t.walk)

    def tuning_for(self, ev_off, d: int, r: float, k: int) -> tuple[int, float, int, bool]:
        """(g_max, cell_scale, walk, cached): the tuning a build with these
        arguments would use, and whether it is an autotuned entry."""
        off = np.ascontiguousarray(ev_off, dtype=np.int64)
        t = frnn_tuning()
        c = ctypes.c_int(0)
        _check(load().frnn_plan_tuning_for(self._h, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                           off.size - 1, int(d), float(r), int(k), ctypes.byref(t),
                                           ctypes.byref(c)), "frnn_plan_tuning_for")
        return int(t.g_max), float(t.cell_scale), int(t.walk), bool(c.value)

    def autotune(self, emb, ev_off, r: float, k: int, stream=None) -> tuple[int, float, float]:
        """frnn_plan_autotune on this batch: returns (g_max, cell_scale, ms) of
        the fastest tuning, which stays set on the plan."""
        ptr, n, d = self._emb_ptr(emb)
        off = np.ascontiguousarray(ev_off, dtype=np.int64)
        t = frnn_tuning()
        ms = ctypes.c_float(0.0)
        _check(load().frnn_plan_autotune(self._h, ptr, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                         off.size - 1, d, float(r), int(k), _stream_handle(stream),
                                         ctypes.byref(t), ctypes.byref(ms)), "frnn_plan_autotune")
        return int(t.g_max), float(t.cell_scale), float(ms.value)

    def _emb_ptr(self, emb):
        torch = _torch()
        if not (isinstance(emb, torch.Tensor) and emb.is_cuda and emb.dtype == torch.float32
                and emb.dim() == 2 and emb.is_contiguous()):
            raise TypeError("emb must be a contiguous float32 CUDA tensor of shape [n, d]")
        return emb.data_ptr(), emb.shape[0], emb.shape[1]

    def build(self, emb, r: float, k: int, stream=None) -> Csr:
        ptr, n, d = self._emb_ptr(emb)
        c = frnn_csr()
        _check(load().frnn_build_graph(self._h, ptr, n, d, float(r), int(k), _stream_handle(stream),
                                       ctypes.byref(c)), "frnn_build_graph")
        self._last_n = n
        return Csr(c, self.device, np.array([0, n], dtype=np.int64), self.edge_capacity)

    def build_batched(self, emb, ev_off, r: float, k: int, stream=None) -> Csr:
        ptr, n, d = self._emb_ptr(emb)
        off = np.ascontiguousarray(ev_off, dtype=np.int64)
        if off.ndim != 1 or off.size < 2 or off[-1] != n:
            raise ValueError("ev_off must hold n_events + 1 offsets ending at emb.shape[0]")
        c = frnn_csr()
        _check(load().frnn_build_graph_batched(self._h, ptr, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                               off.size - 1, d, float(r), int(k), _stream_handle(stream),
                                               ctypes.byref(c)), "frnn_build_graph_batched")
        self._last_n = n
        return Csr(c, self.device, off, self.edge_capacity)

    def knn_batched(self, emb, ev_off, k: int, stream=None) -> Csr:
        """frnn_knn_graph_batched: exact k-nearest-neighbour rows (no radius)
        of every event; row lengths min(k, n_b - 1)."""
        ptr, n, d = self._emb_ptr(emb)
        off = np.ascontiguousarray(ev_off, dtype=np.int64)
        if off.ndim != 1 or off.size < 2 or off[-1] != n:
            raise ValueError("ev_off must hold n_events + 1 offsets ending at emb.shape[0]")
        c = frnn_csr()
        _check(load().frnn_knn_graph_batched(self._h, ptr, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                             off.size - 1, d, int(k), _stream_handle(stream), ctypes.byref(c)),
               "frnn_knn_graph_batched")
        self._last_n = n
        return Csr(c, self.device, off, self.edge_capacity)

    STAGES = ("bbox_plan", "key_hist", "scan_cells", "scatter", "walk_collect", "scan_rows", "walk_emit")

    def build_profiled(self, emb, ev_off, r: float, k: int, stream=None):
        """Batched build with CUDA events between the stages (synchronous).
        Returns (Csr, {stage name: device milliseconds})."""
        ptr, n, d = self._emb_ptr(emb)
        off = np.ascontiguousarray(ev_off, dtype=np.int64)
        c = frnn_csr()
        ms = (ctypes.c_float * len(self.STAGES))()
        _check(load().frnn_build_graph_profiled(self._h, ptr, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                                off.size - 1, d, float(r), int(k), _stream_handle(stream),
                                                ctypes.byref(c), ms, len(self.STAGES)), "frnn_build_graph_profiled")
        return Csr(c, self.device, off, self.edge_capacity), dict(zip(self.STAGES, [float(v) for v in ms]))

    def build_host(self, emb: np.ndarray, ev_off, r: float, k: int, col_capacity: int | None = None,
                   stream=None, out: dict | None = None) -> dict:
        """Host arrays in, host CSR out (frnn_build_graph_host)."""
        emb = np.ascontiguousarray(emb, dtype=np.float32)
        off = np.ascontiguousarray(ev_off, dtype=np.int64)
        n = int(off[-1])
        if emb.ndim != 2 or emb.shape[0] != n:
            raise ValueError("emb must be [ev_off[-1], d]")
        if out is None:
            cap = int(col_capacity) if col_capacity is not None else n * int(k)
            out = dict(row_ptr=np.zeros(n + 1, np.int32), col=np.zeros(max(cap, 1), np.int32),
                       edge_off=np.zeros(off.size, np.int32))
        ne = ctypes.c_int64(0)
        rc = load().frnn_build_graph_host(
            self._h, emb.ctypes.data, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), off.size - 1,
            emb.shape[1], float(r), int(k), out["row_ptr"].ctypes.data, out["col"].ctypes.data,
            out["col"].size, out["edge_off"].ctypes.data, ctypes.byref(ne), _stream_handle(stream))
        out["n_edges"] = int(ne.value)
        _check(rc, "frnn_build_graph_host")
        return out

    def label_components(self, d2_max: float = float("inf"), stream=None, out=None):
        """frnn_label_components on the last build: event-local component
        labels (smallest index of each point's component), as an int32 CUDA
        tensor with one entry per point of the last call."""
        torch = _torch()
        n = int(self._last_n)
        labels = out if out is not None else torch.empty(max(n, 1), dtype=torch.int32, device=self.device)
        _check(load().frnn_label_components(self._h, float(d2_max), _stream_handle(stream),
                                            labels.data_ptr()), "frnn_label_components")
        return labels[:n]

    def edge_features(self, emb, e_begin: int, e_end: int, stream=None, out=None):
        """frnn_edge_features: [x_i, x_j, d2] rows for edges [e_begin, e_end) of
        the last build (emb: the points of that build), as a CUDA tensor of
        shape [e_end - e_begin, 2d + 1]."""
        torch = _torch()
        ptr, n, d = self._emb_ptr(emb)
        m = max(int(e_end) - int(e_begin), 0)
        if out is None:
            out = torch.empty((max(m, 1), 2 * d + 1), dtype=torch.float32, device=self.device)
        _check(load().frnn_edge_features(self._h, ptr, int(e_begin), int(e_end), out.data_ptr(),
                                         _stream_handle(stream)), "frnn_edge_features")
        return out[:m]

    def last_status(self, stream=None) -> int:
        """frnn_get_last_status: synchronise and return (and clear) the device status."""
        return int(load().frnn_get_last_status(self._h, _stream_handle(stream)))

    def check(self, stream=None) -> None:
        _check(self.last_status(stream), "device status")

    def check_last_build(self, stream=None) -> None:
        """frnn_check_last_build: enqueue the debug checks of the last build
        (a failure latches FRNN_ERR_CHECK; see last_check)."""
        _check(load().frnn_check_last_build(self._h, _stream_handle(stream)), "frnn_check_last_build")

    def last_check(self, stream=None) -> tuple[str, int]:
        """frnn_get_last_check: synchronise, return (check name, index) of the
        first recorded failure (("none", -1) if none) and clear the record."""
        cid, idx = ctypes.c_int(0), ctypes.c_int64(0)
        _check(load().frnn_get_last_check(self._h, _stream_handle(stream), ctypes.byref(cid), ctypes.byref(idx)),
               "frnn_get_last_check")
        return CHECKS[cid.value], int(idx.value)

    def test_stall_next_build(self) -> None:
        """frnn_plan_test_stall_next_build: the next build's scan waits run out
        (bounded, about 1 s) and latch FRNN_ERR_TIMEOUT; for failure-detection tests."""
        _check(load().frnn_plan_test_stall_next_build(self._h), "frnn_plan_test_stall_next_build")


def plan_bytes(n_max: int, d_max: int, k_max_cap: int, events_max: int = 1, edge_capacity: int = 0,
               cells_per_point: int = 0, emit_d2: bool = False) -> int:
    """Device bytes a plan with these capacities allocates (frnn_plan_bytes)."""
    prm = frnn_plan_params(device=0, d_max=d_max, n_max=n_max, events_max=events_max, k_max_cap=k_max_cap,
                           edge_capacity=edge_capacity, cells_per_point=cells_per_point,
                           flags=FRNN_EMIT_D2 if emit_d2 else 0)
    b = ctypes.c_uint64(0)
    _check(load().frnn_plan_bytes(ctypes.byref(prm), ctypes.byref(b)), "frnn_plan_bytes")
    return int(b.value)


class Server:
    """Continuous-batching graph server (frnn_server_*): submit host events,
    wait for their CSR; batches run on `slots` concurrent streams per device
    (`devices`: a list of device ordinals, default [device])."""

    def __init__(self, d: int, r: float, k: int, batch_points: int, batch_events: int = 64, slots: int = 2,
                 edges_per_point: int = 0, mem_budget_bytes: int = 0, device: int = 0, devices=None):
        lib = load()
        devs = list(devices) if devices else []
        arr = (ctypes.c_int * max(len(devs), 1))(*devs)
        prm = frnn_server_params(device=device, d=d, r=r, k=k, batch_points=batch_points,
                                 batch_events=batch_events, slots=slots, edges_per_point=edges_per_point,
                                 mem_budget_bytes=mem_budget_bytes, n_devices=len(devs),
                                 devices=ctypes.cast(arr, ctypes.POINTER(ctypes.c_int)) if devs else None)
        h = ctypes.c_void_p()
        _check(lib.frnn_server_create(ctypes.byref(h), ctypes.byref(prm)), "frnn_server_create")
        self._h = h
        self.d, self.k = d, k
        self._held = {}

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            load().frnn_server_destroy(self._h)
            self._h = ctypes.c_void_p()
        self._held = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def reserved_bytes(self) -> int:
        b = ctypes.c_uint64(0)
        _check(load().frnn_server_reserved_bytes(self._h, ctypes.byref(b)), "frnn_server_reserved_bytes")
        return int(b.value)

    def stats(self) -> dict:
        st = frnn_server_stats()
        _check(load().frnn_server_get_stats(self._h, ctypes.byref(st)), "frnn_server_get_stats")
        return {name: int(getattr(st, name)) for name, _ in frnn_server_stats._fields_}

    def poll(self, ticket: int) -> bool:
        """True once the event of `ticket` is done (wait() then returns at once)."""
        done = ctypes.c_int(0)
        _check(load().frnn_server_poll(self._h, ticket, ctypes.byref(done)), "frnn_server_poll")
        return bool(done.value)

    def submit(self, x: np.ndarray) -> int:
        x = np.ascontiguousarray(x, dtype=np.float32)
        if x.ndim != 2 or x.shape[1] != self.d:
            raise ValueError("x must be [n, d]")
        t = ctypes.c_uint64(0)
        _check(load().frnn_server_submit(self._h, x.ctypes.data, x.shape[0], ctypes.byref(t)), "frnn_server_submit")
        self._held[int(t.value)] = x  # the server reads it until the event is done
        return int(t.value)

    def wait(self, ticket: int) -> dict:
        x = self._held.pop(ticket)
        n = x.shape[0]
        row_ptr = np.zeros(n + 1, np.int32)
        col = np.zeros(max(n * self.k, 1), np.int32)
        ne = ctypes.c_int64(0)
        lat = ctypes.c_double(0.0)
        rc = load().frnn_server_wait(self._h, ticket, row_ptr.ctypes.data, col.ctypes.data, col.size,
                                     ctypes.byref(ne), ctypes.byref(lat))
        _check(rc, "frnn_server_wait")
        return dict(row_ptr=row_ptr, col=col[:ne.value], n_edges=int(ne.value), latency_s=float(lat.value))

    def run_trace(self, x_all: np.ndarray, ev_start, ev_len, arrival_s) -> dict:
        """Replay arrivals (seconds from the start, non-decreasing).  Request i
        is the points x_all[ev_start[i] : ev_start[i] + ev_len[i]] (requests may
        share points; pinned memory copies faster)."""
        if not (isinstance(x_all, np.ndarray) and x_all.dtype == np.float32 and x_all.flags["C_CONTIGUOUS"]):
            x_all = np.ascontiguousarray(x_all, dtype=np.float32)
        st = np.ascontiguousarray(ev_start, dtype=np.int64)
        ln = np.ascontiguousarray(ev_len, dtype=np.int64)
        arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
        if not (st.size == ln.size == arr.size) or (st.size and (st + ln).max() > x_all.shape[0]):
            raise ValueError("ev_start, ev_len and arrival_s must have one entry per request inside x_all")
        n_ev = st.size
        lat = np.zeros(n_ev, np.float64)
        ne = np.zeros(n_ev, np.int64)
        wall = ctypes.c_double(0.0)
        P = ctypes.POINTER
        rc = load().frnn_server_run_trace(self._h, x_all.ctypes.data, st.ctypes.data_as(P(ctypes.c_int64)),
                                          ln.ctypes.data_as(P(ctypes.c_int64)), arr.ctypes.data_as(P(ctypes.c_double)),
                                          n_ev, lat.ctypes.data_as(P(ctypes.c_double)),
                                          ne.ctypes.data_as(P(ctypes.c_int64)), ctypes.byref(wall))
        _check(rc, "frnn_server_run_trace")
        return dict(latency_s=lat, n_edges=ne, wall_s=float(wall.value))
