"""Balanced butterfly counting on one GB300 GPU.

A thin ctypes binding over the C ABI of ``libbb.so`` (declared in
``include/bb.h``). Every step of the count runs in the library's CUDA
kernels; this module only marshals arguments. There is no CPU fallback: if
the library is not built or no sm_103 device is present, calls raise.

    from paper_2308_07932_gb300 import Context, synth
    g = synth.uniform_2k_1k()
    with Context() as ctx:
        balanced, total, wedges = ctx.count(g)

``synth`` (seeded input graphs) has no dependency on the library.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbb.so")

BB_OK = 0
STATUS = {
    0: "BB_OK", 1: "BB_ERR_INVALID_ARG", 2: "BB_ERR_TOO_LARGE", 3: "BB_ERR_BUDGET",
    4: "BB_ERR_OOM", 5: "BB_ERR_TIMEOUT", 6: "BB_ERR_OVERFLOW", 7: "BB_ERR_CUDA",
    8: "BB_ERR_NO_DEVICE", 9: "BB_ERR_BUSY",
}


class BBError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class _Csr(ctypes.Structure):
    _fields_ = [("nU", ctypes.c_int64), ("nV", ctypes.c_int64), ("nE", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("col", ctypes.c_void_p)]


KERNELS = ("k_dense", "k_ctah", "k_team", "k_warp")


class _Timing(ctypes.Structure):
    _fields_ = [("build_ms", ctypes.c_double), ("count_ms", ctypes.c_double),
                ("kernel_ms", ctypes.c_double * len(KERNELS)),
                ("wedges", ctypes.c_int64 * len(KERNELS)),
                ("middles", ctypes.c_int64 * len(KERNELS)),
                ("anchors", ctypes.c_int64 * len(KERNELS)),
                ("product_ms", ctypes.c_double)]

class ClassShape(ctypes.Structure):
    """Bucket shape of a graph's work classes (``bb_class_shape``)."""
    _fields_ = [("warp_w_max", ctypes.c_uint32), ("warp_small_w", ctypes.c_uint32),
                ("team_w_max", ctypes.c_uint32), ("split_wedges", ctypes.c_uint32)]
    FIELDS = ("warp_w_max", "warp_small_w", "team_w_max", "split_wedges")
    DEFAULT = {"warp_w_max": 16384, "warp_small_w": 32, "team_w_max": 16384,
               "split_wedges": 65536}

    def to_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k in self.FIELDS}

    @classmethod
    def from_dict(cls, d: dict | None) -> "ClassShape":
        t = cls()
        for k in cls.FIELDS:
            setattr(t, k, int((d or cls.DEFAULT).get(k, cls.DEFAULT[k])))
        return t


NSIZE = 4  # batch size classes: < 2^14, < 2^17, < 2^20 edges, the rest


class BatchTune(ctypes.Structure):
    """Launch and bucket shapes of a batch (``bb_batch_tune``); per-class
    fields in ``KERNELS`` order, bucket shapes per size class."""
    _fields_ = [("warp_chunk", ctypes.c_uint32), ("concurrent", ctypes.c_uint32),
                ("grid_frac", ctypes.c_float * len(KERNELS)), ("dense_staged", ctypes.c_uint32),
                ("shape", ClassShape * NSIZE)]

    def to_dict(self) -> dict:
        return {"warp_chunk": int(self.warp_chunk), "concurrent": int(self.concurrent),
                "grid_frac": {k: round(float(f), 4) for k, f in zip(KERNELS, self.grid_frac)},
                "dense_staged": int(self.dense_staged),
                "shape": [s.to_dict() for s in self.shape]}

    @classmethod
    def from_dict(cls, d: dict) -> "BatchTune":
        t = cls()
        t.warp_chunk = int(d["warp_chunk"])
        t.concurrent = int(d["concurrent"])
        for i, k in enumerate(KERNELS):
            t.grid_frac[i] = float(d["grid_frac"][k])
        t.dense_staged = int(d.get("dense_staged", 0))
        shapes = d.get("shape") or [None] * NSIZE
        for i in range(NSIZE):
            t.shape[i] = ClassShape.from_dict(shapes[i])
        return t


class _Request(ctypes.Structure):
    _fields_ = [("key", ctypes.c_uint64), ("csr", ctypes.POINTER(_Csr)), ("signs", ctypes.c_void_p),
                ("flip_idx", ctypes.c_void_p), ("n_flip", ctypes.c_int64)]


class _ServeStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "failed", "cache_hits",
                                              "uploads", "evictions", "resident_graphs")] + \
               [(n, ctypes.c_uint64) for n in ("arena_bytes", "arena_used", "arena_largest_free")] + \
               [(n, ctypes.c_int64) for n in ("queued", "running", "incremental")]


REQ_NO_CACHE = 1

_lib = None
_VP = ctypes.c_void_p
_I64P = ctypes.POINTER(ctypes.c_int64)


def lib() -> ctypes.CDLL:
    """The loaded CUDA library. Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        S = ctypes.c_int
        sig = {
            "bb_last_error": (ctypes.c_char_p, []),
            "bb_version": (ctypes.c_char_p, []),
            "bb_ctx_create": (S, [ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(_VP)]),
            "bb_ctx_destroy": (None, [_VP]),
            "bb_ctx_set_stream": (S, [_VP, _VP]),
            "bb_ctx_device_bytes": (ctypes.c_uint64, [_VP]),
            "bb_count_csr": (S, [_VP, ctypes.POINTER(_Csr), _VP, _I64P, _I64P, _VP, _I64P]),
            "bb_count_csr_device": (S, [_VP, ctypes.POINTER(_Csr), _VP, _I64P, _I64P, _VP, _I64P]),
            "bb_graph_upload": (S, [_VP, ctypes.POINTER(_Csr), _VP, ctypes.POINTER(_VP)]),
            "bb_graph_upload_device": (S, [_VP, ctypes.POINTER(_Csr), _VP, ctypes.POINTER(_VP)]),
            "bb_count": (S, [_VP, _I64P, _I64P, _VP]),
            "bb_graph_flip_signs": (S, [_VP, _VP, ctypes.c_int64]),
            "bb_count_edges": (S, [_VP, _VP, _I64P, _I64P]),
            "bb_count_base": (S, [_VP, _I64P, _I64P]),
            "bb_count_flipped": (S, [_VP, _VP, ctypes.c_int64, _I64P, _I64P,
                                     ctypes.POINTER(ctypes.c_int)]),
            "bb_graph_info": (S, [_VP, _I64P, _I64P, _I64P, _I64P]),
            "bb_graph_free": (None, [_VP]),
            "bb_ctx_set_timing": (S, [_VP, ctypes.c_int]),
            "bb_ctx_last_timing": (S, [_VP, ctypes.POINTER(_Timing)]),
            "bb_launch_count": (ctypes.c_uint64, []),
            "bb_ctx_set_shape": (S, [_VP, ctypes.POINTER(ClassShape), ctypes.c_int]),
            "bb_graph_set_shape": (S, [_VP, ctypes.POINTER(ClassShape), ctypes.c_int]),
            "bb_batch_create": (S, [_VP, ctypes.POINTER(_VP), ctypes.c_int64, ctypes.POINTER(_VP)]),
            "bb_batch_count": (S, [_VP, _I64P, _I64P, ctypes.POINTER(ctypes.c_int)]),
            "bb_batch_set_tune": (S, [_VP, ctypes.POINTER(BatchTune)]),
            "bb_batch_get_tune": (S, [_VP, ctypes.POINTER(BatchTune)]),
            "bb_batch_autotune": (S, [_VP, ctypes.c_int, ctypes.POINTER(BatchTune),
                                      ctypes.POINTER(ctypes.c_double)]),
            "bb_batch_free": (None, [_VP]),
            "bb_ctx_serve": (S, [_VP, ctypes.c_int, ctypes.c_uint64]),
            "bb_submit": (S, [_VP, _VP, ctypes.c_uint32, ctypes.POINTER(_VP)]),
            "bb_submit_request": (S, [_VP, ctypes.POINTER(_Request), ctypes.c_uint32,
                                      ctypes.POINTER(_VP)]),
            "bb_poll": (S, [_VP, ctypes.POINTER(ctypes.c_int), _I64P, _I64P]),
            "bb_poll_timed": (S, [_VP, ctypes.POINTER(ctypes.c_int), _I64P, _I64P,
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
            "bb_ctx_serve_stats": (S, [_VP, ctypes.POINTER(_ServeStats)]),
            "bb_set_wait_timeout": (S, [ctypes.c_double]),
            "bb_set_alloc_failure": (S, [ctypes.c_int64]),
            "bb_probe_shared_atomics": (S, [ctypes.c_int, ctypes.c_uint32,
                                            ctypes.POINTER(ctypes.c_double)]),
            "bb_graph_bytes": (S, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                   ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
            "bb_set_matrix_product": (ctypes.c_int, [ctypes.c_int]),
            "bb_matrix_product_plan": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64,
                                                      ctypes.c_int64]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != BB_OK:
        raise BBError(status, lib().bb_last_error().decode(errors="replace"))


def _host_arrays(g):
    rowptr = np.ascontiguousarray(g.rowptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    sign = np.ascontiguousarray(g.sign, dtype=np.int8)
    csr = _Csr(g.nU, g.nV, int(col.shape[0]), rowptr.ctypes.data, col.ctypes.data)
    return csr, sign, (rowptr, col, sign)


@dataclass
class Counts:
    balanced: int
    total: int
    wedges: int
    per_vertex: np.ndarray | None = None

    def __iter__(self):
        yield self.balanced
        yield self.total
        yield self.wedges


class Context:
    """A device, a CUDA stream and a device memory budget (``bb_ctx``)."""

    def __init__(self, device: int = 0, budget_bytes: int = 0):
        h = _VP()
        _check(lib().bb_ctx_create(device, budget_bytes, ctypes.byref(h)))
        self._h = h
        self.device = device

    def close(self):
        if getattr(self, "_h", None):
            lib().bb_ctx_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def device_bytes(self) -> int:
        return int(lib().bb_ctx_device_bytes(self._h))

    def set_timing(self, on: bool = True):
        """Record CUDA events around the build and each wedge kernel."""
        _check(lib().bb_ctx_set_timing(self._h, 1 if on else 0))

    def last_timing(self) -> dict:
        """Phase timings (ms) and per-kernel work of the last count."""
        t = _Timing()
        _check(lib().bb_ctx_last_timing(self._h, ctypes.byref(t)))
        return {"build_ms": t.build_ms, "count_ms": t.count_ms, "product_ms": t.product_ms,
                "kernels": {k: {"ms": t.kernel_ms[i], "wedges": t.wedges[i],
                                "middles": t.middles[i], "anchors": t.anchors[i]}
                            for i, k in enumerate(KERNELS)}}

    def set_shape(self, shape: dict | None = None, dense_staged: bool = False):
        """Bucket shape (``bb_ctx_set_shape``) of later one-shot counts and
        uploads: a dict of ``ClassShape.FIELDS`` (missing keys take their
        defaults), None for the defaults."""
        sh = ClassShape.from_dict(shape) if shape is not None else None
        _check(lib().bb_ctx_set_shape(self._h, ctypes.byref(sh) if sh is not None else None,
                                      int(dense_staged)))

    def set_stream(self, stream_ptr: int | None):
        """Run on a cudaStream_t given as an integer handle (e.g.
        ``torch.cuda.current_stream().cuda_stream``); None = own stream."""
        _check(lib().bb_ctx_set_stream(self._h, stream_ptr or None))

    def count(self, g, per_vertex: bool = False) -> Counts:
        """Whole path on a host graph (``bb_count_csr``)."""
        csr, sign, keep = _host_arrays(g)
        b, t, w = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        pv = np.zeros(g.nU + g.nV, np.int64) if per_vertex else None
        _check(lib().bb_count_csr(self._h, ctypes.byref(csr), sign.ctypes.data, ctypes.byref(b),
                                  ctypes.byref(t), pv.ctypes.data if pv is not None else None,
                                  ctypes.byref(w)))
        del keep
        return Counts(b.value, t.value, w.value, pv)

    def count_host_ptrs(self, nU: int, nV: int, nE: int, rowptr_ptr: int, col_ptr: int,
                        sign_ptr: int) -> Counts:
        """``bb_count_csr`` on raw host pointers (e.g. pinned tensors)."""
        csr = _Csr(nU, nV, nE, rowptr_ptr, col_ptr)
        b, t, w = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().bb_count_csr(self._h, ctypes.byref(csr), sign_ptr, ctypes.byref(b),
                                  ctypes.byref(t), None, ctypes.byref(w)))
        return Counts(b.value, t.value, w.value)

    def count_device(self, nU: int, nV: int, nE: int, rowptr_ptr: int, col_ptr: int,
                     sign_ptr: int, per_vertex_ptr: int | None = None) -> Counts:
        """Whole path on device buffers (``bb_count_csr_device``); pointers
        are device addresses, e.g. ``tensor.data_ptr()`` of CUDA tensors."""
        csr = _Csr(nU, nV, nE, rowptr_ptr, col_ptr)
        b, t, w = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().bb_count_csr_device(self._h, ctypes.byref(csr), sign_ptr, ctypes.byref(b),
                                         ctypes.byref(t), per_vertex_ptr, ctypes.byref(w)))
        return Counts(b.value, t.value, w.value)

    def count_tensors(self, nV: int, rowptr, col, sign, per_vertex=None) -> Counts:
        """``count_device`` on torch CUDA tensors (int64 rowptr, int32 col,
        int8 sign; per_vertex: optional int64 CUDA tensor of nU+nV)."""
        nU = rowptr.numel() - 1
        return self.count_device(nU, nV, col.numel(), rowptr.data_ptr(), col.data_ptr(),
                                 sign.data_ptr(),
                                 per_vertex.data_ptr() if per_vertex is not None else None)

    # ------------------------------------------------------------ serving
    def serve(self, slots: int = 4, arena_bytes: int = 0):
        """Start the serving engine (``bb_ctx_serve``): `slots` concurrent
        requests, `arena_bytes` of device memory for the managed cache."""
        _check(lib().bb_ctx_serve(self._h, slots, arena_bytes))

    def submit(self, graph: "Graph") -> "Ticket":
        """Asynchronous count of a resident graph (``bb_submit``)."""
        h = _VP()
        _check(lib().bb_submit(self._h, graph._h, 0, ctypes.byref(h)))
        return Ticket(h, (graph,))

    def submit_request(self, key: int, g=None, flips=None, no_cache: bool = False) -> "Ticket":
        """Asynchronous count of the graph named `key` (``bb_submit_request``):
        uploaded from host graph `g` unless resident; `flips` (edge indices)
        flip signs of the resident graph first. The host arrays are kept
        alive by the ticket until it is done."""
        keep = []
        req = _Request()
        req.key = key
        if g is not None:
            csr, sign, arrays = _host_arrays(g)
            keep += [csr, sign, arrays]
            req.csr = ctypes.pointer(csr)
            req.signs = sign.ctypes.data
        if flips is not None:
            f = np.ascontiguousarray(flips, dtype=np.int64)
            keep.append(f)
            req.flip_idx = f.ctypes.data
            req.n_flip = f.size
        keep.append(req)
        h = _VP()
        _check(lib().bb_submit_request(self._h, ctypes.byref(req), REQ_NO_CACHE if no_cache else 0,
                                       ctypes.byref(h)))
        return Ticket(h, tuple(keep))

    def serve_stats(self) -> dict:
        st = _ServeStats()
        _check(lib().bb_ctx_serve_stats(self._h, ctypes.byref(st)))
        return {n: int(getattr(st, n)) for n, _ in _ServeStats._fields_}

    def upload(self, g) -> "Graph":
        """Resident graph from a host graph (``bb_graph_upload``)."""
        csr, sign, keep = _host_arrays(g)
        h = _VP()
        _check(lib().bb_graph_upload(self._h, ctypes.byref(csr), sign.ctypes.data, ctypes.byref(h)))
        del keep
        return Graph(self, h)


@dataclass
class Served:
    balanced: int
    total: int
    queue_ms: float
    run_ms: float


class Ticket:
    """An asynchronous request. ``poll()`` returns None until it is done,
    then its counts (or raises its error); the handle is released then."""

    def __init__(self, handle, keep):
        self._h = handle
        self._keep = keep
        self.result: Served | None = None

    def poll(self) -> Served | None:
        if self.result is not None:
            return self.result
        done = ctypes.c_int()
        b, t = ctypes.c_int64(), ctypes.c_int64()
        q, r = ctypes.c_double(), ctypes.c_double()
        st = lib().bb_poll_timed(self._h, ctypes.byref(done), ctypes.byref(b), ctypes.byref(t),
                                 ctypes.byref(q), ctypes.byref(r))
        if not done.value:
            _check(st)
            return None
        self._h = None
        self._keep = None
        _check(st)
        self.result = Served(b.value, t.value, q.value, r.value)
        return self.result

    def wait(self, timeout: float = 600.0) -> Served:
        import time
        t0 = time.monotonic()
        while True:
            r = self.poll()
            if r is not None:
                return r
            if time.monotonic() - t0 > timeout:
                raise TimeoutError("request did not finish")
            time.sleep(50e-6)


class Graph:
    """A graph kept resident on the device (``bb_graph``)."""

    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self._h = handle

    def count(self, per_vertex: bool = False) -> Counts:
        b, t = ctypes.c_int64(), ctypes.c_int64()
        nU, nV, nE, w = self.info()
        pv = np.zeros(nU + nV, np.int64) if per_vertex else None
        _check(lib().bb_count(self._h, ctypes.byref(b), ctypes.byref(t),
                              pv.ctypes.data if pv is not None else None))
        return Counts(b.value, t.value, w, pv)

    def set_shape(self, shape: dict | None = None, dense_staged: bool = False):
        """Re-classifies the graph with a bucket shape (``bb_graph_set_shape``)."""
        sh = ClassShape.from_dict(shape) if shape is not None else None
        _check(lib().bb_graph_set_shape(self._h, ctypes.byref(sh) if sh is not None else None,
                                        int(dense_staged)))

    def count_edges(self) -> tuple[np.ndarray, int, int]:
        """Balanced butterflies containing each edge (input CSR order), and
        the graph's (balanced, total) counts (``bb_count_edges``)."""
        nU, nV, nE, w = self.info()
        pe = np.zeros(max(nE, 1), np.int64)
        b, t = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().bb_count_edges(self._h, pe.ctypes.data, ctypes.byref(b), ctypes.byref(t)))
        return pe[:nE], b.value, t.value

    def count_base(self) -> tuple[int, int]:
        """(balanced, total) by BB-Base (Algorithm 1) on the GPU, for comparison
        with the bucket method (``bb_count_base``)."""
        b, t = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().bb_count_base(self._h, ctypes.byref(b), ctypes.byref(t)))
        return b.value, t.value

    def count_flipped(self, edge_idx) -> tuple[int, int, bool]:
        """Flip the listed edges' signs and return (balanced, total,
        incremental) after the flips (``bb_count_flipped``)."""
        e = np.ascontiguousarray(edge_idx, dtype=np.int64)
        b, t, inc = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        _check(lib().bb_count_flipped(self._h, e.ctypes.data, e.size, ctypes.byref(b),
                                      ctypes.byref(t), ctypes.byref(inc)))
        return b.value, t.value, bool(inc.value)

    def flip(self, edge_idx):
        e = np.ascontiguousarray(edge_idx, dtype=np.int64)
        _check(lib().bb_graph_flip_signs(self._h, e.ctypes.data, e.size))

    def info(self):
        v = [ctypes.c_int64() for _ in range(4)]
        _check(lib().bb_graph_info(self._h, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def free(self):
        if getattr(self, "_h", None):
            lib().bb_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Batch:
    """Resident graphs counted together in one captured launch sequence
    (``bb_batch``). Holds references to its graphs so they outlive it."""

    def __init__(self, ctx: Context, graphs: list):
        self.ctx = ctx
        self.graphs = list(graphs)
        arr = (_VP * len(self.graphs))(*[g._h for g in self.graphs])
        h = _VP()
        _check(lib().bb_batch_create(ctx._h, arr, len(self.graphs), ctypes.byref(h)))
        self._h = h

    def count(self, with_status: bool = False):
        """(balanced, total) int64 arrays, one entry per graph; with_status
        also returns the per-graph status array instead of raising."""
        n = len(self.graphs)
        b = np.empty(n, np.int64)
        t = np.empty(n, np.int64)
        st = np.zeros(n, np.int32)
        r = lib().bb_batch_count(self._h, b.ctypes.data_as(_I64P), t.ctypes.data_as(_I64P),
                                 st.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        if with_status:
            return b, t, st
        _check(r)
        return b, t

    def tune(self) -> BatchTune:
        t = BatchTune()
        _check(lib().bb_batch_get_tune(self._h, ctypes.byref(t)))
        return t

    def set_tune(self, t: BatchTune | dict):
        if isinstance(t, dict):
            t = BatchTune.from_dict(t)
        _check(lib().bb_batch_set_tune(self._h, ctypes.byref(t)))

    def autotune(self, reps: int = 3) -> tuple[BatchTune, float]:
        t = BatchTune()
        ms = ctypes.c_double()
        _check(lib().bb_batch_autotune(self._h, reps, ctypes.byref(t), ctypes.byref(ms)))
        return t, ms.value

    def free(self):
        if getattr(self, "_h", None):
            lib().bb_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def graph_bytes(nU: int, nV: int, nE: int) -> tuple[int, int]:
    """(resident, build workspace) device bytes of a graph of these sizes."""
    r, w = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().bb_graph_bytes(nU, nV, nE, ctypes.byref(r), ctypes.byref(w)))
    return r.value, w.value


def request_bytes(g) -> int:
    """Arena bytes a served request for host graph g needs while it builds:
    resident graph, input copy and build workspace, each 256-byte aligned."""
    r, w = graph_bytes(g.nU, g.nV, g.nE)
    a = lambda x: (x + 255) // 256 * 256  # noqa: E731
    return a(r) + a(w) + a((g.nU + 1) * 8) + a(g.nE * 4) + a(g.nE)


def set_wait_timeout(seconds: float):
    """Limit on how long blocking calls wait for device work (process-wide)."""
    _check(lib().bb_set_wait_timeout(seconds))


def set_alloc_failure(nth: int):
    """Makes the nth device allocation of the library from now on fail once
    with BB_ERR_OOM (``bb_set_alloc_failure``; 0 disarms). For tests."""
    _check(lib().bb_set_alloc_failure(nth))


def probe_shared_atomics(device: int = 0, window: int = 2048) -> float:
    """Shared-memory atomic adds per second on the device (all SMs)."""
    r = ctypes.c_double()
    _check(lib().bb_probe_shared_atomics(device, window, ctypes.byref(r)))
    return r.value


def version() -> str:
    return lib().bb_version().decode()


def launch_count() -> int:
    """Kernel launches the library has issued in this process."""
    return int(lib().bb_launch_count())


def set_matrix_product(enabled: bool) -> bool:
    """Whether counts of graphs with a small dense side may take the
    matrix-product path (``bb_set_matrix_product``; process-wide, on by
    default). Returns the previous setting."""
    return lib().bb_set_matrix_product(0 if enabled else 1) == 0


def matrix_product_plan(nU: int, nV: int, nE: int) -> bool:
    """True if a graph of these sizes is counted on the matrix-product path
    under the current setting."""
    r = lib().bb_matrix_product_plan(nU, nV, nE)
    if r < 0:
        raise BBError(1, "negative size")
    return r == 1
