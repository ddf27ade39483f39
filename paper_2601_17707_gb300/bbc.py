"""Python binding of ``libbbc.so`` (include/bbc.h), argument marshalling only.

Every computation runs in the library's CUDA kernels. PyTorch supplies device memory
and streams: device tensors are passed by ``data_ptr()`` and streams by
``torch.cuda.current_stream().cuda_stream``. The library must have been built (see
``paper_2601_17707_gb300._build.build``); loading fails loudly otherwise, and there is
no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import _build

OK = 0
STATUS_NAMES = {
    0: "BBC_OK", 1: "BBC_E_INVALID_ARG", 2: "BBC_E_OUT_OF_RANGE", 3: "BBC_E_BAD_SIGN",
    4: "BBC_E_DUPLICATE_EDGE", 5: "BBC_E_OVERFLOW_RISK", 6: "BBC_E_NO_MEMORY",
    7: "BBC_E_OVER_BUDGET", 8: "BBC_E_CUDA", 9: "BBC_E_TIMEOUT", 10: "BBC_E_CANCELLED",
    11: "BBC_E_NOT_READY", 12: "BBC_E_NO_DEVICE",
}
INPUT_DEVICE = 1
DEDUP_LAST = 2
SIDE_FORCE_U = 4
SIDE_FORCE_V = 8
ORIENT_LOW_ANCHOR = 16

# Every symbol include/bbc.h declares (checked by the tests).
EXPORTS = (
    "bbc_tuning_default", "bbc_prepare", "bbc_count", "bbc_count_async", "bbc_graph_info",
    "bbc_graph_free", "bbc_count_batch", "bbc_autotune_batch", "bbc_server_create", "bbc_submit",
    "bbc_poll", "bbc_wait", "bbc_server_stats", "bbc_server_destroy", "bbc_status_string",
    "bbc_last_error", "bbc_launch_count", "bbc_profile_start", "bbc_profile_stop",
    "bbc_count_noalloc", "bbc_count_motif", "bbc_cost_model_create", "bbc_cost_model_free",
    "bbc_cost_model_num_params", "bbc_cost_model_get_params", "bbc_cost_model_set_params",
    "bbc_cost_model_loss_grad", "bbc_cost_model_fit", "bbc_cost_model_predict", "bbc_item_features",
    "bbc_item_cycles", "bbc_cost_model_order", "bbc_count_delta", "bbc_graph_work",
    "bbc_item_anchors", "bbc_server_counters_get", "bbc_server_request_info", "bbc_memory_usage",
    "bbc_batch_tuning",
)

MOTIF_SIGN_CLASSES = 1
MOTIF_BICLIQUE_2K = 2


class BBCError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} ({detail})")


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class ServerCounters(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
        ("admitted_after_wait", ctypes.c_uint64), ("queued_now", ctypes.c_uint64),
        ("max_queued", ctypes.c_uint64), ("max_resident", ctypes.c_uint64), ("ticks", ctypes.c_uint64),
        ("budget_bytes", ctypes.c_size_t), ("reserved_bytes", ctypes.c_size_t),
        ("peak_reserved_bytes", ctypes.c_size_t), ("tick_wall_us", ctypes.c_double),
        ("tick_gpu_us", ctypes.c_double), ("prep_wall_us", ctypes.c_double), ("elapsed_us", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class RequestInfo(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32), ("ticks", ctypes.c_int32), ("n_edges", ctypes.c_int64),
        ("wedges", ctypes.c_uint64), ("reserved_bytes", ctypes.c_size_t),
        ("waited_for_memory", ctypes.c_int32), ("pad", ctypes.c_int32),
        ("latency_us", ctypes.c_double), ("queued_us", ctypes.c_double), ("prepare_us", ctypes.c_double),
        ("count_us", ctypes.c_double), ("tick_gpu_us", ctypes.c_double), ("submit_us", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class Tuning(ctypes.Structure):
    _fields_ = [
        ("tile_words", ctypes.c_int32),
        ("warp_max_wedges", ctypes.c_int32),
        ("dense_min_permille", ctypes.c_int32),
        ("split_wedges", ctypes.c_int32),
        ("blocks_per_sm", ctypes.c_int32),
        ("plain", ctypes.c_int32),
        ("queue_chunk", ctypes.c_int32),
        ("group_warps", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None
_LOCK = threading.Lock()


def load(path: str | None = None) -> ctypes.CDLL:
    """Loads the compiled library (no build, no fallback)."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        p = path or _build.LIB
        if not os.path.exists(p):
            raise RuntimeError(f"libbbc.so is not built ({p}); run paper_2601_17707_gb300._build.build()")
        lib = ctypes.CDLL(p)
        vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
        pu64 = ctypes.POINTER(ctypes.c_uint64)
        sig = {
            "bbc_tuning_default": ([ctypes.POINTER(Tuning)], ctypes.c_int),
            "bbc_prepare": ([i32, i32, i64, vp, vp, vp, u32, vp, ctypes.POINTER(vp)], ctypes.c_int),
            "bbc_count": ([vp, pu64, pu64, vp, vp, ctypes.POINTER(Tuning), vp], ctypes.c_int),
            "bbc_count_async": ([vp, vp, vp, vp, ctypes.POINTER(Tuning), vp], ctypes.c_int),
            "bbc_graph_info": ([vp, ctypes.POINTER(i32), pu64, ctypes.POINTER(ctypes.c_size_t),
                                ctypes.POINTER(i64)], ctypes.c_int),
            "bbc_graph_free": ([vp], None),
            "bbc_count_batch": ([i32, vp, vp, ctypes.POINTER(Tuning), vp], ctypes.c_int),
            "bbc_autotune_batch": ([i32, vp, ctypes.POINTER(Tuning), vp], ctypes.c_int),
            "bbc_batch_tuning": ([i32, vp, ctypes.POINTER(Tuning)], ctypes.c_int),
            "bbc_server_create": ([ctypes.c_size_t, ctypes.POINTER(Tuning), ctypes.POINTER(vp)],
                                  ctypes.c_int),
            "bbc_submit": ([vp, i32, i32, i64, vp, vp, vp, pu64], ctypes.c_int),
            "bbc_poll": ([vp, ctypes.c_uint64, pu64], ctypes.c_int),
            "bbc_wait": ([vp, ctypes.c_uint64, i64, pu64], ctypes.c_int),
            "bbc_server_stats": ([vp, pu64, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
                                 ctypes.c_int),
            "bbc_server_destroy": ([vp], None),
            "bbc_server_counters_get": ([vp, ctypes.POINTER(ServerCounters)], ctypes.c_int),
            "bbc_server_request_info": ([vp, ctypes.c_uint64, ctypes.POINTER(RequestInfo)], ctypes.c_int),
            "bbc_memory_usage": ([ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t), i32],
                                 ctypes.c_int),
            "bbc_status_string": ([ctypes.c_int], ctypes.c_char_p),
            "bbc_launch_count": ([], ctypes.c_ulonglong),
            "bbc_profile_start": ([], ctypes.c_int),
            "bbc_profile_stop": ([ctypes.POINTER(KernelTime), i32, ctypes.POINTER(i32)], ctypes.c_int),
            "bbc_last_error": ([], ctypes.c_char_p),
            "bbc_count_noalloc": ([vp, vp, vp], ctypes.c_int),
            "bbc_count_motif": ([vp, i32, i32, vp, vp], ctypes.c_int),
            "bbc_cost_model_create": ([ctypes.c_uint64, ctypes.POINTER(vp)], ctypes.c_int),
            "bbc_cost_model_free": ([vp], None),
            "bbc_cost_model_num_params": ([], i32),
            "bbc_cost_model_get_params": ([vp, vp, i32], ctypes.c_int),
            "bbc_cost_model_set_params": ([vp, vp, i32], ctypes.c_int),
            "bbc_cost_model_loss_grad": ([vp, vp, vp, i32, vp, vp, vp], ctypes.c_int),
            "bbc_cost_model_fit": ([vp, vp, vp, i32, i32, ctypes.c_float, vp, vp], ctypes.c_int),
            "bbc_cost_model_predict": ([vp, vp, i32, vp, vp], ctypes.c_int),
            "bbc_item_features": ([vp, vp, i32, ctypes.POINTER(i32), vp], ctypes.c_int),
            "bbc_item_cycles": ([vp, vp, i32, ctypes.POINTER(i32), vp], ctypes.c_int),
            "bbc_item_anchors": ([vp, vp, i32, ctypes.POINTER(i32), vp], ctypes.c_int),
            "bbc_cost_model_order": ([vp, vp, vp], ctypes.c_int),
            "bbc_graph_work": ([vp, vp, vp], ctypes.c_int),
            "bbc_count_delta": ([vp, i64, vp, vp, vp, u32, ctypes.POINTER(i64), ctypes.POINTER(i64), vp],
                                ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _LIB = lib
        return lib


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().bbc_launch_count())


def profile_start() -> None:
    check(load().bbc_profile_start(), "bbc_profile_start")


def profile_stop() -> dict:
    """{kernel name: (launches, total device ms)} since profile_start."""
    arr = (KernelTime * 8)()
    n = ctypes.c_int32()
    check(load().bbc_profile_stop(arr, 8, ctypes.byref(n)), "bbc_profile_stop")
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms))
            for i in range(min(n.value, 8))}


def memory_usage(reset_high: bool = False) -> tuple[int, int]:
    """(bytes the library's device pool holds now, the most it held at once since the
    last reset) on the current device."""
    used = ctypes.c_size_t()
    high = ctypes.c_size_t()
    check(load().bbc_memory_usage(ctypes.byref(used), ctypes.byref(high), int(bool(reset_high))),
          "bbc_memory_usage")
    return int(used.value), int(high.value)


def last_error() -> str:
    return load().bbc_last_error().decode()


def check(status: int, where: str) -> None:
    if status != OK:
        raise BBCError(status, where, last_error())


def default_tuning() -> Tuning:
    t = Tuning()
    check(load().bbc_tuning_default(ctypes.byref(t)), "bbc_tuning_default")
    return t


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _edge_arrays(u, v, sign):
    """Returns (ptr_u, ptr_v, ptr_s, n_edges, on_device, keepalive)."""
    try:
        import torch

        if isinstance(u, torch.Tensor):
            assert u.dtype == torch.int32 and v.dtype == torch.int32 and sign.dtype == torch.int8
            dev = u.is_cuda
            if dev != v.is_cuda or dev != sign.is_cuda:
                raise ValueError("u, v and sign must all live on the same device")
            u, v, sign = u.contiguous(), v.contiguous(), sign.contiguous()
            return u.data_ptr(), v.data_ptr(), sign.data_ptr(), int(u.numel()), dev, (u, v, sign)
    except ImportError:
        pass
    u = np.ascontiguousarray(u, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.int32)
    sign = np.ascontiguousarray(sign, dtype=np.int8)
    if not (u.shape == v.shape == sign.shape):
        raise ValueError("u, v and sign must have the same length")
    return u.ctypes.data, v.ctypes.data, sign.ctypes.data, int(u.shape[0]), False, (u, v, sign)


@dataclass
class Info:
    side: int
    wedges: int
    device_bytes: int
    n_edges: int


class Graph:
    """A prepared graph (owns its device memory until ``free``)."""

    def __init__(self, handle: int, n_u: int, n_v: int):
        self._h = ctypes.c_void_p(handle)
        self.n_u = n_u
        self.n_v = n_v

    @classmethod
    def prepare(cls, n_u: int, n_v: int, u, v, sign, flags: int = 0, stream=None) -> "Graph":
        lib = load()
        pu, pv, ps, n, on_dev, keep = _edge_arrays(u, v, sign)
        if on_dev:
            flags |= INPUT_DEVICE
        h = ctypes.c_void_p()
        st = lib.bbc_prepare(int(n_u), int(n_v), n, pu, pv, ps, flags, _stream_ptr(stream),
                             ctypes.byref(h))
        del keep
        check(st, "bbc_prepare")
        return cls(h.value, int(n_u), int(n_v))

    @classmethod
    def from_synthetic(cls, g, flags: int = 0, device: bool = True, stream=None) -> "Graph":
        """Prepares a ``synth.SignedBipartite`` (copied to the device first if ``device``)."""
        if device:
            import torch

            u = torch.from_numpy(np.ascontiguousarray(g.u)).cuda()
            v = torch.from_numpy(np.ascontiguousarray(g.v)).cuda()
            s = torch.from_numpy(np.ascontiguousarray(g.sign)).cuda()
            return cls.prepare(g.n_u, g.n_v, u, v, s, flags, stream)
        return cls.prepare(g.n_u, g.n_v, g.u, g.v, g.sign, flags, stream)

    @property
    def handle(self) -> int:
        if not self._h.value:
            raise RuntimeError("graph already freed")
        return self._h.value

    def count(self, per_vertex: bool = False, tuning: Tuning | None = None, stream=None):
        """Returns (balanced, unbalanced, per_u, per_v); per-vertex arrays are torch
        uint64-valued int64 CUDA tensors when requested, else None."""
        import torch

        lib = load()
        b = ctypes.c_uint64(0)
        ub = ctypes.c_uint64(0)
        pu = pv = None
        if per_vertex:
            pu = torch.empty(max(self.n_u, 1), dtype=torch.int64, device="cuda")
            pv = torch.empty(max(self.n_v, 1), dtype=torch.int64, device="cuda")
        st = lib.bbc_count(self.handle, ctypes.byref(b), ctypes.byref(ub),
                           pu.data_ptr() if pu is not None else None,
                           pv.data_ptr() if pv is not None else None,
                           ctypes.byref(tuning) if tuning is not None else None,
                           _stream_ptr(stream))
        check(st, "bbc_count")
        if per_vertex:
            pu, pv = pu[: self.n_u], pv[: self.n_v]
        return int(b.value), int(ub.value), pu, pv

    def count_async(self, totals, per_u=None, per_v=None, tuning: Tuning | None = None,
                    stream=None) -> None:
        """Queues a count; ``totals`` is a 2-element int64 CUDA tensor (balanced, unbalanced)."""
        lib = load()
        st = lib.bbc_count_async(self.handle, totals.data_ptr(),
                                 per_u.data_ptr() if per_u is not None else None,
                                 per_v.data_ptr() if per_v is not None else None,
                                 ctypes.byref(tuning) if tuning is not None else None,
                                 _stream_ptr(stream))
        check(st, "bbc_count_async")

    def count_motif(self, kind: str, k: int = 2, stream=None) -> tuple:
        """kind "classes": the six sign-class counts (Table 7's order); kind "biclique":
        (balanced (2,k)-bicliques, all (2,k)-bicliques). The pair side is the graph's S."""
        lib = load()
        kind_id = {"classes": MOTIF_SIGN_CLASSES, "biclique": MOTIF_BICLIQUE_2K}[kind]
        out = (ctypes.c_uint64 * 6)()
        check(lib.bbc_count_motif(self.handle, kind_id, int(k), ctypes.addressof(out),
                                  _stream_ptr(stream)), "bbc_count_motif")
        return tuple(int(x) for x in out[:6 if kind_id == MOTIF_SIGN_CLASSES else 2])

    def work(self, stream=None) -> dict:
        """{path: (items, wedges, pair-side edges)} of the current work lists."""
        out = (ctypes.c_uint64 * 12)()
        check(load().bbc_graph_work(self.handle, ctypes.addressof(out), _stream_ptr(stream)),
              "bbc_graph_work")
        names = ("k_tile", "k_group_tile", "k_warp_tile", "k_warp_hash")
        return {n: (int(out[3 * k]), int(out[3 * k + 1]), int(out[3 * k + 2])) for k, n in enumerate(names)}

    def count_delta(self, u, v, new_sign, stream=None) -> tuple:
        """(change in balanced, change in unbalanced butterflies) if edge (u[i], v[i]) took
        sign new_sign[i] (+1 / -1; 0 deletes). The graph is not modified."""
        lib = load()
        pu, pv, ps, n, on_dev, keep = _edge_arrays(u, v, new_sign)
        db = ctypes.c_int64()
        dub = ctypes.c_int64()
        check(lib.bbc_count_delta(self.handle, n, pu, pv, ps, INPUT_DEVICE if on_dev else 0,
                                  ctypes.byref(db), ctypes.byref(dub), _stream_ptr(stream)),
              "bbc_count_delta")
        del keep
        return int(db.value), int(dub.value)

    def item_features(self, stream=None):
        """Feature rows of the graph's tile items (float32 CUDA tensor [n, 8]), queue order."""
        import torch

        lib = load()
        n = ctypes.c_int32()
        cap = max(1, self._n_tile_items(stream))
        X = torch.empty((cap, 8), dtype=torch.float32, device="cuda")
        check(lib.bbc_item_features(self.handle, X.data_ptr(), cap, ctypes.byref(n), _stream_ptr(stream)),
              "bbc_item_features")
        return X[: n.value]

    def item_cycles(self, stream=None):
        """Per tile item, its duration in SM cycles from one instrumented tile-kernel run
        (int64 CUDA tensor, queue order)."""
        import torch

        lib = load()
        n = ctypes.c_int32()
        cap = max(1, self._n_tile_items(stream))
        c = torch.empty(cap, dtype=torch.int64, device="cuda")
        check(lib.bbc_item_cycles(self.handle, c.data_ptr(), cap, ctypes.byref(n), _stream_ptr(stream)),
              "bbc_item_cycles")
        return c[: n.value]

    def item_anchors(self, stream=None):
        """Per tile item, the original pair-side id of its anchor (int32 CUDA tensor, queue
        order)."""
        import torch

        lib = load()
        n = ctypes.c_int32()
        cap = max(1, self._n_tile_items(stream))
        a = torch.empty(cap, dtype=torch.int32, device="cuda")
        check(lib.bbc_item_anchors(self.handle, a.data_ptr(), cap, ctypes.byref(n), _stream_ptr(stream)),
              "bbc_item_anchors")
        return a[: n.value]

    def _n_tile_items(self, stream=None) -> int:
        lib = load()
        n = ctypes.c_int32()
        check(lib.bbc_item_features(self.handle, None, 0, ctypes.byref(n), _stream_ptr(stream)),
              "bbc_item_features")
        return n.value

    def info(self) -> Info:
        lib = load()
        side = ctypes.c_int32()
        w = ctypes.c_uint64()
        db = ctypes.c_size_t()
        ne = ctypes.c_int64()
        check(lib.bbc_graph_info(self.handle, ctypes.byref(side), ctypes.byref(w), ctypes.byref(db),
                                 ctypes.byref(ne)), "bbc_graph_info")
        return Info(side.value, w.value, db.value, ne.value)

    def free(self) -> None:
        if self._h.value:
            load().bbc_graph_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def as_uint64(t) -> np.ndarray:
    """A per-vertex result tensor as a numpy uint64 array."""
    return t.cpu().numpy().view(np.uint64)


def count_batch(graphs: list[Graph], tuning: Tuning | None = None, stream=None) -> list[int]:
    lib = load()
    n = len(graphs)
    hs = (ctypes.c_void_p * max(n, 1))(*[g.handle for g in graphs])
    out = (ctypes.c_uint64 * max(n, 1))()
    check(lib.bbc_count_batch(n, hs, out, ctypes.byref(tuning) if tuning is not None else None,
                              _stream_ptr(stream)), "bbc_count_batch")
    return [int(out[i]) for i in range(n)]


def autotune_batch(graphs: list[Graph], stream=None) -> Tuning:
    lib = load()
    n = len(graphs)
    hs = (ctypes.c_void_p * max(n, 1))(*[g.handle for g in graphs])
    t = Tuning()
    check(lib.bbc_autotune_batch(n, hs, ctypes.byref(t), _stream_ptr(stream)), "bbc_autotune_batch")
    return t


def batch_tuning(graphs: list[Graph]) -> Tuning:
    """The tuning a NULL-tuning count_batch call would use for these graphs."""
    lib = load()
    n = len(graphs)
    hs = (ctypes.c_void_p * max(n, 1))(*[g.handle for g in graphs])
    t = Tuning()
    check(lib.bbc_batch_tuning(n, hs, ctypes.byref(t)), "bbc_batch_tuning")
    return t


class Server:
    """The continuous-batching request loop (bbc_server_*)."""

    def __init__(self, device_budget_bytes: int, tuning: Tuning | None = None):
        lib = load()
        h = ctypes.c_void_p()
        check(lib.bbc_server_create(int(device_budget_bytes),
                                    ctypes.byref(tuning) if tuning is not None else None,
                                    ctypes.byref(h)), "bbc_server_create")
        self._h = h

    def submit(self, g) -> int:
        lib = load()
        u = np.ascontiguousarray(g.u, dtype=np.int32)
        v = np.ascontiguousarray(g.v, dtype=np.int32)
        s = np.ascontiguousarray(g.sign, dtype=np.int8)
        t = ctypes.c_uint64()
        check(lib.bbc_submit(self._h, int(g.n_u), int(g.n_v), int(u.shape[0]), u.ctypes.data,
                             v.ctypes.data, s.ctypes.data, ctypes.byref(t)), "bbc_submit")
        return int(t.value)

    def poll(self, ticket: int):
        """Returns the count, or None while the request is in flight."""
        b = ctypes.c_uint64()
        st = load().bbc_poll(self._h, ticket, ctypes.byref(b))
        if st == 11:
            return None
        check(st, "bbc_poll")
        return int(b.value)

    def wait(self, ticket: int, timeout_s: float = -1.0) -> int:
        b = ctypes.c_uint64()
        us = -1 if timeout_s < 0 else int(timeout_s * 1e6)
        check(load().bbc_wait(self._h, ticket, us, ctypes.byref(b)), "bbc_wait")
        return int(b.value)

    def stats(self) -> dict:
        c = ctypes.c_uint64()
        p50 = ctypes.c_double()
        p99 = ctypes.c_double()
        mean = ctypes.c_double()
        check(load().bbc_server_stats(self._h, ctypes.byref(c), ctypes.byref(p50), ctypes.byref(p99),
                                      ctypes.byref(mean)), "bbc_server_stats")
        return {"completed": c.value, "p50_us": p50.value, "p99_us": p99.value, "mean_us": mean.value}

    def counters(self) -> dict:
        c = ServerCounters()
        check(load().bbc_server_counters_get(self._h, ctypes.byref(c)), "bbc_server_counters_get")
        return c.as_dict()

    def request_info(self, ticket: int) -> dict:
        """What happened to one finished request (None while it is in flight)."""
        q = RequestInfo()
        st = load().bbc_server_request_info(self._h, ticket, ctypes.byref(q))
        if st == 11:
            return None
        check(st, "bbc_server_request_info")
        return q.as_dict()

    def close(self) -> None:
        if self._h.value:
            load().bbc_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CostModel:
    """The learned cost model of the tile kernel's work items (see include/bbc.h)."""

    def __init__(self, seed: int = 0):
        lib = load()
        h = ctypes.c_void_p()
        check(lib.bbc_cost_model_create(int(seed), ctypes.byref(h)), "bbc_cost_model_create")
        self._h = h

    @staticmethod
    def num_params() -> int:
        return int(load().bbc_cost_model_num_params())

    def get_params(self) -> np.ndarray:
        out = np.empty(self.num_params(), dtype=np.float32)
        check(load().bbc_cost_model_get_params(self._h, out.ctypes.data, out.shape[0]),
              "bbc_cost_model_get_params")
        return out

    def set_params(self, p) -> None:
        p = np.ascontiguousarray(p, dtype=np.float32)
        check(load().bbc_cost_model_set_params(self._h, p.ctypes.data, p.shape[0]),
              "bbc_cost_model_set_params")

    def loss_grad(self, X, t, stream=None):
        """(loss, gradient as float32 numpy) for device tensors X [n, 8] and t [n]."""
        loss = ctypes.c_float()
        g = np.empty(self.num_params(), dtype=np.float32)
        check(load().bbc_cost_model_loss_grad(self._h, X.data_ptr(), t.data_ptr(), int(X.shape[0]),
                                              ctypes.byref(loss), g.ctypes.data, _stream_ptr(stream)),
              "bbc_cost_model_loss_grad")
        return float(loss.value), g

    def fit(self, X, cycles, steps: int = 300, lr: float = 3e-3, stream=None) -> float:
        loss = ctypes.c_float()
        check(load().bbc_cost_model_fit(self._h, X.data_ptr(), cycles.data_ptr(), int(X.shape[0]),
                                        int(steps), float(lr), ctypes.byref(loss), _stream_ptr(stream)),
              "bbc_cost_model_fit")
        return float(loss.value)

    def predict(self, X, stream=None):
        import torch

        y = torch.empty(max(1, X.shape[0]), dtype=torch.float32, device="cuda")
        check(load().bbc_cost_model_predict(self._h, X.data_ptr(), int(X.shape[0]), y.data_ptr(),
                                            _stream_ptr(stream)), "bbc_cost_model_predict")
        return y[: X.shape[0]]

    def order(self, graph: "Graph", stream=None) -> None:
        check(load().bbc_cost_model_order(self._h, graph.handle, _stream_ptr(stream)),
              "bbc_cost_model_order")

    def free(self) -> None:
        if self._h.value:
            load().bbc_cost_model_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
