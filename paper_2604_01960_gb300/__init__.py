"""GB300 (sm_103a) search path for large-k ANN queries on IVF-PQ indexes with
a bucket-based result collector (BBC, arxiv 2604.01960).

This module is a thin ctypes binding over ``libbbc.so`` (the C ABI in
``include/bbc.h``): it marshals pointers and sizes and nothing else.  Every
step of the search runs in the library's CUDA kernels; there is no CPU or
PyTorch fallback.  Importing this package does not need a GPU, but loading
the library does need the compiled ``libbbc.so`` (``build()`` makes it), and
calling into it needs a CUDA device.  PyTorch is used for device memory and
streams only.
"""

from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbbc.so")

BBC_OK = 0
ERRORS = {-1: "BBC_ERR_ARG", -2: "BBC_ERR_IO", -3: "BBC_ERR_FORMAT", -4: "BBC_ERR_OOM", -5: "BBC_ERR_CUDA",
          -6: "BBC_ERR_CAPACITY", -7: "BBC_ERR_TIMEOUT", -8: "BBC_ERR_BUSY", -9: "BBC_ERR_UNSUPPORTED"}
METRICS = {"l2": 0, "ip": 1}

# Exported symbols declared in include/bbc.h (checked by the ABI test).
SYMBOLS = ["bbc_index_create", "bbc_index_create_sign", "bbc_index_load", "bbc_index_free", "bbc_index_info", "bbc_set_param",
           "bbc_get_param", "bbc_search", "bbc_search_ex", "bbc_search_host", "bbc_probe_scores", "bbc_probe", "bbc_lut", "bbc_collect", "bbc_collect_static",
           "bbc_rerank_topk", "bbc_rerank_bounds", "bbc_precision_copy", "bbc_precision_stats", "bbc_early_stats", "bbc_sign_bounds", "bbc_bounded_stats", "bbc_autotune", "bbc_serve_start", "bbc_serve_submit", "bbc_serve_poll",
           "bbc_serve_stats", "bbc_serve_stop", "bbc_profile_read", "bbc_stream_status", "bbc_last_error", "bbc_version"]
NUM_STAGES = 9
STAGES = ["probe_scores", "probe_select", "lut", "scan", "select", "rerank", "topk", "prec_classify",
          "prec_recheck"]


class BBCError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class IndexHost(C.Structure):
    _fields_ = [("n", C.c_int64), ("d", C.c_int32), ("nlist", C.c_int32), ("metric", C.c_int32),
                ("pq_m", C.c_int32), ("pq_bits", C.c_int32), ("centroids", C.c_void_p),
                ("list_offsets", C.c_void_p), ("ids", C.c_void_p), ("codes", C.c_void_p),
                ("codebooks", C.c_void_p), ("vectors", C.c_void_p), ("residual", C.c_int32)]


class IndexInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("d", C.c_int32), ("nlist", C.c_int32), ("metric", C.c_int32),
                ("pq_m", C.c_int32), ("pq_bits", C.c_int32), ("max_list_len", C.c_int32),
                ("vectors_u8_exact", C.c_int32), ("device", C.c_int32), ("device_bytes", C.c_int64),
                ("quantizer", C.c_int32), ("reserved", C.c_int32)]


class SignHost(C.Structure):
    _fields_ = [("n", C.c_int64), ("d", C.c_int32), ("nlist", C.c_int32), ("metric", C.c_int32),
                ("centroids", C.c_void_p), ("list_offsets", C.c_void_p), ("ids", C.c_void_p),
                ("rotation", C.c_void_p), ("vectors", C.c_void_p)]


class ServeConfig(C.Structure):
    _fields_ = [("max_batch", C.c_int32), ("streams", C.c_int32), ("cand_bytes_budget", C.c_int64)]


class ServeStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("batches", C.c_int64),
                ("inflight_bytes_peak", C.c_int64), ("p50_ms", C.c_double), ("p99_ms", C.c_double),
                ("mean_batch", C.c_double), ("wall_s", C.c_double)]


class CollectorState(C.Structure):
    _fields_ = [("d_min", C.c_uint32), ("d_max", C.c_uint32), ("sh", C.c_int32), ("m", C.c_int32),
                ("sample_lists", C.c_int32), ("tau", C.c_int32), ("sample_size", C.c_int64),
                ("scanned", C.c_int64), ("pushed", C.c_int64), ("below", C.c_int64), ("kc", C.c_int64),
                ("hist", C.c_uint32 * 256), ("map", C.c_uint8 * 256)]


STATE_DTYPE = np.dtype([("d_min", "<u4"), ("d_max", "<u4"), ("sh", "<i4"), ("m", "<i4"),
                        ("sample_lists", "<i4"), ("tau", "<i4"), ("sample_size", "<i8"),
                        ("scanned", "<i8"), ("pushed", "<i8"), ("below", "<i8"), ("kc", "<i8"),
                        ("hist", "<u4", (256,)), ("map", "u1", (256,))], align=True)
assert STATE_DTYPE.itemsize == C.sizeof(CollectorState)

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile libbbc.so for sm_103a in-tree."""
    from . import _build
    return _build.build(force=force)


def lib():
    """Load libbbc.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libbbc.so not found at {LIB_PATH}: run paper_2604_01960_gb300.build()")
            L = C.CDLL(LIB_PATH)
            vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
            L.bbc_last_error.restype = C.c_char_p
            L.bbc_version.restype = C.c_char_p
            L.bbc_index_create.argtypes = [C.POINTER(IndexHost), C.c_int, C.POINTER(vp)]
            L.bbc_index_load.argtypes = [C.c_char_p, C.c_int, C.POINTER(vp)]
            L.bbc_index_create_sign.argtypes = [C.POINTER(SignHost), C.c_int, C.POINTER(vp)]
            L.bbc_sign_bounds.argtypes = [vp, vp, i64, i32, vp, i64, vp, vp, vp, vp]
            L.bbc_bounded_stats.argtypes = [vp, vp, C.c_int]
            L.bbc_early_stats.argtypes = [vp, vp, C.c_int]
            L.bbc_index_free.argtypes = [vp]
            L.bbc_index_info.argtypes = [vp, C.POINTER(IndexInfo)]
            L.bbc_set_param.argtypes = [vp, C.c_char_p, C.c_double]
            L.bbc_get_param.argtypes = [vp, C.c_char_p, C.POINTER(C.c_double)]
            L.bbc_search.argtypes = [vp, vp, i64, i32, i32, vp, vp, vp]
            L.bbc_search_host.argtypes = [vp, vp, i64, i32, i32, vp, vp, vp]
            L.bbc_search_ex.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp]
            L.bbc_probe.argtypes = [vp, vp, i64, i32, vp, vp]
            L.bbc_probe_scores.argtypes = [vp, vp, i64, vp, vp]
            L.bbc_lut.argtypes = [vp, vp, i64, vp, vp]
            L.bbc_collect.argtypes = [vp, vp, i64, i32, vp, i64, vp, vp, vp, vp]
            L.bbc_collect_static.argtypes = [vp, vp, i64, i32, vp, i64, vp, vp, vp, vp]
            L.bbc_rerank_topk.argtypes = [vp, vp, i64, vp, vp, i64, i32, vp, vp, vp]
            L.bbc_rerank_bounds.argtypes = [vp, vp, i64, vp, vp, i64, vp, vp, vp]
            L.bbc_precision_copy.argtypes = [vp, vp, vp, vp]
            L.bbc_precision_stats.argtypes = [vp, vp, C.c_int]
            L.bbc_stream_status.argtypes = [vp, vp]
            L.bbc_profile_read.argtypes = [vp, vp, vp, C.c_int]
            L.bbc_autotune.argtypes = [vp, vp, i64, i32, i32, C.c_char_p, vp, vp]
            L.bbc_serve_start.argtypes = [vp, C.POINTER(ServeConfig), C.POINTER(vp)]
            L.bbc_serve_submit.argtypes = [vp, vp, i32, i32, C.POINTER(C.c_uint64)]
            L.bbc_serve_poll.argtypes = [vp, C.c_uint64, vp, vp, i32]
            L.bbc_serve_stats.argtypes = [vp, C.POINTER(ServeStats)]
            L.bbc_serve_stop.argtypes = [vp]
            for name in SYMBOLS:
                if getattr(L, name).restype is None and name not in ("bbc_last_error", "bbc_version"):
                    getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def _check(rc: int):
    if rc != BBC_OK:
        raise BBCError(rc, lib().bbc_last_error().decode())


def _ptr(x) -> int | None:
    """Device/host address of a torch tensor or numpy array (no copies)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------------------
# C-ABI wrappers with the C names
# ---------------------------------------------------------------------------
def bbc_index_create(index, device: int = 0) -> int:
    """Create a device index from a host IVF-PQ index object (numpy arrays;
    ``residual`` true: its codes quantise o - c_l), or from an IVF
    sign-quantizer index (one with a ``rotation``)."""
    if hasattr(index, "rotation"):
        return bbc_index_create_sign(index, device)
    keep = []

    def arr(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a.ctypes.data

    h = IndexHost(int(index.n), int(index.d), int(index.nlist), METRICS[index.metric], int(index.pq_m),
                  int(index.pq_bits), arr(index.centroids, np.float32), arr(index.list_offsets, np.int64),
                  arr(index.ids, np.int64), arr(index.codes, np.uint8), arr(index.codebooks, np.float32),
                  arr(index.vectors, np.float32), 1 if getattr(index, "residual", False) else 0)
    out = C.c_void_p()
    _check(lib().bbc_index_create(C.byref(h), device, C.byref(out)))
    return out.value


def bbc_index_create_sign(index, device: int = 0) -> int:
    """Create a device index with 1-bit sign codes from IVF lists and a rotation."""
    keep = []

    def arr(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a.ctypes.data

    h = SignHost(int(index.n), int(index.d), int(index.nlist), METRICS[index.metric],
                 arr(index.centroids, np.float32), arr(index.list_offsets, np.int64), arr(index.ids, np.int64),
                 arr(index.rotation, np.float32), arr(index.vectors, np.float32))
    out = C.c_void_p()
    _check(lib().bbc_index_create_sign(C.byref(h), device, C.byref(out)))
    return out.value


def bbc_index_load(path: str, device: int = 0) -> int:
    out = C.c_void_p()
    _check(lib().bbc_index_load(path.encode(), device, C.byref(out)))
    return out.value


def bbc_index_free(handle: int) -> None:
    _check(lib().bbc_index_free(handle))


def bbc_index_info(handle: int) -> dict:
    info = IndexInfo()
    _check(lib().bbc_index_info(handle, C.byref(info)))
    return {f: getattr(info, f) for f, _ in IndexInfo._fields_}


def bbc_set_param(handle: int, key: str, value: float) -> None:
    _check(lib().bbc_set_param(handle, key.encode(), float(value)))


def bbc_get_param(handle: int, key: str) -> float:
    v = C.c_double()
    _check(lib().bbc_get_param(handle, key.encode(), C.byref(v)))
    return v.value


def bbc_search(handle: int, queries, nq: int, k: int, nprobe: int, out_ids, out_dists, stream=None) -> None:
    _check(lib().bbc_search(handle, _ptr(queries), nq, k, nprobe, _ptr(out_ids), _ptr(out_dists), _stream(stream)))


def bbc_search_ex(handle: int, queries, nq: int, k, nprobe, out_ids, out_dists, stream=None) -> None:
    """Mixed batch: k and nprobe are host int32 arrays of length nq; outputs packed by prefix sums of k."""
    ka = np.ascontiguousarray(k, dtype=np.int32)
    pa = np.ascontiguousarray(nprobe, dtype=np.int32)
    _check(lib().bbc_search_ex(handle, _ptr(queries), nq, ka.ctypes.data, pa.ctypes.data, _ptr(out_ids),
                               _ptr(out_dists), _stream(stream)))


def bbc_search_host(handle: int, queries, nq: int, k: int, nprobe: int, out_ids, out_dists, stream=None) -> None:
    _check(lib().bbc_search_host(handle, _ptr(queries), nq, k, nprobe, _ptr(out_ids), _ptr(out_dists),
                                 _stream(stream)))


def bbc_probe_scores(handle: int, queries, nq: int, out_scores, stream=None) -> None:
    _check(lib().bbc_probe_scores(handle, _ptr(queries), nq, _ptr(out_scores), _stream(stream)))


def bbc_probe(handle: int, queries, nq: int, nprobe: int, out_lists, stream=None) -> None:
    _check(lib().bbc_probe(handle, _ptr(queries), nq, nprobe, _ptr(out_lists), _stream(stream)))


def bbc_lut(handle: int, queries, nq: int, out_lut16, stream=None) -> None:
    _check(lib().bbc_lut(handle, _ptr(queries), nq, _ptr(out_lut16), _stream(stream)))


def bbc_collect(handle: int, queries, nq: int, nprobe: int, probe_lists, kc: int, out_ids, out_count,
                out_state=None, stream=None) -> None:
    _check(lib().bbc_collect(handle, _ptr(queries), nq, nprobe, _ptr(probe_lists), kc, _ptr(out_ids),
                             _ptr(out_count), _ptr(out_state), _stream(stream)))


def bbc_collect_static(handle: int, queries, nq: int, nprobe: int, probe_lists, kc: int, out_ids, out_count,
                       out_state=None, stream=None) -> None:
    """bbc_collect without any allocation: scratch comes from the library's static device array.

    For callers that must not allocate device memory (see include/bbc.h)."""
    _check(lib().bbc_collect_static(handle, _ptr(queries), nq, nprobe, _ptr(probe_lists), kc, _ptr(out_ids),
                                    _ptr(out_count), _ptr(out_state), _stream(stream)))


def bbc_rerank_topk(handle: int, queries, nq: int, cand_ids, cand_count, kc: int, k: int, out_ids, out_dists,
                    stream=None) -> None:
    _check(lib().bbc_rerank_topk(handle, _ptr(queries), nq, _ptr(cand_ids), _ptr(cand_count), kc, k,
                                 _ptr(out_ids), _ptr(out_dists), _stream(stream)))


def bbc_rerank_bounds(handle: int, queries, nq: int, cand_ids, cand_count, kc: int, out_dist, out_rho,
                      stream=None) -> None:
    """Scores of the candidates from the low-precision copy and their bounds."""
    _check(lib().bbc_rerank_bounds(handle, _ptr(queries), nq, _ptr(cand_ids), _ptr(cand_count), kc,
                                   _ptr(out_dist), _ptr(out_rho), _stream(stream)))


def bbc_precision_copy(handle: int, out_rows, out_meta, stream=None) -> None:
    _check(lib().bbc_precision_copy(handle, _ptr(out_rows), _ptr(out_meta), _stream(stream)))


def bbc_precision_stats(handle: int, reset: bool = True) -> dict:
    """Totals of the precision re-rank since the last reset."""
    t = (C.c_int64 * 4)()
    _check(lib().bbc_precision_stats(handle, t, 1 if reset else 0))
    return {"scored": t[0], "fp32_rechecked": t[1], "fp64_scored": t[2], "final": t[3]}


def bbc_sign_bounds(handle: int, queries, nq: int, nprobe: int, probe_lists, stride: int, out_lb, out_ub,
                    out_count, stream=None) -> None:
    """Bounds of every object of the probed lists (sign-code index), probe order."""
    _check(lib().bbc_sign_bounds(handle, _ptr(queries), nq, nprobe, _ptr(probe_lists), stride, _ptr(out_lb),
                                 _ptr(out_ub), _ptr(out_count), _stream(stream)))


def bbc_bounded_stats(handle: int, reset: bool = True) -> dict:
    """Totals of the bounded re-rank since the last reset."""
    t = (C.c_int64 * 4)()
    _check(lib().bbc_bounded_stats(handle, t, 1 if reset else 0))
    return {"scanned": t[0], "in_S": t[1], "exact": t[2], "queries": t[3]}


def bbc_early_stats(handle: int, reset: bool = True) -> dict:
    """Totals of the early re-rank since the last reset."""
    t = (C.c_int64 * 2)()
    _check(lib().bbc_early_stats(handle, t, 1 if reset else 0))
    return {"scored_early": t[0], "used": t[1]}


def bbc_profile_read(handle: int, reset: bool = True):
    """(per-stage milliseconds dict, kernels launched) since the last reset."""
    ms = (C.c_double * NUM_STAGES)()
    n = C.c_int64()
    _check(lib().bbc_profile_read(handle, ms, C.byref(n), 1 if reset else 0))
    return dict(zip(STAGES, list(ms))), n.value


def bbc_autotune(handle: int, queries, nq: int, k: int, nprobe: int, cache_path: str | None = None,
                 stream=None) -> float:
    """Pick 'split' and 'buckets' for this call shape; returns the best ms per call (0 if cached)."""
    ms = C.c_double()
    _check(lib().bbc_autotune(handle, _ptr(queries), nq, k, nprobe, cache_path.encode() if cache_path else None,
                              C.byref(ms), _stream(stream)))
    return ms.value


def bbc_serve_start(handle: int, max_batch: int = 256, streams: int = 4, cand_bytes_budget: int = 8 << 30) -> int:
    out = C.c_void_p()
    cfg = ServeConfig(max_batch, streams, cand_bytes_budget)
    _check(lib().bbc_serve_start(handle, C.byref(cfg), C.byref(out)))
    return out.value


def bbc_serve_submit(server: int, host_query, k: int, nprobe: int) -> int:
    qa = np.ascontiguousarray(host_query, dtype=np.float32)
    t = C.c_uint64()
    _check(lib().bbc_serve_submit(server, qa.ctypes.data, k, nprobe, C.byref(t)))
    return t.value


def bbc_serve_poll(server: int, ticket: int, k: int, timeout_ms: int = -1):
    """(ids int64[k], dists float32[k]) once ready; raises BBCError(-7) on timeout."""
    ids = np.empty(k, dtype=np.int64)
    dd = np.empty(k, dtype=np.float32)
    _check(lib().bbc_serve_poll(server, ticket, ids.ctypes.data, dd.ctypes.data, timeout_ms))
    return ids, dd


def bbc_serve_stats(server: int) -> dict:
    st = ServeStats()
    _check(lib().bbc_serve_stats(server, C.byref(st)))
    return {f: getattr(st, f) for f, _ in ServeStats._fields_}


def bbc_serve_stop(server: int) -> None:
    _check(lib().bbc_serve_stop(server))


def bbc_stream_status(handle: int, stream=None) -> None:
    _check(lib().bbc_stream_status(handle, _stream(stream)))


def bbc_version() -> str:
    return lib().bbc_version().decode()


# ---------------------------------------------------------------------------
# Convenience object over the same calls (torch tensors in, torch tensors out)
# ---------------------------------------------------------------------------
class Index:
    """Owns one device index.  ``search`` takes a CUDA f32 tensor [nq, d]."""

    def __init__(self, host_index=None, path: str | None = None, device: int = 0):
        import torch
        self.device = torch.device("cuda", device)
        self.handle = bbc_index_load(path, device) if path else bbc_index_create(host_index, device)
        self.info = bbc_index_info(self.handle)

    def set(self, **params):
        for k, v in params.items():
            bbc_set_param(self.handle, k, v)
        return self

    def get(self, key: str) -> float:
        return bbc_get_param(self.handle, key)

    def search(self, queries, k: int, nprobe: int, stream=None):
        import torch
        q = queries.contiguous()
        nq = q.shape[0]
        ids = torch.empty((nq, k), dtype=torch.int64, device=q.device)
        dists = torch.empty((nq, k), dtype=torch.float32, device=q.device)
        bbc_search(self.handle, q, nq, k, nprobe, ids, dists, stream)
        return ids, dists

    def kc(self, k: int) -> int:
        import math
        return max(k, int(math.ceil(self.get("kc_ratio") * k - 1e-9)))

    def close(self):
        if self.handle:
            bbc_index_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
