"""CPU oracle for the BBC large-k IVF search path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or runs it, and this package never
imports the product.

The arithmetic lives in ``bbc_oracle.c`` (plain C, single-threaded, FP64
except for the FP32 lookup-table recipe).  This module compiles it with gcc
(``-ffp-contract=off``) into ``oracle/_build`` and wraps it with ctypes.
Every function documents the passage of the paper it follows.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bbc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libbbc_oracle.so")
_lock = threading.Lock()
_lib = None

L2, IP = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libbbc_oracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Index(C.Structure):
    _fields_ = [("n", C.c_int64), ("d", C.c_int32), ("nlist", C.c_int32), ("metric", C.c_int32),
                ("M", C.c_int32), ("bits", C.c_int32),
                ("centroids", C.c_void_p), ("list_offsets", C.c_void_p), ("ids", C.c_void_p),
                ("codes", C.c_void_p), ("books", C.c_void_p), ("vectors", C.c_void_p),
                ("residual", C.c_int32), ("lut_levels", C.c_int32)]


class Codebook(C.Structure):
    """Result-buffer codebook (Section 3.2) plus the collector's final state."""
    _fields_ = [("d_min", C.c_uint32), ("d_max", C.c_uint32), ("sh", C.c_int32), ("m", C.c_int32),
                ("sample_lists", C.c_int32), ("sample_size", C.c_int64), ("tau", C.c_int32),
                ("pushed", C.c_int64), ("below", C.c_int64), ("map", C.c_uint8 * 256)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp, i32, i64, u32 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32
            L.oracle_dist.restype = C.c_double
            L.oracle_dist.argtypes = [vp, vp, i32, i32]
            L.oracle_probe.argtypes = [vp, vp, i32, i32, i32, i32, vp, vp]
            L.oracle_lut_f32.argtypes = [vp, vp, i32, i32, i32, i32, vp]
            L.oracle_lut16.argtypes = [vp, vp, i32, i32, i32, i32, vp, vp]
            L.oracle_lut_q.argtypes = [vp, vp, i32, i32, i32, i32, i32, vp, vp]
            L.oracle_adc.argtypes = [vp, vp, i64, i32, i32, vp]
            L.oracle_lut16_scale.restype = C.c_float
            L.oracle_lut16_scale.argtypes = [vp, vp, i32, i32, i32, i32, vp]
            L.oracle_resid_a.restype = C.c_float
            L.oracle_resid_a.argtypes = [vp, vp, i32, i32]
            L.oracle_resid_base.restype = i32
            L.oracle_resid_base.argtypes = [C.c_float, C.c_float]
            L.oracle_resid_w.restype = i32
            L.oracle_resid_w.argtypes = [C.c_float, C.c_float]
            L.oracle_resid_v.argtypes = [vp, vp, i64, vp, i32, i32, i32, i32, vp]
            L.oracle_adc_resid.argtypes = [vp, vp, i64, i32, i32, vp, vp, vp, i32, i32, C.c_float, vp]
            for f in (L.oracle_topkc_sort, L.oracle_topkc_heap):
                f.restype = i64
                f.argtypes = [vp, vp, i64, i64, vp, vp]
            L.oracle_update.restype = i32
            L.oracle_update.argtypes = [vp, i32, i64]
            L.oracle_build_codebook.argtypes = [vp, i64, i64, i32, C.POINTER(Codebook)]
            L.oracle_bucket_collect.restype = i64
            L.oracle_bucket_collect.argtypes = [vp, vp, vp, i32, i64, i32, i32,
                                                C.POINTER(Codebook), vp, vp, vp]
            L.oracle_rerank.argtypes = [vp, vp, i32, i32, vp, i64, vp]
            L.oracle_alg4.restype = i64
            L.oracle_alg4.argtypes = [vp, vp, vp, i32, i64, i32, i32, vp, vp, vp, vp]
            L.oracle_topk_final.argtypes = [vp, vp, i64, i32, vp, vp]
            L.oracle_bf16_bits.restype = C.c_uint16
            L.oracle_bf16_bits.argtypes = [C.c_float]
            L.oracle_bf16_value.restype = C.c_double
            L.oracle_bf16_value.argtypes = [C.c_uint16]
            L.oracle_e4m3_bits.restype = C.c_uint8
            L.oracle_e4m3_bits.argtypes = [C.c_float]
            L.oracle_e4m3_value.restype = C.c_double
            L.oracle_e4m3_value.argtypes = [C.c_uint8]
            L.oracle_prec_copy.argtypes = [vp, i64, i32, i32, i32, vp, vp]
            L.oracle_sign_encode.argtypes = [vp, i32, vp, i32, vp, vp, vp, vp, vp]
            L.oracle_rotation_eps.restype = C.c_double
            L.oracle_rotation_eps.argtypes = [vp, i32]
            L.oracle_sign_bounds.argtypes = [vp, i32, vp, vp, C.c_double, vp, vp, i64, C.c_double, vp, vp]
            L.oracle_sign_bounds_rq.argtypes = [vp, i32, vp, vp, C.c_double, vp, vp, i64, C.c_double, vp, vp]
            L.oracle_alg2.restype = i64
            L.oracle_alg2.argtypes = [vp, vp, vp, i64, i32, vp, vp]
            L.oracle_obs1_count.restype = i64
            L.oracle_obs1_count.argtypes = [vp, vp, vp, i64, i32]
            L.oracle_rounds.restype = i64
            L.oracle_rounds.argtypes = [vp, vp, vp, i64, i32, C.c_double, vp, vp]
            L.oracle_oneshot.restype = i64
            L.oracle_oneshot.argtypes = [vp, vp, i64, i32, vp, vp]
            L.oracle_search.restype = i32
            L.oracle_search.argtypes = [C.POINTER(_Index), vp, i64, i32, i32, i64, i32, i32, i32,
                                        vp, vp, vp]
            L.oracle_bruteforce.argtypes = [vp, i64, vp, i64, i32, i32, i32, vp, vp]
            _ = u32
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _metric(m) -> int:
    return m if isinstance(m, int) else (L2 if m == "l2" else IP)


# --------------------------------------------------------------------------
# step-by-step entry points
# --------------------------------------------------------------------------
def dist(a, b, metric="l2") -> float:
    """Squared L2 or negated inner product in FP64 (exact distance of Section 3.3)."""
    a, b = _f32(a), _f32(b)
    return lib().oracle_dist(_p(a), _p(b), a.shape[0], _metric(metric))


def probe(q, centroids, nprobe: int, metric="l2"):
    """IVF routing (Section 2): the nprobe nearest lists, nearest first, FP64 scores."""
    q, c = _f32(q), _f32(centroids)
    lists = np.empty(nprobe, dtype=np.int32)
    scores = np.empty(nprobe, dtype=np.float64)
    rc = lib().oracle_probe(_p(q), _p(c), c.shape[0], c.shape[1], _metric(metric), nprobe,
                            _p(lists), _p(scores))
    if rc:
        raise ValueError("bad nprobe")
    return lists, scores


def lut_f32(q, books, metric="l2"):
    """Per-sub-space query-to-codeword distances in FP32 (Section 2, step (1))."""
    q, b = _f32(q), _f32(books)
    M, K, ds = b.shape
    out = np.empty((M, K), dtype=np.float32)
    lib().oracle_lut_f32(_p(q), _p(b), M * ds, M, int(np.log2(K)), _metric(metric), _p(out))
    return out


def lut16(q, books, metric="l2", levels: int = 65535):
    """Integer-quantised lookup table (offset per sub-space, one scale per
    query) with entries in [0, levels]: the uint16 table at 65535, the table
    whose entries FP16 holds exactly at 2047."""
    q, b = _f32(q), _f32(books)
    M, K, ds = b.shape
    out = np.empty((M, K), dtype=np.uint16)
    if levels == 65535:
        lib().oracle_lut16(_p(q), _p(b), M * ds, M, int(np.log2(K)), _metric(metric), _p(out), None)
    else:
        lib().oracle_lut_q(_p(q), _p(b), M * ds, M, int(np.log2(K)), _metric(metric), int(levels), _p(out), None)
    return out


def adc(table16, codes, M: int, bits: int):
    """Integer estimated distances sum_m LUT16[m][code_m] (Section 2, step (2))."""
    t = np.ascontiguousarray(table16, dtype=np.uint16)
    c = np.ascontiguousarray(codes, dtype=np.uint8)
    out = np.empty(c.shape[0], dtype=np.uint32)
    lib().oracle_adc(_p(t), _p(c), c.shape[0], M, bits, _p(out))
    return out


def lut16_scale(q, books, metric="l2"):
    """The uint16 table's scale inv (integer units per unit of distance) and
    sum_m lo_m, the offsets the table drops."""
    q, b = _f32(q), _f32(books)
    M, K, ds = b.shape
    lo = C.c_double(0.0)
    inv = lib().oracle_lut16_scale(_p(q), _p(b), M * ds, M, int(np.log2(K)), _metric(metric), C.byref(lo))
    return float(np.float32(inv)), lo.value


def resid_a(q, c, metric="l2") -> float:
    """Residual IVF-PQ: the per-(query, list) term A_ql in FP32
    (||c||^2 - 2 <q, c> for L2, -<q, c> for IP)."""
    q, c = _f32(q), _f32(c)
    return float(np.float32(lib().oracle_resid_a(_p(q), _p(c), c.shape[0], _metric(metric))))


def resid_base(a: float, inv: float) -> int:
    """2^30 + rint(clamp(a * inv, +-2^29)) in the table's integer units."""
    return int(lib().oracle_resid_base(C.c_float(a), C.c_float(inv)))


def resid_w(v: float, inv: float) -> int:
    """rint(clamp(v * inv, +-2^28)) in the table's integer units."""
    return int(lib().oracle_resid_w(C.c_float(v), C.c_float(inv)))


def resid_v(c, codes, books, metric="l2"):
    """Residual IVF-PQ: the per-object term V_o = 2 <c, y_o> (L2; 0 for IP) of
    each code row of a list with centroid c, in FP32."""
    c, b = _f32(c), _f32(books)
    M, K, ds = b.shape
    cr = np.ascontiguousarray(codes, dtype=np.uint8)
    out = np.empty(cr.shape[0], dtype=np.float32)
    lib().oracle_resid_v(_p(c), _p(cr), cr.shape[0], _p(b), M * ds, M, int(np.log2(K)), _metric(metric),
                         _p(out))
    return out


def adc_resid(table16, codes, q, c, books, inv: float, metric="l2"):
    """Residual IVF-PQ keys of one list's code rows (the table sums plus the
    per-list and per-object terms, integer units)."""
    t = np.ascontiguousarray(table16, dtype=np.uint16)
    cr = np.ascontiguousarray(codes, dtype=np.uint8)
    q, c, b = _f32(q), _f32(c), _f32(books)
    M, K, ds = b.shape
    out = np.empty(cr.shape[0], dtype=np.uint32)
    lib().oracle_adc_resid(_p(t), _p(cr), cr.shape[0], M, int(np.log2(K)), _p(q), _p(c), _p(b), M * ds,
                           _metric(metric), C.c_float(inv), _p(out))
    return out


def topkc(e, ids, kc: int, how: str = "sort"):
    """The kc smallest (e, id), ascending; ``how`` = "sort" or "heap"."""
    e = np.ascontiguousarray(e, dtype=np.uint32)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    oi = np.empty(max(kc, 1), dtype=np.int64)
    oe = np.empty(max(kc, 1), dtype=np.uint32)
    f = lib().oracle_topkc_sort if how == "sort" else lib().oracle_topkc_heap
    c = f(_p(e), _p(ids), e.shape[0], kc, _p(oi), _p(oe))
    return oi[:c], oe[:c]


def update(counts, kc: int) -> int:
    """Algorithm 1 Update: first bucket whose running count reaches kc (m if none)."""
    c = np.ascontiguousarray(counts, dtype=np.int64)
    return int(lib().oracle_update(_p(c), c.shape[0], kc))


def build_codebook(sample_e, kc: int, m: int) -> Codebook:
    """Sampled equal-width -> equal-depth codebook of Section 3.2."""
    s = np.ascontiguousarray(sample_e, dtype=np.uint32)
    cb = Codebook()
    lib().oracle_build_codebook(_p(s), s.shape[0], kc, m, C.byref(cb))
    return cb


def bucket_collect(e, ids, list_ofs, kc: int, m: int, sample_min: int = 8):
    """Algorithm 1 Collect over lists in probe order.

    Returns (ids, e, codebook, counts) with ids/e ascending by (e, id).
    """
    e = np.ascontiguousarray(e, dtype=np.uint32)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    lo = np.ascontiguousarray(list_ofs, dtype=np.int64)
    cb = Codebook()
    counts = np.empty(m, dtype=np.int64)
    oi = np.empty(max(kc, 1), dtype=np.int64)
    oe = np.empty(max(kc, 1), dtype=np.uint32)
    c = lib().oracle_bucket_collect(_p(e), _p(ids), _p(lo), lo.shape[0] - 1, kc, m, sample_min,
                                    C.byref(cb), _p(counts), _p(oi), _p(oe))
    return oi[:c], oe[:c], cb, counts


def alg4(e, ids, list_ofs, kc: int, m: int, sample_min: int = 8):
    """Algorithm 4 (IVF+PQ with early re-ranking) over lists in probe order.

    Returns (candidate ids ascending by (e, id), early flag per candidate,
    objects scored early, early-scored objects among the candidates)."""
    e = np.ascontiguousarray(e, dtype=np.uint32)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    lo = np.ascontiguousarray(list_ofs, dtype=np.int64)
    oi = np.empty(max(kc, 1), dtype=np.int64)
    fl = np.zeros(max(kc, 1), dtype=np.uint8)
    ne, nec = C.c_int64(), C.c_int64()
    c = lib().oracle_alg4(_p(e), _p(ids), _p(lo), lo.shape[0] - 1, kc, m, sample_min, _p(oi), _p(fl),
                          C.byref(ne), C.byref(nec))
    return oi[:c], fl[:c].astype(bool), ne.value, nec.value


def rerank(q, vectors, ids, metric="l2"):
    """Exact FP64 distances of the candidates."""
    q, v = _f32(q), _f32(vectors)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    out = np.empty(ids.shape[0], dtype=np.float64)
    lib().oracle_rerank(_p(q), _p(v), v.shape[1], _metric(metric), _p(ids), ids.shape[0], _p(out))
    return out


def topk_final(dist_, ids, k: int):
    """The k smallest (dist, id), ascending; padded with (-1, +inf)."""
    dd = np.ascontiguousarray(dist_, dtype=np.float64)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    oi = np.empty(k, dtype=np.int64)
    od = np.empty(k, dtype=np.float64)
    lib().oracle_topk_final(_p(dd), _p(ids), dd.shape[0], k, _p(oi), _p(od))
    return oi, od


COLLECTORS = {"sort": 0, "heap": 1, "bucket": 2}


def search(index, queries, k: int, nprobe: int, kc: int, collector: str = "sort",
           m: int = 64, sample_min: int = 8, with_stats: bool = False, lut_levels: int = 65535):
    """The whole search path for a batch of queries (single-threaded).

    ``index`` is a ``synth.IvfPqIndex``-like object.  Returns (ids [nq, k],
    dists [nq, k] FP64) and, with ``with_stats``, per-query stats
    [S_q, candidates, tau, pushed].  ``lut_levels`` is the integer table's
    top level (65535: the uint16 table).
    """
    q = _f32(queries).reshape(-1, index.d)
    keep = []

    def arr(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return _p(a)

    ix = _Index(index.n, index.d, index.nlist, _metric(index.metric), index.pq_m, index.pq_bits,
                arr(index.centroids, np.float32), arr(index.list_offsets, np.int64),
                arr(index.ids, np.int64), arr(index.codes, np.uint8),
                arr(index.codebooks, np.float32), arr(index.vectors, np.float32),
                1 if getattr(index, "residual", False) else 0, int(lut_levels))
    nq = q.shape[0]
    oi = np.empty((nq, k), dtype=np.int64)
    od = np.empty((nq, k), dtype=np.float64)
    st = np.empty((nq, 4), dtype=np.int64)
    rc = lib().oracle_search(C.byref(ix), _p(q), nq, k, nprobe, kc, COLLECTORS[collector], m,
                             sample_min, _p(oi), _p(od), _p(st))
    if rc:
        raise ValueError(f"oracle_search: bad arguments (rc={rc})")
    return (oi, od, st) if with_stats else (oi, od)


def bruteforce(queries, x, k: int, metric="l2"):
    """Exact kNN over the whole data set in FP64: (ids [nq, k], dists [nq, k])."""
    q, xv = _f32(queries), _f32(x)
    q = q.reshape(-1, xv.shape[1])
    oi = np.empty((q.shape[0], k), dtype=np.int64)
    od = np.empty((q.shape[0], k), dtype=np.float64)
    lib().oracle_bruteforce(_p(q), q.shape[0], _p(xv), xv.shape[0], xv.shape[1], _metric(metric),
                            k, _p(oi), _p(od))
    return oi, od


# ---------------------------------------------------------------------------
# Low-precision copies for the precision form of the re-rank
# ---------------------------------------------------------------------------
def bf16_bits(x) -> np.ndarray:
    """bfloat16 bits of each FP32 value (nearest, ties to even)."""
    L = lib()
    x = np.ascontiguousarray(x, dtype=np.float32).ravel()
    return np.array([L.oracle_bf16_bits(float(v)) for v in x], dtype=np.uint16)


def bf16_value(bits) -> np.ndarray:
    L = lib()
    return np.array([L.oracle_bf16_value(int(b)) for b in np.ravel(bits)], dtype=np.float64)


def e4m3_bits(x) -> np.ndarray:
    """OCP E4M3 bits of each FP32 value (nearest, ties to even, saturating)."""
    L = lib()
    x = np.ascontiguousarray(x, dtype=np.float32).ravel()
    return np.array([L.oracle_e4m3_bits(float(v)) for v in x], dtype=np.uint8)


def e4m3_value(bits) -> np.ndarray:
    L = lib()
    return np.array([L.oracle_e4m3_value(int(b)) for b in np.ravel(bits)], dtype=np.float64)


def prec_copy(vectors: np.ndarray, prec: int, dpad: int | None = None):
    """Low-precision copy of the vectors (prec 1 BF16, 2 E4M3 with one scale
    per vector) and per-vector (s, e_v, ||x||, 0) in FP64.  Rows are padded
    with zeros to dpad (default: d rounded up to 16)."""
    v = np.ascontiguousarray(vectors, dtype=np.float32)
    n, d = v.shape
    dpad = dpad or (d + 15) // 16 * 16
    rows = np.zeros((n, dpad), dtype=np.uint16 if prec == 1 else np.uint8)
    meta = np.zeros((n, 4), dtype=np.float64)
    lib().oracle_prec_copy(_p(v), n, d, dpad, prec, _p(rows), _p(meta))
    return rows, meta


# ---------------------------------------------------------------------------
# 1-bit sign quantizer and the bounded re-rank (Section 3.4, Obs. 1, Alg. 2)
# ---------------------------------------------------------------------------
def sign_encode(index):
    """Codes (u32 [n, d/32], list order) and factors (f64 [n, 4] = alpha, e,
    ||o - c||^2, popcount) of the rotated residuals of an IVF sign index."""
    d = index.d
    codes = np.zeros((index.n, d // 32), dtype=np.uint32)
    fac = np.zeros((index.n, 4), dtype=np.float64)
    v, c, r = _f32(index.vectors), _f32(index.centroids), _f32(index.rotation)
    offs = np.ascontiguousarray(index.list_offsets, dtype=np.int64)
    ids = np.ascontiguousarray(index.ids, dtype=np.int64)
    lib().oracle_sign_encode(_p(v), d, _p(c), index.nlist, _p(offs), _p(ids), _p(r), _p(codes), _p(fac))
    return codes, fac


def rotation_eps(rot) -> float:
    r = _f32(rot)
    return float(lib().oracle_rotation_eps(_p(r), r.shape[0]))


def sign_bounds(q, centroid, rot, eps, codes, fac, scale: float = 1.0):
    """Bounds [lb, ub] on ||q - o||^2 for the objects whose codes / factors are given."""
    q, c, r = _f32(q), _f32(centroid), _f32(rot)
    codes = np.ascontiguousarray(codes, dtype=np.uint32)
    fac = np.ascontiguousarray(fac, dtype=np.float64)
    n = codes.shape[0]
    lb = np.empty(n, dtype=np.float64)
    ub = np.empty(n, dtype=np.float64)
    lib().oracle_sign_bounds(_p(q), q.shape[0], _p(c), _p(r), eps, _p(codes), _p(fac), n, scale, _p(lb), _p(ub))
    return lb, ub


def sign_bounds_rq(q, centroid, rot, eps, codes, fac, eps0: float = 1.9):
    """Bounds [lb, ub] on ||q - o||^2 from the RaBitQ estimator and its
    probabilistic error bound (epsilon_0 = eps0), for the given objects."""
    q, c, r = _f32(q), _f32(centroid), _f32(rot)
    codes = np.ascontiguousarray(codes, dtype=np.uint32)
    fac = np.ascontiguousarray(fac, dtype=np.float64)
    n = codes.shape[0]
    lb = np.empty(n, dtype=np.float64)
    ub = np.empty(n, dtype=np.float64)
    lib().oracle_sign_bounds_rq(_p(q), q.shape[0], _p(c), _p(r), eps, _p(codes), _p(fac), n, eps0, _p(lb), _p(ub))
    return lb, ub


def alg2(lb, ub, ex, k: int):
    """Algorithm 2: (number of exact distances computed, result indices)."""
    lb, ub, ex = (np.ascontiguousarray(a, dtype=np.float64) for a in (lb, ub, ex))
    n = lb.shape[0]
    out = np.empty(max(k, 1), dtype=np.int64)
    no = C.c_int64()
    cnt = lib().oracle_alg2(_p(lb), _p(ub), _p(ex), n, k, _p(out), C.byref(no))
    return int(cnt), out[:no.value].copy()


def obs1_count(lb, ub, ex, k: int) -> int:
    lb, ub, ex = (np.ascontiguousarray(a, dtype=np.float64) for a in (lb, ub, ex))
    return int(lib().oracle_obs1_count(_p(lb), _p(ub), _p(ex), lb.shape[0], k))


def oneshot(lb, ub, k: int):
    """One-pass classification: (|S|, |certainly in|, |to decide|)."""
    lb, ub = (np.ascontiguousarray(a, dtype=np.float64) for a in (lb, ub))
    a, b = C.c_int64(), C.c_int64()
    ns = lib().oracle_oneshot(_p(lb), _p(ub), lb.shape[0], k, C.byref(a), C.byref(b))
    return int(ns), a.value, b.value


def rounds(lb, ub, ex, k: int, first: float = 2.0):
    """Two-round bounded re-rank (first round: the first * k smallest interval
    centres of S): (exact distances computed, result indices sorted)."""
    lb, ub, ex = (np.ascontiguousarray(a, dtype=np.float64) for a in (lb, ub, ex))
    out = np.empty(max(k, 1), dtype=np.int64)
    no = C.c_int64()
    cnt = lib().oracle_rounds(_p(lb), _p(ub), _p(ex), lb.shape[0], k, float(first), _p(out), C.byref(no))
    return int(cnt), out[:no.value].copy()


def sign_encode_lists(index, lists):
    """Codes and factors for the objects of the given lists only (others zero),
    with the rotation applied as one FP64 matrix product per list (numpy); the
    same definitions as ``sign_encode``.  For preparing a bounded sample."""
    d = index.d
    codes = np.zeros((index.n, d // 32), dtype=np.uint32)
    fac = np.zeros((index.n, 4), dtype=np.float64)
    P = np.asarray(index.rotation, dtype=np.float64)
    for l in sorted(set(int(x) for x in np.ravel(lists))):
        a, b = int(index.list_offsets[l]), int(index.list_offsets[l + 1])
        if b == a:
            continue
        u = index.vectors[index.ids[a:b]].astype(np.float64) - index.centroids[l].astype(np.float64)
        r = u @ P.T
        s = np.where(r > 0, 1.0, -1.0)
        alpha = np.abs(r).sum(1) / d
        codes[a:b] = np.packbits(r > 0, axis=1, bitorder="little").view(np.uint32)
        fac[a:b, 0] = alpha
        fac[a:b, 1] = np.sqrt(((r - alpha[:, None] * s) ** 2).sum(1))
        fac[a:b, 2] = (u * u).sum(1)
        fac[a:b, 3] = (r > 0).sum(1)
    return codes, fac


def sign_search(index, queries, k: int, nprobe: int, scale: float = 1.0, codes=None, fac=None, eps=None,
                estimator: int = 0, eps0: float = 1.9, first: float = 2.0):
    """Bounded search over an IVF sign index (single-threaded).

    Probe as in ``search``; bounds for every object of the probed lists
    (estimator 0: the hard bounds, scaled by ``scale``; 1: the RaBitQ
    estimator's probabilistic bounds with epsilon_0 = eps0).  With hard bounds
    the result is the k smallest (exact FP64 distance, id) of the probed lists;
    with the estimator's bounds it is what the two-round bounded re-rank
    returns on them (which differs from the exact top-k only where a bound
    fails).  Returns (ids [nq, k], dists [nq, k]) and per-query stats [S_q,
    |S|, |certainly in|, |to decide|, Alg. 2 count, Obs. 1 count, two-round
    count]."""
    if codes is None:
        codes, fac = sign_encode(index)
    if eps is None:
        eps = rotation_eps(index.rotation)
    q = _f32(queries).reshape(-1, index.d)
    nq = q.shape[0]
    oi = np.empty((nq, k), dtype=np.int64)
    od = np.empty((nq, k), dtype=np.float64)
    st = np.zeros((nq, 7), dtype=np.int64)
    offs = index.list_offsets
    for i in range(nq):
        lists, _ = probe(q[i], index.centroids, nprobe, index.metric)
        lbs, ubs, sel = [], [], []
        for l in lists:
            a, b = offs[l], offs[l + 1]
            if estimator:
                lb, ub = sign_bounds_rq(q[i], index.centroids[l], index.rotation, eps, codes[a:b], fac[a:b], eps0)
            else:
                lb, ub = sign_bounds(q[i], index.centroids[l], index.rotation, eps, codes[a:b], fac[a:b], scale)
            lbs.append(lb); ubs.append(ub); sel.append(np.arange(a, b))
        lb, ub, sel = np.concatenate(lbs), np.concatenate(ubs), np.concatenate(sel)
        gid = index.ids[sel]
        ex = rerank(q[i], index.vectors, gid, index.metric)
        oi[i], od[i] = topk_final(ex, gid, k)
        ns, nin, nr = oneshot(lb, ub, k)
        a2, _ = alg2(lb, ub, ex, k)
        rc, ridx = rounds(lb, ub, ex, k, first)
        if scale >= 1.0 and not estimator and not np.array_equal(gid[ridx], oi[i][:len(ridx)]):
            raise AssertionError("two-round bounded re-rank disagrees with the exact top-k")
        if estimator:
            # the bounded procedure's own result on the estimator's bounds
            oi[i] = -1
            od[i] = np.inf
            oi[i][:len(ridx)] = gid[ridx]
            od[i][:len(ridx)] = ex[ridx]
        st[i] = [len(sel), ns, nin, nr, a2, obs1_count(lb, ub, ex, k), rc]
    return oi, od, st
