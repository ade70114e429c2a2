"""Offline IVF index construction over synthetic data (seeded, deterministic).

The index is an input to the search path, built once before any query runs:

* IVF: k-means centroids (seed 3); every vector goes to its nearest centroid's
  inverted list (the paper's indexing phase, Section 2 "Quantization").
* PQ: product quantisation, M sub-spaces of d/M dimensions with 2^b
  codewords each, trained by k-means on raw sub-vectors (seed 4); or, for a
  residual index, on the sub-vectors of o - c_l, the residual to the list's
  centroid, which the codes then quantise.
* Sign quantizer: IVF lists plus a seeded random rotation (seed 5); the sign
  codes of each rotated residual and their per-vector factors are derived
  from these by the library and by the oracle, each on its own (see
  ``build_ivf_sign``).

Lists keep vectors in ascending id order.  The canonical code layout is one
row per vector in list order; for 8-bit PQ byte m holds sub-space m, for
4-bit PQ byte m/2 holds sub-space m in its low nibble when m is even and in
its high nibble when m is odd.

File format (little-endian, written by ``write_index``): a 64-byte header
``b"BBCIDX01"``, u32 version, u32 quantizer (0 PQ, 1 sign, 2 residual PQ), u32 metric
(0 L2, 1 IP), u32 d, u64 n, u32 nlist, u32 pq_m, u32 pq_bits, then padding;
followed by the arrays, each starting on a 64-byte boundary, in this order:
centroids f32[nlist*d], list_offsets i64[nlist+1], ids i64[n] (list order),
codes u8[n*code_bytes] (list order), codebooks f32[pq_m*2^b*(d/pq_m)],
vectors f32[n*d] (id order).  A sign-quantizer index (quantizer 1, pq_m and
pq_bits 0, written by ``write_sign_index``) stores centroids, list_offsets,
ids, the rotation f32[d*d] (row-major, r = P u) and vectors, in that order.
"""

from __future__ import annotations

import dataclasses
import struct

import numpy as np

SEED_KMEANS = 3
SEED_PQ = 4
SEED_ROT = 5

MAGIC = b"BBCIDX01"
HEADER_FMT = "<8sIIIIQIII"  # magic, version, quantizer, metric, d, n, nlist, pq_m, pq_bits
HEADER_BYTES = 64


def _sqnorms(x: np.ndarray) -> np.ndarray:
    return np.einsum("ij,ij->i", x, x, dtype=np.float32)


def nearest(x: np.ndarray, c: np.ndarray, chunk: int = 1 << 16, device: str | None = None) -> np.ndarray:
    """Index of the nearest row of ``c`` (squared L2) for each row of ``x``.

    Runs through torch (multi-threaded on CPU, or on ``device``) in FP32;
    the result only has to be deterministic for a given machine.
    """
    import torch
    dev = torch.device(device or _DEVICE)
    ct = torch.from_numpy(np.ascontiguousarray(c, dtype=np.float32)).to(dev)
    cn = (ct * ct).sum(1)
    out = np.empty(x.shape[0], dtype=np.int64)
    for s in range(0, x.shape[0], chunk):
        xs = torch.from_numpy(np.ascontiguousarray(x[s:s + chunk], dtype=np.float32)).to(dev)
        dist = cn[None, :] - 2.0 * (xs @ ct.T)
        out[s:s + chunk] = torch.argmin(dist, dim=1).cpu().numpy()
    return out


_DEVICE = "cpu"


def set_build_device(device: str) -> None:
    """Run the index builder's nearest-centroid searches on ``device`` (e.g. "cuda")."""
    global _DEVICE
    _DEVICE = device


def kmeans(x: np.ndarray, k: int, iters: int = 12, seed: int = SEED_KMEANS,
           sample: int | None = None) -> np.ndarray:
    """Lloyd's k-means with a seeded initialisation from the data."""
    rng = np.random.default_rng(seed)
    n = x.shape[0]
    if sample is not None and sample < n:
        train = x[np.sort(rng.choice(n, size=sample, replace=False))]
    else:
        train = x
    nt = train.shape[0]
    if nt < k:
        raise ValueError(f"k-means needs at least k={k} points, got {nt}")
    cent = train[rng.choice(nt, size=k, replace=False)].astype(np.float32).copy()
    for _ in range(iters):
        assign = nearest(train, cent)
        counts = np.bincount(assign, minlength=k)
        sums = np.zeros((k, train.shape[1]), dtype=np.float64)
        np.add.at(sums, assign, train) if nt < 4096 else _segment_sum(sums, assign, train)
        nz = counts > 0
        cent[nz] = (sums[nz] / counts[nz, None]).astype(np.float32)
        empty = np.flatnonzero(~nz)
        if empty.size:
            cent[empty] = train[rng.choice(nt, size=empty.size, replace=False)]
    return cent


def _segment_sum(sums: np.ndarray, assign: np.ndarray, x: np.ndarray) -> None:
    order = np.argsort(assign, kind="stable")
    a = assign[order]
    starts = np.flatnonzero(np.r_[True, a[1:] != a[:-1]])
    red = np.add.reduceat(x[order].astype(np.float64), starts, axis=0)
    sums[a[starts]] = red


@dataclasses.dataclass
class IvfPqIndex:
    metric: str                 # "l2" or "ip"
    d: int
    nlist: int
    pq_m: int
    pq_bits: int
    centroids: np.ndarray       # f32 [nlist, d]
    list_offsets: np.ndarray    # i64 [nlist + 1]
    ids: np.ndarray             # i64 [n], list order
    codes: np.ndarray           # u8 [n, code_bytes], list order, canonical layout
    codebooks: np.ndarray       # f32 [pq_m, 2^pq_bits, d / pq_m]
    vectors: np.ndarray         # f32 [n, d], id order
    residual: bool = False      # codes quantise o - c_l (residual IVF-PQ)

    @property
    def n(self) -> int:
        return int(self.vectors.shape[0])

    @property
    def code_bytes(self) -> int:
        return self.pq_m * self.pq_bits // 8

    @property
    def list_sizes(self) -> np.ndarray:
        return np.diff(self.list_offsets)


def _pack4(codes: np.ndarray) -> np.ndarray:
    lo = codes[:, 0::2].astype(np.uint8)
    hi = codes[:, 1::2].astype(np.uint8)
    return (lo | (hi << 4)).astype(np.uint8)


def unpack_codes(codes: np.ndarray, pq_m: int, pq_bits: int) -> np.ndarray:
    """Canonical code rows -> one integer code per sub-space, shape [n, pq_m]."""
    if pq_bits == 8:
        return codes.astype(np.int64)
    out = np.empty((codes.shape[0], pq_m), dtype=np.int64)
    out[:, 0::2] = codes & 0x0F
    out[:, 1::2] = codes >> 4
    return out


def _inverted_lists(assign: np.ndarray, nlist: int):
    order = np.argsort(assign, kind="stable")          # ascending id inside each list
    counts = np.bincount(assign, minlength=nlist)
    offsets = np.zeros(nlist + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    return order.astype(np.int64), offsets


def _nearest_dev(x, c, chunk: int):
    """Nearest row of c for each row of x, both torch tensors on one device."""
    import torch
    cn = (c * c).sum(1)
    out = torch.empty(x.shape[0], dtype=torch.int64, device=x.device)
    for s in range(0, x.shape[0], chunk):
        out[s:s + chunk] = torch.argmin(cn[None, :] - 2.0 * (x[s:s + chunk] @ c.T), dim=1)
    return out


def _kmeans_dev(train, k: int, iters: int, rng, chunk: int):
    """Lloyd's k-means on the device; same seeded initialisation as ``kmeans``."""
    import torch
    nt, d = train.shape
    if nt < k:
        raise ValueError(f"k-means needs at least k={k} points, got {nt}")
    pick = torch.from_numpy(rng.choice(nt, size=k, replace=False)).to(train.device)
    cent = train[pick].clone()
    for _ in range(iters):
        assign = _nearest_dev(train, cent, chunk)
        counts = torch.bincount(assign, minlength=k)
        sums = torch.zeros((k, d), dtype=torch.float64, device=train.device)
        for s in range(0, nt, 1 << 20):
            sums.index_add_(0, assign[s:s + (1 << 20)], train[s:s + (1 << 20)].double())
        nz = counts > 0
        cent[nz] = (sums[nz] / counts[nz, None]).float()
        empty = torch.nonzero(~nz).flatten()
        if empty.numel():
            repl = torch.from_numpy(rng.choice(nt, size=int(empty.numel()), replace=False)).to(train.device)
            cent[empty] = train[repl]
    return cent


def _build_ivf_pq_dev(x, nlist, pq_m, pq_bits, metric, kmeans_iters, pq_iters, kmeans_sample, pq_sample,
                      residual=False):
    """The same construction as ``build_ivf_pq`` with torch on the build device
    (for large inputs); results are deterministic for a given machine."""
    import torch
    n, d = x.shape
    dev = torch.device(_DEVICE)
    xt = torch.from_numpy(x).to(dev)
    rng = np.random.default_rng(SEED_KMEANS)
    if kmeans_sample < n:
        sel = torch.from_numpy(np.sort(rng.choice(n, size=kmeans_sample, replace=False))).to(dev)
        train = xt[sel]
    else:
        train = xt
    cent = _kmeans_dev(train, nlist, kmeans_iters, rng, 1 << 15)
    del train
    assign = _nearest_dev(xt, cent, 1 << 15).cpu().numpy()
    ids, offsets = _inverted_lists(assign, nlist)
    if residual:
        xt = xt - cent[torch.from_numpy(assign).to(dev)]
    dsub, ksub = d // pq_m, 1 << pq_bits
    rng = np.random.default_rng(SEED_PQ)
    samp = xt[torch.from_numpy(np.sort(rng.choice(n, size=min(n, pq_sample), replace=False))).to(dev)]
    books = np.empty((pq_m, ksub, dsub), dtype=np.float32)
    codes_full = torch.empty((n, pq_m), dtype=torch.uint8, device=dev)
    for m in range(pq_m):
        sub = samp[:, m * dsub:(m + 1) * dsub].contiguous()
        bk = _kmeans_dev(sub, ksub, pq_iters, np.random.default_rng(SEED_PQ + 17 * m), 1 << 20)
        books[m] = bk.cpu().numpy()
        codes_full[:, m] = _nearest_dev(xt[:, m * dsub:(m + 1) * dsub], bk, 1 << 20).to(torch.uint8)
    codes_full = codes_full[torch.from_numpy(ids).to(dev)].cpu().numpy()
    del xt, samp
    codes = codes_full if pq_bits == 8 else _pack4(codes_full)
    return IvfPqIndex(metric, d, nlist, pq_m, pq_bits, cent.cpu().numpy(), offsets, ids,
                      np.ascontiguousarray(codes), books, x, residual)


def build_ivf_pq(x: np.ndarray, nlist: int, pq_m: int, pq_bits: int, metric: str = "l2",
                 kmeans_iters: int = 12, pq_iters: int = 12, kmeans_sample: int | None = None,
                 pq_sample: int = 65536, residual: bool = False) -> IvfPqIndex:
    """Build an IVF-PQ index over ``x`` (f32 [n, d]).

    ``residual`` = False: PQ of the raw vectors.  True: PQ of each vector's
    residual to its list centroid, o - c_l (codebooks trained on sampled
    residuals), the residual form of Section 2's "Quantization"."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    n, d = x.shape
    if d % pq_m:
        raise ValueError("pq_m must divide d")
    if pq_bits not in (4, 8):
        raise ValueError("pq_bits must be 4 or 8")
    if pq_bits == 4 and pq_m % 2:
        raise ValueError("4-bit PQ needs an even pq_m")
    if kmeans_sample is None:
        kmeans_sample = min(n, 256 * nlist)
    if _DEVICE != "cpu" and n * d >= (1 << 28):
        return _build_ivf_pq_dev(x, nlist, pq_m, pq_bits, metric, kmeans_iters, pq_iters, kmeans_sample,
                                 pq_sample, residual)
    cent = kmeans(x, nlist, iters=kmeans_iters, seed=SEED_KMEANS, sample=kmeans_sample)
    assign = nearest(x, cent)
    ids, offsets = _inverted_lists(assign, nlist)
    xq = (x - cent[assign]).astype(np.float32) if residual else x

    dsub = d // pq_m
    ksub = 1 << pq_bits
    rng = np.random.default_rng(SEED_PQ)
    samp = xq[np.sort(rng.choice(n, size=min(n, pq_sample), replace=False))]
    books = np.empty((pq_m, ksub, dsub), dtype=np.float32)
    codes_full = np.empty((n, pq_m), dtype=np.uint8)
    for m in range(pq_m):
        sub = np.ascontiguousarray(samp[:, m * dsub:(m + 1) * dsub])
        books[m] = kmeans(sub, ksub, iters=pq_iters, seed=SEED_PQ + 17 * m)
        codes_full[:, m] = nearest(np.ascontiguousarray(xq[:, m * dsub:(m + 1) * dsub]), books[m])
    codes_full = codes_full[ids]
    codes = codes_full if pq_bits == 8 else _pack4(codes_full)
    return IvfPqIndex(metric, d, nlist, pq_m, pq_bits, cent, offsets, ids,
                      np.ascontiguousarray(codes), books, x, residual)


def _align(f, a: int = 64) -> None:
    pos = f.tell()
    pad = (-pos) % a
    if pad:
        f.write(b"\0" * pad)


def write_index(path: str, idx: IvfPqIndex) -> None:
    """Write an IVF-PQ index in the BBCIDX01 format described in the module docstring."""
    with open(path, "wb") as f:
        hdr = struct.pack(HEADER_FMT, MAGIC, 1, 2 if getattr(idx, "residual", False) else 0,
                          0 if idx.metric == "l2" else 1,
                          idx.d, idx.n, idx.nlist, idx.pq_m, idx.pq_bits)
        f.write(hdr + b"\0" * (HEADER_BYTES - len(hdr)))
        for arr, dt in ((idx.centroids, np.float32), (idx.list_offsets, np.int64),
                        (idx.ids, np.int64), (idx.codes, np.uint8),
                        (idx.codebooks, np.float32), (idx.vectors, np.float32)):
            _align(f)
            f.write(np.ascontiguousarray(arr, dtype=dt).tobytes())


def write_sign_index(path: str, idx: "IvfSignIndex") -> None:
    """Write an IVF index with the 1-bit sign quantizer in the BBCIDX01 format."""
    with open(path, "wb") as f:
        hdr = struct.pack(HEADER_FMT, MAGIC, 1, 1, 0, idx.d, idx.n, idx.nlist, 0, 0)
        f.write(hdr + b"\0" * (HEADER_BYTES - len(hdr)))
        for arr, dt in ((idx.centroids, np.float32), (idx.list_offsets, np.int64),
                        (idx.ids, np.int64), (idx.rotation, np.float32), (idx.vectors, np.float32)):
            _align(f)
            f.write(np.ascontiguousarray(arr, dtype=dt).tobytes())


@dataclasses.dataclass
class IvfSignIndex:
    """IVF lists plus the seeded rotation of the 1-bit sign quantizer; the
    codes and per-object factors are derived from these by their users."""
    metric: str
    d: int
    nlist: int
    centroids: np.ndarray       # f32 [nlist, d]
    list_offsets: np.ndarray    # i64 [nlist + 1]
    ids: np.ndarray             # i64 [n], list order
    rotation: np.ndarray        # f32 [d, d], orthonormal rows (r = P u)
    vectors: np.ndarray         # f32 [n, d], id order
    residual: bool = False      # codes quantise o - c_l (residual IVF-PQ)

    @property
    def n(self) -> int:
        return int(self.vectors.shape[0])


def random_rotation(d: int, seed: int = SEED_ROT) -> np.ndarray:
    """Seeded orthonormal d x d matrix (QR of a Gaussian matrix, FP64), stored FP32."""
    rng = np.random.default_rng(seed)
    q, r = np.linalg.qr(rng.standard_normal((d, d)))
    q = q * np.sign(np.diag(r))[None, :]
    return np.ascontiguousarray(q.astype(np.float32))


def build_ivf_sign(x: np.ndarray, nlist: int, kmeans_iters: int = 12,
                   kmeans_sample: int | None = None) -> IvfSignIndex:
    """IVF (L2) with a seeded rotation for 1-bit sign codes of P (o - c_l)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    n, d = x.shape
    if d % 32:
        raise ValueError("d must be a multiple of 32 for sign codes")
    if kmeans_sample is None:
        kmeans_sample = min(n, 256 * nlist)
    if _DEVICE != "cpu" and n * d >= (1 << 28):
        import torch
        dev = torch.device(_DEVICE)
        xt = torch.from_numpy(x).to(dev)
        rng = np.random.default_rng(SEED_KMEANS)
        if kmeans_sample < n:
            sel = torch.from_numpy(np.sort(rng.choice(n, size=kmeans_sample, replace=False))).to(dev)
            train = xt[sel]
        else:
            train = xt
        ct = _kmeans_dev(train, nlist, kmeans_iters, rng, 1 << 15)
        del train
        assign = _nearest_dev(xt, ct, 1 << 15).cpu().numpy()
        cent = ct.cpu().numpy()
        del xt, ct
    else:
        cent = kmeans(x, nlist, iters=kmeans_iters, seed=SEED_KMEANS, sample=kmeans_sample)
        assign = nearest(x, cent)
    ids, offsets = _inverted_lists(assign, nlist)
    return IvfSignIndex("l2", d, nlist, cent, offsets, ids, random_rotation(d), x)
