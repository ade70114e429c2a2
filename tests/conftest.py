"""Shared fixtures: seeded small workloads and their IVF-PQ indexes.

Marker ``gpu``: the test needs a CUDA device and the compiled libbbc.so.
"""

import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled CUDA library")


_CACHE = {}


def small_workload(kind: str):
    """Seeded small workloads spanning the configurations of the search path.

    Each returns (index, queries).  Sizes keep the CPU oracle to seconds while
    spanning several 32-vector blocks per list and ragged list tails.
    """
    if kind in _CACHE:
        return _CACHE[kind]
    from synth import build_ivf_pq
    from synth.data import gaussian_mixture_tiny, sift_shaped, embedding_shaped
    if kind == "tiny":        # FP32 Gaussian mixture, L2, PQ 16 x 8 bit
        x, q = gaussian_mixture_tiny(12000, 24, d=64, n_centers=200, sigma=0.3)
        idx = build_ivf_pq(x, 48, 16, 8, "l2", kmeans_iters=6, pq_iters=6, pq_sample=8000)
    elif kind == "sift":      # integer [0,255] components, L2, PQ 32 x 8 bit
        x, q = sift_shaped(12000, 24, d=128, n_centers=300)
        idx = build_ivf_pq(x, 64, 32, 8, "l2", kmeans_iters=6, pq_iters=6, pq_sample=8000)
    elif kind == "sift4":     # same data, PQ 64 x 4 bit
        x, q = sift_shaped(12000, 24, d=128, n_centers=300)
        idx = build_ivf_pq(x, 64, 64, 4, "l2", kmeans_iters=6, pq_iters=6, pq_sample=8000)
    elif kind == "sift4m32":  # same data, PQ 32 x 4 bit (M = d / 4, the paper's PQ setting)
        x, q = sift_shaped(12000, 24, d=128, n_centers=300)
        idx = build_ivf_pq(x, 64, 32, 4, "l2", kmeans_iters=6, pq_iters=6, pq_sample=8000)
    elif kind == "embed4":    # unit norm, inner product, PQ 32 x 4 bit
        x, q = embedding_shaped(12000, 24, d=64)
        idx = build_ivf_pq(x, 48, 32, 4, "ip", kmeans_iters=6, pq_iters=6, pq_sample=8000)
    elif kind == "embed":     # unit norm, inner product, PQ 32 x 8 bit
        x, q = embedding_shaped(12000, 24, d=64)
        idx = build_ivf_pq(x, 48, 32, 8, "ip", kmeans_iters=6, pq_iters=6, pq_sample=8000)
    elif kind == "medium":    # 60k integer vectors: enough for K_c above 16,384
        x, q = sift_shaped(60000, 12, d=128, n_centers=1200)
        idx = build_ivf_pq(x, 128, 32, 8, "l2", kmeans_iters=6, pq_iters=6, pq_sample=20000)
    elif kind == "pad":       # d = 40: rows of the low-precision copies are zero padded to 48
        x, q = gaussian_mixture_tiny(6000, 16, d=40, n_centers=100, sigma=0.3)
        idx = build_ivf_pq(x, 32, 8, 8, "l2", kmeans_iters=6, pq_iters=6, pq_sample=6000)
    elif kind == "wide":      # d = 768 unit norm, inner product, PQ 96 x 8 bit
        x, q = embedding_shaped(8000, 12, d=768)
        idx = build_ivf_pq(x, 24, 96, 8, "ip", kmeans_iters=5, pq_iters=5, pq_sample=8000)
    elif kind == "rtiny":     # residual IVF-PQ: the tiny data, PQ 16 x 8 bit of o - c_l
        x, q = gaussian_mixture_tiny(12000, 24, d=64, n_centers=200, sigma=0.3)
        idx = build_ivf_pq(x, 48, 16, 8, "l2", kmeans_iters=6, pq_iters=6, pq_sample=8000, residual=True)
    elif kind == "rsift":     # residual IVF-PQ on integer data, PQ 32 x 8 bit
        x, q = sift_shaped(12000, 24, d=128, n_centers=300)
        idx = build_ivf_pq(x, 64, 32, 8, "l2", kmeans_iters=6, pq_iters=6, pq_sample=8000, residual=True)
    elif kind == "rsift4":    # residual IVF-PQ, PQ 64 x 4 bit
        x, q = sift_shaped(12000, 24, d=128, n_centers=300)
        idx = build_ivf_pq(x, 64, 64, 4, "l2", kmeans_iters=6, pq_iters=6, pq_sample=8000, residual=True)
    elif kind == "rembed":    # residual IVF-PQ, inner product, PQ 32 x 8 bit
        x, q = embedding_shaped(12000, 24, d=64)
        idx = build_ivf_pq(x, 48, 32, 8, "ip", kmeans_iters=6, pq_iters=6, pq_sample=8000, residual=True)
    elif kind == "rragged":   # residual IVF-PQ over few vectors, many short and empty lists
        x, q = gaussian_mixture_tiny(700, 8, d=32, n_centers=40, sigma=0.5)
        idx = build_ivf_pq(x, 40, 8, 8, "l2", kmeans_iters=4, pq_iters=4, pq_sample=700, residual=True)
    elif kind == "ragged4":   # few vectors, many short and empty lists, PQ 32 x 4 bit
        x, q = gaussian_mixture_tiny(700, 8, d=32, n_centers=40, sigma=0.5)
        idx = build_ivf_pq(x, 40, 32, 4, "l2", kmeans_iters=4, pq_iters=4, pq_sample=700)
    elif kind == "medium4":   # 60k integer vectors, 400 queries: lists of several 256-vector
        # tiles, each list probed by more than 128 queries of a batch; PQ 32 x 4 bit
        x, q = sift_shaped(60000, 400, d=128, n_centers=1200)
        idx = build_ivf_pq(x, 128, 32, 4, "l2", kmeans_iters=6, pq_iters=6, pq_sample=20000)
    elif kind == "many4":     # 400 short lists, every fifth one emptied (its objects join the list
        # before it), 320 queries: more list-grouped items than a GPU has CTAs; PQ 32 x 4 bit
        import dataclasses
        x, q = gaussian_mixture_tiny(6000, 320, d=32, n_centers=40, sigma=0.5)
        idx = build_ivf_pq(x, 400, 32, 4, "l2", kmeans_iters=4, pq_iters=4, pq_sample=6000)
        offs = idx.list_offsets.copy()
        for l in range(5, idx.nlist, 5):
            offs[l] = offs[l + 1]
        idx = dataclasses.replace(idx, list_offsets=offs)
    elif kind == "ragged":    # few vectors, many short and empty lists
        x, q = gaussian_mixture_tiny(700, 8, d=32, n_centers=40, sigma=0.5)
        idx = build_ivf_pq(x, 40, 8, 8, "l2", kmeans_iters=4, pq_iters=4, pq_sample=700)
    else:
        raise KeyError(kind)
    _CACHE[kind] = (idx, q)
    return idx, q


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle


def scanned_set(idx, lists):
    """Positions of the probed lists in probe order and their list offsets."""
    offs = idx.list_offsets
    sel = [np.arange(offs[l], offs[l + 1]) for l in lists]
    lofs = np.zeros(len(sel) + 1, dtype=np.int64)
    lofs[1:] = np.cumsum([len(s) for s in sel])
    return (np.concatenate(sel) if sel else np.zeros(0, np.int64)), lofs


def check_topk(oracle_lib, idx, qv, gi, gd, oi, od, exact, rtol=1e-5):
    """One query's GPU result (gi, gd) against the oracle's (oi, od).

    exact: integer data, where the FP32 re-rank is exact, so ids and distances
    match bit for bit.  Otherwise every reported distance is within rtol of
    the FP64 distance of its id (relative to itself for squared L2, to
    ||q|| ||v||_max for inner products), the two lists agree as order
    statistics, and ids differ only among objects tied with the k-th distance
    within that tolerance."""
    k = len(oi)
    valid = oi >= 0
    assert np.array_equal(gi >= 0, valid)
    assert np.all(np.isinf(gd[~valid]))
    if exact:
        assert np.array_equal(gi, oi)
        assert np.array_equal(gd[valid].astype(np.float64), od[valid])
        return
    g = gi[valid]
    d64 = oracle_lib.rerank(qv, idx.vectors, g, idx.metric)
    if idx.metric == "ip":
        # -<q, v> near 0 has no relative accuracy: measure against ||q|| ||v||
        qn = float(np.linalg.norm(qv.astype(np.float64)))
        vmax = float(np.linalg.norm(idx.vectors.astype(np.float64), axis=1).max())
        floor = qn * vmax
    else:
        # a squared L2 distance is a sum of non-negative terms: its FP32 value is
        # within a small multiple of 2^-24 of the FP64 one relative to itself, so
        # the tolerance is purely relative (no absolute floor)
        floor = 0.0
    tol = rtol * np.maximum(np.abs(d64), floor)
    assert np.all(np.abs(gd[valid] - d64) <= tol)                      # FP32 vs FP64 per result
    assert np.all(np.abs(d64 - od[valid]) <= 2 * tol + rtol * np.abs(od[valid]))   # same order statistics
    diff = set(g.tolist()) ^ set(oi[valid].tolist())
    if diff:                                                           # only ties at the boundary
        dk = od[valid][-1]
        dd = oracle_lib.rerank(qv, idx.vectors, np.array(sorted(diff)), idx.metric)
        assert np.all(np.abs(dd - dk) <= 2 * rtol * max(abs(dk), floor))
