"""Seeded generators for the vector workloads the search path is measured on.

The paper evaluates on Wiki, C4, MSMARCO and Deep100M (Table 1), which are
not available here.  These generators stand in for them with mixtures whose
shape follows the evaluated workloads: clustered Gaussian data, integer
SIFT-like components, non-negative anisotropic GIST-like data and unit-norm
embedding-like data with a power-law spectrum.  Queries are drawn from the
same mixture as the data (not as a subset of it).

Seeds: data 1, queries 2 (k-means 3, PQ 4 and rotation 5 live in
``synth.index``; request arrivals 6 in ``synth.requests``).
"""

from __future__ import annotations

import dataclasses
from typing import Callable, Tuple

import numpy as np

SEED_DATA = 1
SEED_QUERIES = 2


def _centers_and_assign(rng: np.random.Generator, n: int, n_centers: int):
    return rng.integers(0, n_centers, size=n)


def gaussian_mixture_tiny(n: int, nq: int, d: int = 128, n_centers: int = 1000,
                          sigma: float = 0.3, seed: int = SEED_DATA,
                          qseed: int = SEED_QUERIES) -> Tuple[np.ndarray, np.ndarray]:
    """Clustered FP32 data: centers ~ N(0, I_d); points = center + N(0, sigma^2 I)."""
    rc = np.random.default_rng(seed)
    centers = rc.standard_normal((n_centers, d)).astype(np.float32)
    x = _mixture_points(centers, n, sigma, np.random.default_rng(seed + 1000))
    q = _mixture_points(centers, nq, sigma, np.random.default_rng(qseed))
    return x, q


def _mixture_points(centers: np.ndarray, n: int, sigma, rng: np.random.Generator,
                    chunk: int = 1 << 18) -> np.ndarray:
    d = centers.shape[1]
    out = np.empty((n, d), dtype=np.float32)
    lab = rng.integers(0, centers.shape[0], size=n)
    sig = np.asarray(sigma, dtype=np.float32)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        noise = rng.standard_normal((e - s, d), dtype=np.float32)
        out[s:e] = centers[lab[s:e]] + noise * sig
    return out


def sift_shaped(n: int, nq: int, d: int = 128, n_centers: int = 10000, rank: int = 16,
                center_std: float = 1.0, point_std: float = 0.2, scale: float = 60.0,
                iso_std: float = 4.0, seed: int = SEED_DATA,
                qseed: int = SEED_QUERIES) -> Tuple[np.ndarray, np.ndarray]:
    """Integer components in [0, 255]: a clipped, rounded Gaussian mixture.

    Descriptor data such as SIFT has a low intrinsic dimension, which is what
    lets an IVF partition capture a query's large neighbourhoods.  The mixture
    therefore lives on a ``rank``-dimensional latent space: 10,000 latent
    centers ~ N(0, center_std^2 I_rank), latent points = center +
    N(0, point_std^2 I_rank), mapped by a fixed random d x rank matrix B
    (entries N(0, 1/rank)) as x = 128 + scale * B z + N(0, iso_std^2 I_d),
    then rounded and clipped to [0, 255].  Each component is Gaussian in R^d
    with covariance scale^2 point_std^2 B B^T + iso_std^2 I.  Values are
    stored as FP32 holding exact integers.
    """
    rc = np.random.default_rng(seed)
    B = (rc.standard_normal((d, rank)) / np.sqrt(rank)).astype(np.float32)
    zc = (center_std * rc.standard_normal((n_centers, rank))).astype(np.float32)

    def draw(m, rng, chunk=1 << 18):
        out = np.empty((m, d), dtype=np.float32)
        lab = rng.integers(0, n_centers, size=m)
        for s in range(0, m, chunk):
            e = min(m, s + chunk)
            z = zc[lab[s:e]] + point_std * rng.standard_normal((e - s, rank), dtype=np.float32)
            x = 128.0 + scale * (z @ B.T) + iso_std * rng.standard_normal((e - s, d), dtype=np.float32)
            np.rint(x, out=x)
            np.clip(x, 0.0, 255.0, out=x)
            out[s:e] = x
        return out

    return draw(n, np.random.default_rng(seed + 1000)), draw(nq, np.random.default_rng(qseed))


def sift_iid_mixture(n: int, nq: int, d: int = 128, n_centers: int = 10000, center_std: float = 40.0,
                     point_std: float = 20.0, seed: int = SEED_DATA,
                     qseed: int = SEED_QUERIES) -> Tuple[np.ndarray, np.ndarray]:
    """Integer components in [0, 255] from a full-dimensional mixture: 10,000
    centers ~ N(128, center_std^2) per component, points = center +
    N(0, point_std^2) per component, rounded and clipped to [0, 255].  Kept
    beside ``sift_shaped`` to show what an i.i.d. mixture does to IVF recall
    at large k (its neighbourhoods spread over the whole space)."""
    rc = np.random.default_rng(seed)
    centers = (128.0 + center_std * rc.standard_normal((n_centers, d))).astype(np.float32)

    def draw(m, rng, chunk=1 << 18):
        out = np.empty((m, d), dtype=np.float32)
        lab = rng.integers(0, n_centers, size=m)
        for s in range(0, m, chunk):
            e = min(m, s + chunk)
            x = centers[lab[s:e]] + point_std * rng.standard_normal((e - s, d), dtype=np.float32)
            np.rint(x, out=x)
            np.clip(x, 0.0, 255.0, out=x)
            out[s:e] = x
        return out

    return draw(n, np.random.default_rng(seed + 1000)), draw(nq, np.random.default_rng(qseed))


def gist_shaped(n: int, nq: int, d: int = 960, n_centers: int = 4096,
                seed: int = SEED_DATA, qseed: int = SEED_QUERIES) -> Tuple[np.ndarray, np.ndarray]:
    """Non-negative anisotropic mixture: per-dimension variance lambda_i ~ i^-0.5.

    centers = |N(0, diag(lambda))|; points = |center + N(0, 0.1 diag(lambda))|.
    """
    lam = (np.arange(1, d + 1, dtype=np.float64) ** -0.5).astype(np.float32)
    sd = np.sqrt(lam)
    rc = np.random.default_rng(seed)
    centers = np.abs(rc.standard_normal((n_centers, d)).astype(np.float32) * sd)
    x = np.abs(_mixture_points(centers, n, np.sqrt(0.1) * sd, np.random.default_rng(seed + 1000)))
    q = np.abs(_mixture_points(centers, nq, np.sqrt(0.1) * sd, np.random.default_rng(qseed)))
    return x, q


def embedding_shaped(n: int, nq: int, d: int = 768, seed: int = SEED_DATA,
                     qseed: int = SEED_QUERIES, chunk: int = 1 << 18) -> Tuple[np.ndarray, np.ndarray]:
    """Unit-norm anisotropic Gaussian with a power-law spectrum (variance i^-1),
    expressed in a seeded random orthonormal basis."""
    rr = np.random.default_rng(seed + 2000)
    basis, _ = np.linalg.qr(rr.standard_normal((d, d)))
    basis = basis.astype(np.float32)
    sd = (np.arange(1, d + 1, dtype=np.float64) ** -0.5).astype(np.float32)

    def draw(m, rng):
        out = np.empty((m, d), dtype=np.float32)
        for s in range(0, m, chunk):
            e = min(m, s + chunk)
            z = rng.standard_normal((e - s, d), dtype=np.float32) * sd
            z = z @ basis.T
            z /= np.linalg.norm(z, axis=1, keepdims=True)
            out[s:e] = z
        return out

    return draw(n, np.random.default_rng(seed)), draw(nq, np.random.default_rng(qseed))


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic search workload: data shape, index shape and query knobs."""
    name: str
    n: int
    d: int
    nlist: int
    metric: str            # "l2" or "ip"
    quantizer: str         # "pq" or "sign"
    pq_m: int
    pq_bits: int
    nq: int
    k: int
    nprobe: int
    gen: Callable[..., Tuple[np.ndarray, np.ndarray]]

    def scaled(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


WORKLOADS = {
    # 100k x 128 FP32 Gaussian mixture, 256 lists, PQ 16 x 8 bit, k = 1,000, nprobe = 32.
    "tiny": Workload("ivfpq-tiny-100k-d128", 100_000, 128, 256, "l2", "pq", 16, 8,
                     100, 1000, 32, gaussian_mixture_tiny),
    # 1M x 128 integer components, 1,024 lists, PQ 32 x 8 bit, k = 10,000.
    "sift": Workload("ivfpq-sift-1m-d128", 1_000_000, 128, 1024, "l2", "pq", 32, 8,
                     10_000, 10_000, 256, sift_shaped),
    # 1M x 128 integer components from the i.i.d. mixture (10,000 centers), same index shape.
    "sift_iid": Workload("ivfpq-siftiid-1m-d128", 1_000_000, 128, 1024, "l2", "pq", 32, 8,
                         10_000, 10_000, 256, sift_iid_mixture),
    # Same data, PQ 64 x 4 bit.
    "sift4": Workload("ivfpq4-sift-1m-d128", 1_000_000, 128, 1024, "l2", "pq", 64, 4,
                      10_000, 10_000, 256, sift_shaped),
    # Same data, PQ 32 x 4 bit (M = d / 4, the paper's PQ setting).
    "sift4m32": Workload("ivfpq4m32-sift-1m-d128", 1_000_000, 128, 1024, "l2", "pq", 32, 4,
                         10_000, 10_000, 256, sift_shaped),
    # 1M x 960 non-negative, 4,096 lists, 1-bit sign codes.
    "gist": Workload("ivfsign-gist-1m-d960", 1_000_000, 960, 4096, "l2", "sign", 0, 1,
                     4096, 10_000, 256, gist_shaped),
    # 10M x 768 unit norm, inner product, 16,384 lists, PQ 96 x 8 bit.
    "embed": Workload("ivfpq-embed-10m-d768", 10_000_000, 768, 16384, "ip", "pq", 96, 8,
                      8192, 50_000, 512, embedding_shaped),
}


def make_workload(w: Workload, n: int | None = None, nq: int | None = None):
    """Generate (data, queries) for workload ``w``, optionally at reduced sizes."""
    return w.gen(n if n is not None else w.n, nq if nq is not None else w.nq, d=w.d)
