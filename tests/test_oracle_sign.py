"""Pins of the oracle's bounded re-rank (1-bit sign quantizer, Section 3.4).

* Sign codes and factors: closed forms for the identity rotation, and the
  Pythagorean identity e^2 + d alpha^2 = ||o - c||^2 that holds because
  alpha = <s, r> / d makes r - alpha s orthogonal to s.
* Bounds: they enclose the exact distance on random data; they collapse to it
  when the residual is a scaled sign vector and the query sits on the 4-bit
  grid (e = eta = 0).
* Algorithm 2: hand-worked cases; on random instances its result is the exact
  top-k and it re-ranks no more objects than the set of Observation 1 (it can
  re-rank fewer: an object whose interval holds Dist_k but lies wholly below
  every other object's interval needs no exact distance).
* The one-shot classification and the two-round re-rank: results equal the
  exact top-k; |Obs. 1| <= two-round count <= |S|.
"""

import numpy as np
import pytest

import oracle
from synth.index import IvfSignIndex, build_ivf_sign, random_rotation
from synth.data import gist_shaped


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _single_list_index(x, c, rot):
    n, d = x.shape
    return IvfSignIndex("l2", d, 1, c[None, :].astype(np.float32), np.array([0, n], dtype=np.int64),
                        np.arange(n, dtype=np.int64), rot.astype(np.float32), x.astype(np.float32))


def test_encode_identity_rotation_closed_form():
    d = 64
    rng = np.random.default_rng(1)
    s = np.where(rng.random((5, d)) < 0.5, -1.0, 1.0)
    a = np.array([0.5, 1.0, 2.0, 0.25, 4.0])
    c = rng.integers(-4, 4, d).astype(np.float64)
    x = c[None, :] + a[:, None] * s                          # residual = alpha * sign vector, exact in FP32
    idx = _single_list_index(x, c, np.eye(d))
    codes, fac = oracle.sign_encode(idx)
    for i in range(5):
        bits = np.unpackbits(codes[i].view(np.uint8), bitorder="little").astype(bool)
        assert np.array_equal(bits, s[i] > 0)
        assert fac[i, 0] == a[i]                              # alpha = mean |r_i|
        assert fac[i, 1] == 0.0                               # e = ||r - alpha s|| = 0
        assert fac[i, 2] == d * a[i] ** 2                     # ||o - c||^2
        assert fac[i, 3] == (s[i] > 0).sum()


def test_encode_pythagoras_random_rotation():
    x, _ = gist_shaped(2000, 1, d=96, n_centers=20)
    idx = build_ivf_sign(x, 8, kmeans_iters=3)
    codes, fac = oracle.sign_encode(idx)
    eps = oracle.rotation_eps(idx.rotation)
    assert eps < 1e-5
    alpha, e, un2 = fac[:, 0], fac[:, 1], fac[:, 2]
    d = idx.d
    # ||r||^2 = ||u||^2 up to the rotation's departure from orthogonality
    assert np.allclose(e ** 2 + d * alpha ** 2, un2, rtol=4 * eps + 1e-12)
    assert np.all(alpha > 0) and np.all(e >= 0)


def test_list_encoder_matches_object_encoder():
    x, _ = gist_shaped(1500, 1, d=64, n_centers=20)
    idx = build_ivf_sign(x, 6, kmeans_iters=3)
    c1, f1 = oracle.sign_encode(idx)
    c2, f2 = oracle.sign_encode_lists(idx, [0, 2, 5])
    for l in (0, 2, 5):
        a, b = idx.list_offsets[l], idx.list_offsets[l + 1]
        assert np.array_equal(c1[a:b], c2[a:b])
        assert np.allclose(f1[a:b], f2[a:b], rtol=1e-12, atol=1e-12)
    a, b = idx.list_offsets[1], idx.list_offsets[2]
    assert not c2[a:b].any() and not f2[a:b].any()


def test_bounds_enclose_exact_distance():
    x, q = gist_shaped(4000, 6, d=96, n_centers=30)
    idx = build_ivf_sign(x, 12, kmeans_iters=3)
    codes, fac = oracle.sign_encode(idx)
    eps = oracle.rotation_eps(idx.rotation)
    offs = idx.list_offsets
    for qi in range(len(q)):
        for l in range(idx.nlist):
            a, b = offs[l], offs[l + 1]
            lb, ub = oracle.sign_bounds(q[qi], idx.centroids[l], idx.rotation, eps, codes[a:b], fac[a:b])
            ex = oracle.rerank(q[qi], idx.vectors, idx.ids[a:b], "l2")
            assert np.all(lb <= ex) and np.all(ex <= ub)
            # narrower intervals with a smaller scale of the residual term
            lb2, ub2 = oracle.sign_bounds(q[qi], idx.centroids[l], idx.rotation, eps, codes[a:b], fac[a:b], 0.1)
            assert np.all(lb2 >= lb) and np.all(ub2 <= ub)


def test_bounds_collapse_without_quantisation_error():
    d = 64
    rng = np.random.default_rng(2)
    c = np.zeros(d)
    s = np.where(rng.random((8, d)) < 0.5, -1.0, 1.0)
    x = 0.5 * s
    # query on the 4-bit grid: q'_i = lo + Delta u_i with lo = -3, Delta = 0.5, u in [0, 15], both ends used
    u = rng.integers(0, 16, d)
    u[0], u[1] = 0, 15
    qv = -3.0 + 0.5 * u
    idx = _single_list_index(x, c, np.eye(d))
    codes, fac = oracle.sign_encode(idx)
    lb, ub = oracle.sign_bounds(qv, c, np.eye(d), 0.0, codes, fac)
    ex = ((x - qv[None, :]) ** 2).sum(1)
    assert np.allclose(lb, ex, rtol=1e-10) and np.allclose(ub, ex, rtol=1e-10)


# ---------------------------------------------------------------- Algorithm 2
@pytest.mark.parametrize("lb, ub, ex, k, count, obs1, result", [
    # disjoint: A is certainly first, nothing is re-ranked, although A's interval holds Dist_k
    ([0, 20], [10, 30], [3, 25], 1, 0, 1, [0]),
    ([0, 5], [10, 30], [3, 20], 1, 1, 1, [0]),        # A re-ranked; then 3 < 5 ends it
    ([0, 2, 2.5], [1, 3, 10], [0.5, 2.7, 5], 2, 2, 2, [0, 1]),
    ([0, 0.5], [10, 20], [1, 2], 1, 2, 2, [0]),       # both intervals hold Dist_k = 1
])
def test_alg2_hand_cases(lb, ub, ex, k, count, obs1, result):
    c, res = oracle.alg2(lb, ub, ex, k)
    assert c == count
    assert sorted(res.tolist()) == result
    assert oracle.obs1_count(lb, ub, ex, k) == obs1


def _random_instance(rng, n, width):
    ex = rng.random(n) * 10
    lb = ex - rng.random(n) * width
    ub = ex + rng.random(n) * width
    return lb, ub, ex


@pytest.mark.parametrize("seed", range(8))
def test_alg2_oneshot_rounds_random(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(50, 400))
    k = int(rng.integers(1, n // 2))
    lb, ub, ex = _random_instance(rng, n, float(rng.choice([0.05, 0.5, 3.0])))
    exact = np.lexsort((np.arange(n), ex))[:k]
    c2, res = oracle.alg2(lb, ub, ex, k)
    assert set(res.tolist()) == set(exact.tolist())
    m = oracle.obs1_count(lb, ub, ex, k)
    assert c2 <= m                                        # Alg. 2 re-ranks no more than the Obs. 1 set
    ns, nin, nr = oracle.oneshot(lb, ub, k)
    uk = np.sort(ub)[k - 1]
    S = np.flatnonzero(lb <= uk)
    assert ns == len(S) and set(exact.tolist()) <= set(S.tolist())
    # certainly-in members are in the exact top-k
    lk1 = np.sort(lb[S])[k] if len(S) > k else np.inf
    sure = S[ub[S] < lk1]
    assert len(sure) == nin and set(sure.tolist()) <= set(exact.tolist())
    cr, rres = oracle.rounds(lb, ub, ex, k)
    assert np.array_equal(rres, exact)
    assert m <= cr <= ns


# ---- the RaBitQ estimator's probabilistic bounds ----------------------------

def test_rq_bounds_collapse_closed_form():
    """Identity rotation, o = alpha s (e = 0, so <o_bar, o_r> = 1) and a query on
    the 4-bit grid (eta = 0): the estimator ||r||^2 / (d alpha) <s, q~> equals
    alpha <s, q> = <q, o> exactly and the interval collapses to ||q - o||^2.
    alpha != 1 separates ||r||^2 / (d alpha) from ||r||^2 / (d alpha^2)."""
    d = 64
    rng = np.random.default_rng(5)
    s = np.where(rng.random((6, d)) < 0.5, -1.0, 1.0)
    alpha = np.array([0.5, 2.0, 3.0, 0.25, 1.5, 7.0])
    o = alpha[:, None] * s
    q = rng.integers(0, 16, size=d).astype(np.float64)
    q[0], q[1] = 0.0, 15.0                           # lo = 0, Delta = 1: every component on the grid
    codes = np.packbits(s > 0, axis=1, bitorder="little").view(np.uint32)
    fac = np.stack([alpha, np.zeros(6), (o * o).sum(1), (s > 0).sum(1)], axis=1)
    lb, ub = oracle.sign_bounds_rq(q.astype(np.float32), np.zeros(d, np.float32), np.eye(d, dtype=np.float32),
                                   0.0, codes, fac, eps0=1.9)
    exact = ((q[None, :] - o) ** 2).sum(1)
    assert np.allclose(lb, exact, rtol=1e-10, atol=0) and np.allclose(ub, exact, rtol=1e-10, atol=0)


def _rq_instance(d, n, seed):
    rng = np.random.default_rng(seed)
    rot = random_rotation(d, seed=seed)
    c = rng.standard_normal(d).astype(np.float32)
    x = (c + rng.standard_normal((n, d))).astype(np.float32)
    q = (c + 0.8 * rng.standard_normal(d)).astype(np.float32)
    idx = _single_list_index(x, c, rot)
    codes, fac = oracle.sign_encode(idx)
    eps = oracle.rotation_eps(idx.rotation)
    exact = oracle.rerank(q, idx.vectors, idx.ids, "l2")
    return idx, q, codes, fac, eps, exact


@pytest.mark.parametrize("d", [128, 256])
def test_rq_bounds_cover_with_high_probability(d):
    """On Gaussian residuals under a random rotation the estimator's intervals
    (epsilon_0 = 1.9, about 1.9 standard deviations of the estimator) hold the
    exact distance for most objects, are much narrower than the hard bounds,
    and the estimator is unbiased: the mean error of the interval centres is
    within four standard errors of 0."""
    idx, q, codes, fac, eps, exact = _rq_instance(d, 4000, seed=d)
    lb, ub = oracle.sign_bounds_rq(q, idx.centroids[0], idx.rotation, eps, codes, fac, eps0=1.9)
    hl, hu = oracle.sign_bounds(q, idx.centroids[0], idx.rotation, eps, codes, fac, 1.0)
    assert np.all((hl <= exact) & (exact <= hu))                     # hard bounds: always
    inside = (lb <= exact) & (exact <= ub)
    assert 0.90 <= inside.mean() < 1.0
    assert np.median((hu - hl) / (ub - lb)) > 3.0
    err = 0.5 * (lb + ub) - exact
    assert abs(err.mean()) <= 4.0 * err.std() / np.sqrt(len(err))


def test_rq_search_equals_rounds_on_its_bounds_and_recall():
    """With the estimator's bounds the oracle's result is the two-round re-rank
    on those bounds: k distinct ids, exact distances, ascending; most of the
    exact top-k of the probed lists is kept."""
    x, q = gist_shaped(8000, 4, d=128, n_centers=60)
    idx = build_ivf_sign(x, 16, kmeans_iters=3)
    k, nprobe = 200, 6
    hi_, hd_, _ = oracle.sign_search(idx, q, k, nprobe)
    ri, rd, st = oracle.sign_search(idx, q, k, nprobe, estimator=1, eps0=1.9)
    for i in range(len(q)):
        v = ri[i] >= 0
        assert len(set(ri[i][v].tolist())) == v.sum() == k
        assert np.all(np.diff(rd[i][v]) >= 0)
        assert np.allclose(rd[i][v], oracle.rerank(q[i], idx.vectors, ri[i][v], "l2"), rtol=0, atol=0)
        assert len(set(ri[i].tolist()) & set(hi_[i].tolist())) >= 0.9 * k
        assert st[i, 1] < st[i, 0]                                   # S smaller than the scanned set
