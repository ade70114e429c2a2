"""Pins of the oracle's Algorithm 4 (IVF+PQ with early re-ranking, Section 3.3).

* A hand-worked instance: three lists, m = 4 buckets, n_cand = 4, the sample
  one list; the predicted threshold bucket after the sample is the bucket of
  the ceil(4/12 * 4) = 2nd smallest sampled estimate, so exactly one object of
  the second list (estimate 1, bucket 0 < 1) is scored early, and it is one of
  the four candidates.
* Random instances: the candidates are the sort-based top-n_cand by
  (estimated distance, id) (early re-ranking changes when exact distances are
  computed, not which objects are candidates), early-scored candidates <=
  early-scored objects <= objects outside the sample.
* A sample covering every list leaves nothing to score early.
"""

import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def test_alg4_hand_case():
    e = np.array([1, 2, 3, 4, 1, 5, 2, 6, 3, 3, 9, 9], dtype=np.uint32)
    ids = np.arange(12, dtype=np.int64)
    lofs = np.array([0, 4, 8, 12], dtype=np.int64)
    cand, early, ne, nec = oracle.alg4(e, ids, lofs, kc=4, m=4, sample_min=1)
    assert cand.tolist() == [0, 4, 1, 6]
    assert early.tolist() == [False, True, False, False]
    assert (ne, nec) == (1, 1)


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_alg4_candidates_equal_sort_and_counts_are_consistent(seed):
    rng = np.random.default_rng(seed)
    nl = int(rng.integers(5, 30))
    lens = rng.integers(0, 200, size=nl)
    lofs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    n = int(lofs[-1])
    # estimates drift upwards with the probe rank, as for lists visited nearest first
    e = (rng.integers(0, 5000, size=n) + 300 * np.repeat(np.arange(nl), lens)).astype(np.uint32)
    ids = rng.permutation(n).astype(np.int64)
    for kc in (1, 50, 400, max(1, n // 2)):
        cand, early, ne, nec = oracle.alg4(e, ids, lofs, kc=kc, m=32, sample_min=3)
        ref, _ = oracle.topkc(e, ids, kc, "sort")
        assert np.array_equal(np.sort(cand), np.sort(ref))
        assert nec == int(early.sum()) <= ne
        _, _, cb, _ = oracle.bucket_collect(e, ids, lofs, kc, 32, sample_min=3)
        assert ne <= n - int(lofs[cb.sample_lists])


def test_alg4_sample_covering_all_lists_scores_nothing_early():
    rng = np.random.default_rng(9)
    lofs = np.array([0, 40, 90, 120], dtype=np.int64)
    e = rng.integers(0, 1000, size=120).astype(np.uint32)
    ids = np.arange(120, dtype=np.int64)
    cand, early, ne, nec = oracle.alg4(e, ids, lofs, kc=500, m=16, sample_min=1)
    assert len(cand) == 120 and (ne, nec) == (0, 0)
