"""Host checks of the identities the GPU collector relies on, against the oracle.

* Update on per-bin counts: the scan counts pushed objects per equal-width
  bin; the first bin whose running count reaches K_c, mapped to its bucket,
  must be the bucket the oracle's Update (Algorithm 1) picks from the bucket
  counts, for codebooks the oracle builds (Section 3.2).
* Push as one compare: bucket(e) <= tau exactly when e <= d_min + (c << sh) - 1,
  c = number of bins whose bucket is <= tau (the map is monotone).
* d_max in two passes: the t-th smallest sampled estimate from a coarse
  histogram of e >> s and a fine histogram of the low s bits of the coarse
  bin that holds rank t - 1.
"""

import numpy as np
import pytest


def _sample(rng, n, hi):
    # estimates below 2^21 (32 sub-spaces x 65535), clustered like real ADC sums
    base = rng.integers(0, hi // 2)
    return np.clip(base + rng.gamma(3.0, hi / 40.0, n), 0, hi - 1).astype(np.uint32)


def _bin(e, cb):
    e = np.asarray(e, dtype=np.int64)
    b = np.where(e <= cb.d_min, 0, (e - cb.d_min) >> cb.sh)
    return np.minimum(b, 255)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("m", [2, 16, 64, 256])
def test_update_on_bins_equals_update_on_buckets(oracle_lib, seed, m):
    rng = np.random.default_rng(seed)
    s = _sample(rng, 5000, 1 << 21)
    kc = int(rng.integers(1, 4000))
    cb = oracle_lib.build_codebook(s, kc, m)
    mp = np.frombuffer(bytes(cb.map), dtype=np.uint8).astype(np.int64)
    assert np.all(np.diff(mp) >= 0) and mp.max() < m
    for trial in range(20):
        # counts of pushed objects per bin (later pushes sit in any bin)
        bins = np.bincount(_bin(_sample(rng, int(rng.integers(0, 9000)), 1 << 21), cb), minlength=256)
        buckets = np.bincount(mp, weights=bins, minlength=m).astype(np.int64)
        for k in (1, kc, int(bins.sum()), int(bins.sum()) + 1):
            want = oracle_lib.update(buckets, k)
            run = np.cumsum(bins)
            hit = np.nonzero(run >= k)[0]
            got = int(mp[hit[0]]) if len(hit) else m
            assert got == want, (trial, k)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("m", [4, 64, 256])
def test_push_threshold_is_one_compare(oracle_lib, seed, m):
    rng = np.random.default_rng(100 + seed)
    s = _sample(rng, 3000, 1 << 21)
    cb = oracle_lib.build_codebook(s, 2000, m)
    mp = np.frombuffer(bytes(cb.map), dtype=np.uint8).astype(np.int64)
    e = np.unique(np.concatenate([s, rng.integers(0, 1 << 21, 20000), [0, cb.d_min, cb.d_max, (1 << 21) - 1]]))
    bucket = mp[_bin(e, cb)]
    for tau in range(m + 1):
        c = int(np.count_nonzero(mp <= tau))
        etau = (1 << 32) - 1 if c >= 256 else min(cb.d_min + (c << cb.sh) - 1, (1 << 32) - 1)
        assert np.array_equal(bucket <= tau, e <= etau), tau


@pytest.mark.parametrize("seed", range(8))
def test_dmax_from_coarse_and_fine_histograms(seed):
    rng = np.random.default_rng(200 + seed)
    for eb in (19, 21, 23):                       # estimate bits for M = 8, 32, 96 / 128
        shc = eb - 11
        s = _sample(rng, int(rng.integers(1, 20000)), 1 << eb)
        t = int(rng.integers(1, len(s) + 1))
        coarse = np.bincount(s >> shc, minlength=2048)
        run = np.cumsum(coarse)
        hi = int(np.nonzero(run >= t)[0][0])
        r1 = t - 1 - (int(run[hi - 1]) if hi else 0)
        low = s[(s >> shc) == hi] & ((1 << shc) - 1)
        fine = np.cumsum(np.bincount(low, minlength=1 << shc))
        lo = int(np.nonzero(fine >= r1 + 1)[0][0])
        assert (hi << shc) | lo == np.sort(s)[t - 1]
