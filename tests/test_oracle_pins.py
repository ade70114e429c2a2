"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Each test checks the oracle against something it does not compute the same
way: values the paper states for its worked example, mathematical identities
(the PQ table sum equals the distance to the PQ reconstruction), brute force
computed by numpy on tiny inputs, and cross-checks between independent
collectors (sort, binary heap, bucket-based result buffer).
"""

import json
import os

import numpy as np
import pytest

from conftest import scanned_set, small_workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Algorithm 1 Update / Push: the Figure 3 example (Section 3.1)
# ---------------------------------------------------------------------------
def test_update_matches_figure3_example(oracle_lib):
    g = json.load(open(os.path.join(GOLDEN, "fig3_result_buffer.json")))
    facts, cons = g["paper_facts"], g["constructed_to_match"]
    cb = np.array(cons["codebook_1based"], dtype=np.float64)
    m = len(cb) - 1

    def bucket0(x):                       # 0-based bucket with B[i] = [c_i, c_{i+1})
        return int(np.searchsorted(cb, x, side="right")) - 1

    counts = np.zeros(m, dtype=np.int64)
    for x in cons["distances_before_insert"]:
        counts[bucket0(x)] += 1
    k = facts["k"]
    tau = oracle_lib.update(counts, k)
    assert tau + 1 == facts["threshold_bucket_before_insert_1based"]
    assert cb[tau + 1] == facts["relaxed_threshold_before_insert"]      # upper bound of B[tau]
    b = bucket0(facts["inserted_object_distance"])
    assert b + 1 == facts["inserted_object_bucket_1based"]
    assert b <= tau                                                     # Push admits it
    counts[b] += 1
    tau2 = oracle_lib.update(counts, k)
    assert tau2 + 1 == facts["threshold_bucket_after_insert_1based"]


def test_update_infinity_when_fewer_than_k(oracle_lib):
    assert oracle_lib.update(np.array([1, 2, 0, 1]), 5) == 4           # m = "infinity"
    assert oracle_lib.update(np.array([1, 2, 0, 2]), 5) == 3
    assert oracle_lib.update(np.array([5, 0]), 5) == 0


# ---------------------------------------------------------------------------
# PQ lookup table and ADC (Section 2, "Quantization")
# ---------------------------------------------------------------------------
def _reconstruct(codes_unpacked, books):
    M, K, ds = books.shape
    return np.concatenate([books[m][codes_unpacked[:, m]] for m in range(M)], axis=1).astype(np.float64)


@pytest.mark.parametrize("kind", ["tiny", "sift", "sift4", "embed"])
def test_lut_sum_equals_distance_to_reconstruction(oracle_lib, kind):
    from synth.index import unpack_codes
    idx, q = small_workload(kind)
    codes = idx.codes[:500]
    un = unpack_codes(codes, idx.pq_m, idx.pq_bits)
    rec = _reconstruct(un, idx.codebooks.astype(np.float64))
    for qi in range(4):
        qq = q[qi].astype(np.float64)
        lut = oracle_lib.lut_f32(q[qi], idx.codebooks, idx.metric).astype(np.float64)
        est = lut[np.arange(idx.pq_m)[None, :], un].sum(axis=1)
        if idx.metric == "l2":
            ref = ((rec - qq[None, :]) ** 2).sum(axis=1)
        else:
            ref = -(rec @ qq)
        scale = np.abs(lut).max() * idx.pq_m
        np.testing.assert_allclose(est, ref, rtol=0, atol=1e-5 * scale)


@pytest.mark.parametrize("levels", [65535, 2047])
@pytest.mark.parametrize("kind", ["tiny", "sift", "sift4", "sift4m32", "embed"])
def test_uint16_table_within_rounding_bound(oracle_lib, kind, levels):
    """ADC over the integer table equals the FP32 table sum minus sum(lo_m),
    rescaled, within M half-steps of the quantiser (top level 65535: the
    uint16 table; 2047: the table whose entries FP16 holds exactly)."""
    from synth.index import unpack_codes
    idx, q = small_workload(kind)
    un = unpack_codes(idx.codes[:2000], idx.pq_m, idx.pq_bits)
    for qi in range(4):
        lut = oracle_lib.lut_f32(q[qi], idx.codebooks, idx.metric).astype(np.float64)
        t16 = oracle_lib.lut16(q[qi], idx.codebooks, idx.metric, levels=levels)
        assert t16.dtype == np.uint16 and t16.max() <= levels
        lo = lut.min(axis=1)
        span = (lut.max(axis=1) - lo).max()
        assert (t16.max(axis=1) == levels).any()            # the widest sub-space fills the range
        assert (t16.min(axis=1) == 0).all()                 # offsets remove the minimum
        e = oracle_lib.adc(t16, idx.codes[:2000], idx.pq_m, idx.pq_bits).astype(np.float64)
        exact = (lut[np.arange(idx.pq_m)[None, :], un] - lo[None, :]).sum(axis=1)
        step = span / levels
        assert np.abs(e * step - exact).max() <= idx.pq_m * 0.5 * step * 1.001 + 1e-6 * span


def test_table_levels_rescale_the_same_entries(oracle_lib):
    """The 2047-level table is the 65535-level recipe at a coarser step: each
    entry is the FP32 value's nearest level, so rescaled it lies within one
    coarse step (plus the FP32 rounding of the scale) of the fine table's."""
    idx, q = small_workload("sift4")
    for qi in range(6):
        fine = oracle_lib.lut16(q[qi], idx.codebooks, idx.metric).astype(np.float64)
        coarse = oracle_lib.lut16(q[qi], idx.codebooks, idx.metric, levels=2047).astype(np.float64)
        assert np.abs(coarse * (65535.0 / 2047.0) - fine).max() <= 65535.0 / 2047.0 * 0.5 + 1.0


@pytest.mark.parametrize("kind", ["sift4", "sift4m32", "embed4"])
def test_fp16_holds_the_2047_level_table_and_its_sums(oracle_lib, kind):
    """Why 2047 levels: FP16 has an 11-bit significand, so every integer in
    [0, 2048] is exact, and a product with 0 or 1 is exact; the sum of M such
    entries stays below 2^24, where every FP32 partial sum of integers is
    exact in any order.  So an FP16 x FP16 -> FP32 contraction of one-hot
    code rows with this table returns the integer ADC sum exactly."""
    from synth.index import unpack_codes
    idx, q = small_workload(kind)
    un = unpack_codes(idx.codes[:1500], idx.pq_m, idx.pq_bits)
    for qi in range(3):
        t = oracle_lib.lut16(q[qi], idx.codebooks, idx.metric, levels=2047)
        assert np.array_equal(t.astype(np.float16).astype(np.uint16), t)
        assert idx.pq_m * 2047 < 2 ** 24
        # the contraction in float32 with a shuffled summation order
        rng = np.random.default_rng(qi)
        order = rng.permutation(idx.pq_m)
        acc = np.zeros(len(un), dtype=np.float32)
        for m in order:
            acc = acc + t[m][un[:, m]].astype(np.float16).astype(np.float32)
        e = oracle_lib.adc(t, idx.codes[:1500], idx.pq_m, idx.pq_bits)
        assert np.array_equal(acc.astype(np.uint32), e)


def test_adc_is_sum_of_selected_entries_4bit_nibbles(oracle_lib):
    """4-bit rows: low nibble = even sub-space, high nibble = odd sub-space."""
    M, K = 4, 16
    t16 = np.arange(M * K, dtype=np.uint16).reshape(M, K) * 3
    codes = np.array([[0x21, 0x43], [0xF0, 0x0F]], dtype=np.uint8)   # [1,2,3,4], [0,15,15,0]
    e = oracle_lib.adc(t16, codes, M, 4)
    assert e[0] == t16[0, 1] + t16[1, 2] + t16[2, 3] + t16[3, 4]
    assert e[1] == t16[0, 0] + t16[1, 15] + t16[2, 15] + t16[3, 0]


# ---------------------------------------------------------------------------
# probe, re-rank, brute force against numpy
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["tiny", "embed"])
def test_probe_matches_numpy_sort(oracle_lib, kind):
    idx, q = small_workload(kind)
    c = idx.centroids.astype(np.float64)
    for qi in range(6):
        qq = q[qi].astype(np.float64)
        s = ((c - qq) ** 2).sum(1) if idx.metric == "l2" else -(c @ qq)
        order = np.lexsort((np.arange(len(s)), s))
        lists, scores = oracle_lib.probe(q[qi], idx.centroids, 9, idx.metric)
        np.testing.assert_allclose(scores, s[lists], rtol=1e-12)
        # the same set, and ascending scores
        assert set(lists.tolist()) == set(order[:9].tolist()) or np.isclose(s[order[8]], s[order[9]])
        assert np.all(np.diff(scores) >= 0)


def test_rerank_and_bruteforce_match_numpy(oracle_lib):
    idx, q = small_workload("tiny")
    x = idx.vectors
    ids = np.arange(0, 3000, 7)
    d = oracle_lib.rerank(q[0], x, ids, "l2")
    ref = ((x[ids].astype(np.float64) - q[0].astype(np.float64)) ** 2).sum(1)
    np.testing.assert_allclose(d, ref, rtol=1e-12)
    bi, bd = oracle_lib.bruteforce(q[:3], x, 50, "l2")
    for i in range(3):
        full = ((x.astype(np.float64) - q[i].astype(np.float64)) ** 2).sum(1)
        order = np.lexsort((np.arange(len(full)), full))[:50]
        np.testing.assert_allclose(bd[i], full[order], rtol=1e-12)
        assert set(bi[i].tolist()) == set(order.tolist())


def test_topk_final_pads_and_orders(oracle_lib):
    ids, d = oracle_lib.topk_final(np.array([3.0, 1.0, 1.0, 2.0]), np.array([10, 7, 5, 2]), 6)
    assert ids.tolist() == [5, 7, 2, 10, -1, -1]
    assert d[:4].tolist() == [1.0, 1.0, 2.0, 3.0] and np.isinf(d[4:]).all()


# ---------------------------------------------------------------------------
# collectors: sort = heap = bucket-based result buffer; superset invariant
# ---------------------------------------------------------------------------
def test_heap_equals_sort_with_ties(oracle_lib):
    rng = np.random.default_rng(0)
    e = rng.integers(0, 50, size=5000).astype(np.uint32)       # many ties
    ids = rng.permutation(5000).astype(np.int64)
    for kc in (1, 7, 100, 4999, 5000, 6000):
        a = oracle_lib.topkc(e, ids, kc, "sort")
        b = oracle_lib.topkc(e, ids, kc, "heap")
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        # brute force: lexicographic (e, id)
        order = np.lexsort((ids, e))[:kc]
        assert np.array_equal(a[0], ids[order])


def _scan(oracle_lib, idx, qv, nprobe):
    lists, _ = oracle_lib.probe(qv, idx.centroids, nprobe, idx.metric)
    sel, lofs = scanned_set(idx, lists)
    t16 = oracle_lib.lut16(qv, idx.codebooks, idx.metric)
    e = oracle_lib.adc(t16, idx.codes[sel], idx.pq_m, idx.pq_bits)
    return e, idx.ids[sel], lofs


@pytest.mark.parametrize("kind,nprobe,kc,m", [("tiny", 12, 300, 64), ("sift", 16, 900, 32),
                                               ("sift4", 16, 500, 256), ("embed", 10, 400, 2),
                                               ("ragged", 40, 1000, 16), ("tiny", 3, 5, 64)])
def test_bucket_collector_equals_sort(oracle_lib, kind, nprobe, kc, m):
    idx, q = small_workload(kind)
    for qi in range(4):
        e, ids, lofs = _scan(oracle_lib, idx, q[qi], nprobe)
        si, se = oracle_lib.topkc(e, ids, kc, "sort")
        bi, be, cb, counts = oracle_lib.bucket_collect(e, ids, lofs, kc, m, sample_min=3)
        assert np.array_equal(si, bi) and np.array_equal(se, be)
        # codebook properties (Section 3.2): monotone remap starting at bucket 0
        mp = np.frombuffer(bytes(cb.map), dtype=np.uint8)
        assert mp[0] == 0 and np.all(np.diff(mp.astype(int)) >= 0) and mp.max() < m
        assert cb.d_min <= cb.d_max and ((cb.d_max - cb.d_min) >> cb.sh) <= 255
        assert cb.sh == 0 or ((cb.d_max - cb.d_min) >> (cb.sh - 1)) > 255
        # superset invariant: every scanned object at or below the Kc-th estimate
        # lies in a bucket <= tau, so it was kept
        if len(e) >= kc:
            ekc = np.sort(e)[kc - 1]
            b = _bucket(e, cb)
            assert cb.tau < m and np.all(b[e <= ekc] <= cb.tau)
            assert counts[:cb.tau].sum() < kc <= counts[:cb.tau + 1].sum()


def _bucket(e, cb):
    mp = np.frombuffer(bytes(cb.map), dtype=np.uint8)
    e = e.astype(np.int64)
    b = np.where(e <= cb.d_min, 0, np.minimum((e - cb.d_min) >> cb.sh, 255))
    return mp[b]


def test_codebook_equal_depth_on_sample(oracle_lib):
    """Buckets of the equal-depth remap hold roughly equal shares of the sample."""
    rng = np.random.default_rng(1)
    e = (rng.normal(5000, 600, size=20000)).clip(0).astype(np.uint32)
    m = 16
    cb = oracle_lib.build_codebook(e, 20000, m)
    assert cb.d_min == e.min() and cb.d_max == e.max()
    counts = np.bincount(_bucket(e, cb), minlength=m)
    assert counts.min() > 0.4 * len(e) / m and counts.max() < 2.0 * len(e) / m


# ---------------------------------------------------------------------------
# whole path: special case that reduces to exact kNN
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("collector", ["sort", "heap", "bucket"])
def test_full_probe_full_candidates_is_exact_knn(oracle_lib, collector):
    idx, q = small_workload("ragged")
    k = 25
    gi, gd = oracle_lib.search(idx, q, k, nprobe=idx.nlist, kc=idx.n, collector=collector, m=16)
    bi, bd = oracle_lib.bruteforce(q, idx.vectors, k, idx.metric)
    assert np.array_equal(gi, bi)
    np.testing.assert_array_equal(gd, bd)


def test_search_collectors_agree_and_pad(oracle_lib):
    idx, q = small_workload("sift")
    a = oracle_lib.search(idx, q[:6], 200, 8, 400, "sort")
    b = oracle_lib.search(idx, q[:6], 200, 8, 400, "bucket", m=64)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # the same on the 2047-level table (coarser keys, more ties)
    idx4, q4 = small_workload("sift4")
    a = oracle_lib.search(idx4, q4[:6], 200, 8, 400, "sort", lut_levels=2047)
    b = oracle_lib.search(idx4, q4[:6], 200, 8, 400, "bucket", m=64, lut_levels=2047)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # more results requested than objects scanned: padded with (-1, inf)
    idx2, q2 = small_workload("ragged")
    ids, d, st = oracle_lib.search(idx2, q2[:2], 500, 1, 600, "bucket", m=8, with_stats=True)
    for i in range(2):
        sq = st[i, 0]
        assert (ids[i, :sq] >= 0).all() and (ids[i, sq:] == -1).all() and np.isinf(d[i, sq:]).all()


def test_recall_improves_with_candidates(oracle_lib):
    """Re-ranking more candidates cannot lose recall (same probe)."""
    idx, q = small_workload("sift")
    k = 100
    bi, bd = oracle_lib.bruteforce(q[:8], idx.vectors, k, idx.metric)
    prev = -1.0
    for kc in (100, 200, 400, 800):
        gi, gd = oracle_lib.search(idx, q[:8], k, 16, kc)
        rec = np.mean([(gd[i] <= bd[i, -1]).sum() / k for i in range(8)])
        assert rec >= prev - 1e-12
        prev = rec
