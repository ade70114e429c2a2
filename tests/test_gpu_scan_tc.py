"""The list-grouped scan on the tensor cores ("scan_tc") against the oracle.

With tables of top level 2047 the FP32 accumulators of the one-hot x table
contraction are the integer table sums, so everything integer matches the
oracle bit for bit: probe lists, candidate sets and the result buffer's
codebook, threshold and counts (Algorithm 1 run by the oracle on keys from
oracle.lut16(levels=2047)).  The one-query SIMT scan on the same tables gives
the same candidates and state, and search results equal the oracle's search
at lut_levels=2047 (bit for bit on integer data).
"""

import numpy as np
import pytest

from conftest import check_topk, scanned_set, small_workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LEVELS = 2047


@pytest.fixture(scope="module")
def bbc():
    import paper_2604_01960_gb300 as bbc
    bbc.build()
    assert torch.cuda.is_available(), "CUDA device required"
    return bbc


_IDX = {}


def dev_index(bbc, kind):
    if kind not in _IDX:
        idx, q = small_workload(kind)
        _IDX[kind] = (bbc.bbc_index_create(idx, 0), idx, q)
    return _IDX[kind]


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def sync_ok(bbc, h):
    torch.cuda.synchronize()
    bbc.bbc_stream_status(h)


def _collect(bbc, h, q, nprobe, kc):
    nq = len(q)
    qd = cuda(q)
    lists = torch.empty((nq, nprobe), dtype=torch.int32, device="cuda")
    bbc.bbc_probe(h, qd, nq, nprobe, lists)
    ids = torch.full((nq, kc), -1, dtype=torch.int32, device="cuda")
    cnt = torch.empty(nq, dtype=torch.int64, device="cuda")
    st = torch.zeros(nq * bbc.STATE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    bbc.bbc_collect(h, qd, nq, nprobe, lists, kc, ids, cnt, st)
    sync_ok(bbc, h)
    return (lists.cpu().numpy(), ids.cpu().numpy().view(np.uint32), cnt.cpu().numpy(),
            st.cpu().numpy().view(bbc.STATE_DTYPE))


def _set(bbc, h, **kv):
    for k, v in kv.items():
        bbc.bbc_set_param(h, k, v)


def _reset(bbc, h):
    _set(bbc, h, scan_tc=0, lut_levels=65535, buckets=64, sample_lists=8, kc_ratio=1.5, split=0)


CASES = [("sift4", 20, 1200, 64, 4), ("sift4", 64, 12000, 48, 8), ("sift4m32", 16, 900, 32, 8),
         ("embed4", 10, 400, 2, 8), ("ragged4", 40, 300, 16, 3), ("ragged4", 2, 1000, 64, 8),
         ("sift4", 5, 1, 64, 8), ("medium4", 48, 3000, 64, 8), ("medium4", 128, 20000, 64, 8),
         ("many4", 200, 600, 64, 8), ("many4", 40, 150, 16, 4)]


@pytest.mark.parametrize("kind,nprobe,kc,m,smin", CASES)
def test_tc_collect_candidates_and_state(bbc, oracle_lib, kind, nprobe, kc, m, smin):
    """Candidates and collector state of the tensor-core scan equal the
    oracle's Algorithm 1 on the 2047-level table's keys, and the one-query
    SIMT scan's on the same table."""
    h, idx, q = dev_index(bbc, kind)
    try:
        _set(bbc, h, buckets=m, sample_lists=smin, scan_tc=1)
        assert bbc.bbc_get_param(h, "lut_levels") == LEVELS
        lists, ids, cnt, state = _collect(bbc, h, q, nprobe, kc)
        _set(bbc, h, scan_tc=0, split=1)
        lists2, ids2, cnt2, state2 = _collect(bbc, h, q, nprobe, kc)
    finally:
        _reset(bbc, h)
    assert np.array_equal(lists, lists2) and np.array_equal(cnt, cnt2)
    nchk = len(q) if len(q) <= 64 else 64
    for i in range(len(q)):
        n = int(cnt[i])
        assert np.array_equal(np.sort(ids[i, :n]), np.sort(ids2[i, :n])), f"query {i} vs SIMT"
        for f in ("d_min", "d_max", "sh", "sample_lists", "sample_size", "tau", "below", "scanned"):
            assert state[i][f] == state2[i][f], (i, f)
        assert np.array_equal(state[i]["map"], state2[i]["map"])
    for i in range(nchk):
        ol, _ = oracle_lib.probe(q[i], idx.centroids, nprobe, idx.metric)
        assert np.array_equal(lists[i], ol)
        sel, lofs = scanned_set(idx, ol)
        t = oracle_lib.lut16(q[i], idx.codebooks, idx.metric, levels=LEVELS)
        e = oracle_lib.adc(t, idx.codes[sel], idx.pq_m, idx.pq_bits)
        sid = idx.ids[sel]
        ref_ids, _ = oracle_lib.topkc(e, sid, kc, "sort")
        n = int(cnt[i])
        assert n == min(kc, len(e))
        assert np.array_equal(np.sort(ids[i, :n].astype(np.int64)), np.sort(ref_ids)), f"query {i}"
        _, _, cb, counts = oracle_lib.bucket_collect(e, sid, lofs, kc, m, sample_min=smin)
        s = state[i]
        assert s["scanned"] == len(e)
        assert (s["d_min"], s["d_max"], s["sh"], s["sample_lists"]) == (cb.d_min, cb.d_max, cb.sh, cb.sample_lists)
        assert s["sample_size"] == cb.sample_size
        assert np.array_equal(s["map"], np.frombuffer(bytes(cb.map), dtype=np.uint8))
        assert s["tau"] == cb.tau
        if cb.tau < m:
            assert np.array_equal(s["hist"][:cb.tau + 1].astype(np.int64), counts[:cb.tau + 1])
            assert s["below"] == cb.below
        assert s["pushed"] >= min(kc, len(e))


@pytest.mark.parametrize("kind,k,nprobe,ratio", [("sift4", 300, 24, 2.0), ("sift4m32", 500, 16, 1.5),
                                                 ("embed4", 200, 10, 1.5), ("ragged4", 50, 40, 1.0),
                                                 ("medium4", 2000, 64, 1.5), ("sift4", 1, 3, 1.0),
                                                 ("many4", 300, 200, 1.5)])
def test_tc_search_end_to_end(bbc, oracle_lib, kind, k, nprobe, ratio):
    h, idx, q = dev_index(bbc, kind)
    kc = max(k, int(np.ceil(ratio * k - 1e-9)))
    nq = len(q)
    ids = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    dd = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    try:
        _set(bbc, h, kc_ratio=ratio, scan_tc=1)
        bbc.bbc_search(h, cuda(q), nq, k, nprobe, ids, dd)
        sync_ok(bbc, h)
    finally:
        _reset(bbc, h)
    gi, gd = ids.cpu().numpy(), dd.cpu().numpy()
    nchk = min(nq, 48)
    oi, od = oracle_lib.search(idx, q[:nchk], k, nprobe, kc, "sort", lut_levels=LEVELS)
    exact = kind in ("sift4", "sift4m32", "medium4")
    for i in range(nchk):
        check_topk(oracle_lib, idx, q[i], gi[i], gd[i], oi[i], od[i], exact)


@pytest.mark.parametrize("kind", ["sift4", "embed4", "medium4"])
def test_tc_mixed_batch(bbc, oracle_lib, kind):
    """Per-query k and nprobe in one bbc_search_ex call: every query gets the
    oracle's result at its own k, nprobe and K_c."""
    h, idx, q = dev_index(bbc, kind)
    ratio = 1.5
    rng = np.random.default_rng(23)
    nq = min(len(q), 200)
    q = q[:nq]
    ks = rng.integers(1, 1500, size=nq).astype(np.int32)
    ps = rng.integers(1, idx.nlist + 1, size=nq).astype(np.int32)
    tot = int(ks.sum())
    ids = torch.empty(tot, dtype=torch.int64, device="cuda")
    dd = torch.empty(tot, dtype=torch.float32, device="cuda")
    try:
        _set(bbc, h, kc_ratio=ratio, scan_tc=1)
        bbc.bbc_search_ex(h, cuda(q), nq, ks, ps, ids, dd)
        sync_ok(bbc, h)
    finally:
        _reset(bbc, h)
    gi, gd = ids.cpu().numpy(), dd.cpu().numpy()
    off = np.concatenate([[0], np.cumsum(ks)])
    exact = kind in ("sift4", "medium4")
    for i in range(min(nq, 40)):
        k = int(ks[i])
        kc = max(k, int(np.ceil(ratio * k - 1e-9)))
        oi, od = oracle_lib.search(idx, q[i:i + 1], k, int(ps[i]), kc, "sort", lut_levels=LEVELS)
        check_topk(oracle_lib, idx, q[i], gi[off[i]:off[i + 1]], gd[off[i]:off[i + 1]], oi[0], od[0], exact)


def test_tc_lut_levels_bit_exact(bbc, oracle_lib):
    h, idx, q = dev_index(bbc, "sift4")
    nq = len(q)
    out = torch.empty((nq, idx.pq_m, 16), dtype=torch.int16, device="cuda")
    try:
        _set(bbc, h, lut_levels=LEVELS)
        bbc.bbc_lut(h, cuda(q), nq, out)
        sync_ok(bbc, h)
    finally:
        _reset(bbc, h)
    got = out.cpu().numpy().view(np.uint16)
    for i in range(nq):
        assert np.array_equal(got[i], oracle_lib.lut16(q[i], idx.codebooks, idx.metric, levels=LEVELS))


def test_tc_refused_where_it_does_not_apply(bbc):
    h, idx, q = dev_index(bbc, "sift4")
    try:
        bbc.bbc_set_param(h, "scan_tc", 1)
        with pytest.raises(bbc.BBCError) as ei:
            bbc.bbc_set_param(h, "lut_levels", 4095)        # entries FP16 cannot hold exactly
        assert ei.value.code == -1
        bbc.bbc_set_param(h, "buckets", 100)                # more buckets than the kernel counts per row
        ids = torch.empty((2, 10), dtype=torch.int64, device="cuda")
        dd = torch.empty((2, 10), dtype=torch.float32, device="cuda")
        with pytest.raises(bbc.BBCError) as ei:
            bbc.bbc_search(h, cuda(q[:2]), 2, 10, 4, ids, dd)
        assert ei.value.code == -9
    finally:
        _reset(bbc, h)
    h8, _, _ = dev_index(bbc, "sift")                       # 8-bit codes
    with pytest.raises(bbc.BBCError) as ei:
        bbc.bbc_set_param(h8, "scan_tc", 1)
    assert ei.value.code == -9
