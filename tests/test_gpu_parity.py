"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Integer work (probe lists, uint16 tables, estimated distances, candidate sets,
collector state) must match bit for bit.  Re-rank distances are FP32 and
must lie within 1e-5 relative of the FP64 oracle; result ids may differ only
among objects whose exact distances tie with the k-th within that tolerance.
For integer-valued data the FP32 distances are exact, so results match bit
for bit end to end.
"""

import numpy as np
import pytest

from conftest import check_topk as _check_topk, scanned_set, small_workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu



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
        h = bbc.bbc_index_create(idx, 0)
        _IDX[kind] = (h, idx, q)
    return _IDX[kind]


def cuda(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.to("cuda") if dtype is None else t.to("cuda", dtype)


def sync_ok(bbc, h):
    torch.cuda.synchronize()
    bbc.bbc_stream_status(h)


KINDS = ["tiny", "sift", "sift4", "embed", "ragged", "wide"]


@pytest.mark.parametrize("kind", KINDS)
def test_lut16_bit_exact(bbc, oracle_lib, kind):
    h, idx, q = dev_index(bbc, kind)
    nq = len(q)
    K = 1 << idx.pq_bits
    out = torch.empty((nq, idx.pq_m, K), dtype=torch.int16, device="cuda")
    bbc.bbc_lut(h, cuda(q), nq, out)
    sync_ok(bbc, h)
    got = out.cpu().numpy().view(np.uint16)
    for i in range(nq):
        ref = oracle_lib.lut16(q[i], idx.codebooks, idx.metric)
        assert np.array_equal(got[i], ref), f"query {i}"


def _probe_eps(d, qn, cm, metric, tc):
    """The pruning bound the selection kernel uses for the approximate scores."""
    if not tc:
        return (d + 4) * 2.0 ** -22 * (qn + cm) ** 2
    rel = 3.1 * 2.0 ** -16 + 3.06 * d * 2.0 ** -23
    if metric == "l2":
        return 2.0 * (2.0 * rel * qn * cm + 2.0 ** -23 * (cm * cm + 2.0 * qn * cm))
    return 2.0 * (rel * qn * cm + 2.0 ** -24 * qn * cm)


@pytest.mark.parametrize("tc", [1, 0])
@pytest.mark.parametrize("kind", ["tiny", "sift", "embed", "ragged", "wide"])
def test_probe_scores_within_bound(bbc, kind, tc):
    """Approximate scores (tensor-core BF16 split GEMM, or FP32) lie within the
    stated bound of the FP64 score minus ||q||^2."""
    h, idx, q = dev_index(bbc, kind)
    bbc.bbc_set_param(h, "probe_gemm", tc)
    try:
        nq = len(q)
        out = torch.empty((nq, idx.nlist), dtype=torch.float32, device="cuda")
        bbc.bbc_probe_scores(h, cuda(q), nq, out)
        sync_ok(bbc, h)
    finally:
        bbc.bbc_set_param(h, "probe_gemm", 1)
    a = out.cpu().numpy().astype(np.float64)
    c = idx.centroids.astype(np.float64)
    cm = np.sqrt((c * c).sum(1)).max()
    for i in range(nq):
        qq = q[i].astype(np.float64)
        if idx.metric == "l2":
            ref = ((c - qq) ** 2).sum(1) - (qq * qq).sum()
        else:
            ref = -(c @ qq)
        eps = _probe_eps(idx.d, np.sqrt((qq * qq).sum()), cm, idx.metric, tc)
        assert np.abs(a[i] - ref).max() <= eps, (i, np.abs(a[i] - ref).max(), eps)


@pytest.mark.parametrize("tc", [1, 0])
@pytest.mark.parametrize("kind,nprobe", [("tiny", 1), ("tiny", 13), ("sift", 32), ("embed", 48),
                                         ("ragged", 40), ("sift4", 64), ("wide", 5)])
def test_probe_exact_order(bbc, oracle_lib, kind, nprobe, tc):
    h, idx, q = dev_index(bbc, kind)
    nq = len(q)
    out = torch.empty((nq, nprobe), dtype=torch.int32, device="cuda")
    bbc.bbc_set_param(h, "probe_gemm", tc)
    try:
        bbc.bbc_probe(h, cuda(q), nq, nprobe, out)
        sync_ok(bbc, h)
    finally:
        bbc.bbc_set_param(h, "probe_gemm", 1)
    got = out.cpu().numpy()
    for i in range(nq):
        ref, _ = oracle_lib.probe(q[i], idx.centroids, nprobe, idx.metric)
        assert np.array_equal(got[i], ref), f"query {i}"


def _collect(bbc, h, idx, q, nprobe, kc):
    nq = len(q)
    qd = cuda(q)
    lists = torch.empty((nq, nprobe), dtype=torch.int32, device="cuda")
    bbc.bbc_probe(h, qd, nq, nprobe, lists)
    ids = torch.full((nq, kc), -1, dtype=torch.int32, device="cuda")
    cnt = torch.empty(nq, dtype=torch.int64, device="cuda")
    st = torch.empty(nq * bbc.STATE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    bbc.bbc_collect(h, qd, nq, nprobe, lists, kc, ids, cnt, st)
    sync_ok(bbc, h)
    state = st.cpu().numpy().view(bbc.STATE_DTYPE)
    return lists.cpu().numpy(), ids.cpu().numpy().view(np.uint32), cnt.cpu().numpy(), state


# scan schedules: one CTA per query, two queries per CTA (pair form), several CTAs per query
MODES = {"single": (1, 0), "pair": (1, 1), "split": (0, 0)}


def set_mode(bbc, h, mode):
    split, pair = MODES[mode]
    bbc.bbc_set_param(h, "split", split)
    bbc.bbc_set_param(h, "pair", pair)


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("kind,nprobe,kc,m,smin", [
    ("tiny", 12, 300, 64, 8), ("tiny", 48, 5000, 32, 8), ("sift", 16, 900, 64, 8),
    ("sift4", 20, 1200, 256, 4), ("embed", 10, 400, 2, 8), ("ragged", 40, 300, 16, 3),
    ("ragged", 2, 1000, 64, 8), ("sift", 64, 12000, 64, 8), ("tiny", 5, 1, 64, 8),
    ("wide", 6, 1500, 64, 8)])
def test_collect_candidates_and_state(bbc, oracle_lib, kind, nprobe, kc, m, smin, mode):
    h, idx, q = dev_index(bbc, kind)
    bbc.bbc_set_param(h, "buckets", m)
    bbc.bbc_set_param(h, "sample_lists", smin)
    set_mode(bbc, h, mode)
    if mode == "pair":
        q = q[:len(q) - 1]                                # an odd batch: one CTA holds a single query
    try:
        lists, ids, cnt, state = _collect(bbc, h, idx, q, nprobe, kc)
    finally:
        bbc.bbc_set_param(h, "buckets", 64)
        bbc.bbc_set_param(h, "sample_lists", 8)
        set_mode(bbc, h, "split")
    for i in range(len(q)):
        ol, _ = oracle_lib.probe(q[i], idx.centroids, nprobe, idx.metric)
        assert np.array_equal(lists[i], ol)
        sel, lofs = scanned_set(idx, ol)
        t16 = oracle_lib.lut16(q[i], idx.codebooks, idx.metric)
        e = oracle_lib.adc(t16, idx.codes[sel], idx.pq_m, idx.pq_bits)
        sid = idx.ids[sel]
        ref_ids, _ = oracle_lib.topkc(e, sid, kc, "sort")
        n = int(cnt[i])
        assert n == min(kc, len(e))
        assert np.array_equal(np.sort(ids[i, :n].astype(np.int64)), np.sort(ref_ids)), f"query {i}"
        # collector state vs Algorithm 1 run by the oracle
        _, _, cb, counts = oracle_lib.bucket_collect(e, sid, lofs, kc, m, sample_min=smin)
        s = state[i]
        assert s["scanned"] == len(e)
        assert (s["d_min"], s["d_max"], s["sh"], s["sample_lists"]) == (cb.d_min, cb.d_max, cb.sh, cb.sample_lists)
        assert s["sample_size"] == cb.sample_size
        assert np.array_equal(s["map"], np.frombuffer(bytes(cb.map), dtype=np.uint8))
        assert s["tau"] == cb.tau
        t = min(cb.tau, m - 1) if cb.tau < m else m - 1
        if cb.tau < m:
            assert np.array_equal(s["hist"][:t + 1].astype(np.int64), counts[:t + 1])
            assert s["below"] == cb.below
        assert s["pushed"] >= min(kc, len(e))


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("kind,k,nprobe,ratio", [("tiny", 100, 12, 2.0), ("sift", 500, 16, 1.5),
                                                 ("sift4", 300, 24, 2.0), ("embed", 200, 10, 1.5),
                                                 ("ragged", 50, 40, 1.0), ("tiny", 1, 3, 1.0),
                                                 ("sift", 4000, 64, 1.0), ("wide", 300, 6, 2.0)])
def test_search_end_to_end(bbc, oracle_lib, kind, k, nprobe, ratio, mode):
    h, idx, q = dev_index(bbc, kind)
    bbc.bbc_set_param(h, "kc_ratio", ratio)
    set_mode(bbc, h, mode)
    kc = max(k, int(np.ceil(ratio * k - 1e-9)))
    nq = len(q)
    ids = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    dd = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    bbc.bbc_search(h, cuda(q), nq, k, nprobe, ids, dd)
    sync_ok(bbc, h)
    gi, gd = ids.cpu().numpy(), dd.cpu().numpy()
    set_mode(bbc, h, "split")
    oi, od = oracle_lib.search(idx, q, k, nprobe, kc, "sort")
    exact = kind in ("sift", "sift4")
    for i in range(nq):
        _check_topk(oracle_lib, idx, q[i], gi[i], gd[i], oi[i], od[i], exact)


def test_full_probe_full_candidates_is_exact_knn(bbc, oracle_lib):
    h, idx, q = dev_index(bbc, "ragged")
    k = 40
    bbc.bbc_set_param(h, "kc_ratio", float(idx.n) / k + 1)
    nq = len(q)
    ids = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    dd = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    bbc.bbc_search(h, cuda(q), nq, k, idx.nlist, ids, dd)
    sync_ok(bbc, h)
    bi, bd = oracle_lib.bruteforce(q, idx.vectors, k, idx.metric)
    for i in range(nq):
        _check_topk(oracle_lib, idx, q[i], ids[i].cpu().numpy(), dd[i].cpu().numpy(), bi[i], bd[i], False)


def test_padding_when_fewer_than_k_scanned(bbc):
    h, idx, q = dev_index(bbc, "ragged")
    bbc.bbc_set_param(h, "kc_ratio", 1.0)
    k = 300
    ids = torch.empty((2, k), dtype=torch.int64, device="cuda")
    dd = torch.empty((2, k), dtype=torch.float32, device="cuda")
    bbc.bbc_search(h, cuda(q[:2]), 2, k, 1, ids, dd)
    sync_ok(bbc, h)
    gi, gd = ids.cpu().numpy(), dd.cpu().numpy()
    lens = np.diff(idx.list_offsets)
    for i in range(2):
        n = int((gi[i] >= 0).sum())
        assert n < k and n in set(lens.tolist())
        assert (gi[i, n:] == -1).all() and np.isinf(gd[i, n:]).all()
        assert np.all(np.diff(gd[i, :n]) >= 0)


def test_host_entry_point_matches_device(bbc):
    h, idx, q = dev_index(bbc, "sift")
    bbc.bbc_set_param(h, "kc_ratio", 1.5)
    nq, k = len(q), 200
    ids = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    dd = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    bbc.bbc_search(h, cuda(q), nq, k, 16, ids, dd)
    hq = torch.from_numpy(q).pin_memory()
    hi = torch.empty((nq, k), dtype=torch.int64).pin_memory()
    hd = torch.empty((nq, k), dtype=torch.float32).pin_memory()
    bbc.bbc_search_host(h, hq, nq, k, 16, hi, hd)
    sync_ok(bbc, h)
    assert torch.equal(hi, ids.cpu()) and torch.equal(hd, dd.cpu())
    # a small workspace: many sub-batches whose result buffers alternate while copies overlap
    bbc.bbc_set_param(h, "workspace_mb", 1)
    try:
        hi2 = torch.empty((nq, k), dtype=torch.int64).pin_memory()
        hd2 = torch.empty((nq, k), dtype=torch.float32).pin_memory()
        bbc.bbc_search_host(h, hq, nq, k, 16, hi2, hd2)
        sync_ok(bbc, h)
    finally:
        bbc.bbc_set_param(h, "workspace_mb", 8192)
    assert torch.equal(hi2, ids.cpu()) and torch.equal(hd2, dd.cpu())


def test_chunked_workspace_same_result(bbc):
    h, idx, q = dev_index(bbc, "tiny")
    bbc.bbc_set_param(h, "kc_ratio", 2.0)
    nq, k = len(q), 64
    outs = []
    for mb in (8192, 1):
        bbc.bbc_set_param(h, "workspace_mb", mb)
        ids = torch.empty((nq, k), dtype=torch.int64, device="cuda")
        dd = torch.empty((nq, k), dtype=torch.float32, device="cuda")
        bbc.bbc_search(h, cuda(q), nq, k, 12, ids, dd)
        sync_ok(bbc, h)
        outs.append((ids.cpu(), dd.cpu()))
    bbc.bbc_set_param(h, "workspace_mb", 8192)
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


def test_argument_errors(bbc):
    h, idx, q = dev_index(bbc, "tiny")
    ids = torch.empty((1, 5), dtype=torch.int64, device="cuda")
    dd = torch.empty((1, 5), dtype=torch.float32, device="cuda")
    qd = cuda(q[:1])
    for k, nprobe in ((0, 4), (5, 0), (5, idx.nlist + 1)):
        with pytest.raises(bbc.BBCError) as ei:
            bbc.bbc_search(h, qd, 1, k, nprobe, ids, dd)
        assert ei.value.code == -1
    with pytest.raises(bbc.BBCError):
        bbc.bbc_set_param(h, "buckets", 1)
    with pytest.raises(bbc.BBCError):
        bbc.bbc_set_param(h, "no_such_key", 1)
    bbc.bbc_search(h, qd, 0, 5, 4, ids, dd)      # nq = 0 is a no-op


@pytest.mark.parametrize("mode", ["pair", "split"])
@pytest.mark.parametrize("kind", ["sift", "tiny", "sift4", "embed"])
def test_search_ex_mixed_batch_equals_alone(bbc, oracle_lib, kind, mode):
    """A mixed batch (different k and nprobe per query) returns, for every
    query, the oracle's result at that query's own k, nprobe and K_c
    (Algorithm 1's candidate set re-ranked), and exactly what searching that
    query alone returns."""
    h, idx, q = dev_index(bbc, kind)
    ratio = 1.5
    bbc.bbc_set_param(h, "kc_ratio", ratio)
    rng = np.random.default_rng(11)
    nq = len(q)
    ks = rng.integers(1, 1500, size=nq).astype(np.int32)
    ps = rng.integers(1, idx.nlist + 1, size=nq).astype(np.int32)
    tot = int(ks.sum())
    ids = torch.empty(tot, dtype=torch.int64, device="cuda")
    dd = torch.empty(tot, dtype=torch.float32, device="cuda")
    qd = cuda(q)
    set_mode(bbc, h, mode)
    try:
        bbc.bbc_search_ex(h, qd, nq, ks, ps, ids, dd)
        sync_ok(bbc, h)
    finally:
        set_mode(bbc, h, "split")
    gi, gd = ids.cpu().numpy(), dd.cpu().numpy()
    off = np.concatenate([[0], np.cumsum(ks)])
    exact = kind in ("sift", "sift4")
    for i in range(nq):
        k = int(ks[i])
        kc = max(k, int(np.ceil(ratio * k - 1e-9)))
        oi, od = oracle_lib.search(idx, q[i:i + 1], k, int(ps[i]), kc, "sort")
        _check_topk(oracle_lib, idx, q[i], gi[off[i]:off[i + 1]], gd[off[i]:off[i + 1]], oi[0], od[0], exact)
        ai = torch.empty((1, k), dtype=torch.int64, device="cuda")
        ad = torch.empty((1, k), dtype=torch.float32, device="cuda")
        bbc.bbc_search(h, qd[i:i + 1], 1, k, int(ps[i]), ai, ad)
        sync_ok(bbc, h)
        assert np.array_equal(gi[off[i]:off[i + 1]], ai.cpu().numpy()[0]), f"query {i}"
        assert np.array_equal(gd[off[i]:off[i + 1]], ad.cpu().numpy()[0]), f"query {i}"


def test_large_candidate_pool_topk(bbc, oracle_lib):
    """K_c above 16,384 (more candidates than the shared-memory top-k keeps), exact on integer data."""
    h, idx, q = dev_index(bbc, "medium")
    k, nprobe, ratio = 12000, 96, 1.5
    bbc.bbc_set_param(h, "kc_ratio", ratio)
    kc = int(np.ceil(ratio * k))
    assert kc > 16384
    nq = 6
    ids = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    dd = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    bbc.bbc_search(h, cuda(q[:nq]), nq, k, nprobe, ids, dd)
    sync_ok(bbc, h)
    oi, od = oracle_lib.search(idx, q[:nq], k, nprobe, kc, "sort")
    gi, gd = ids.cpu().numpy(), dd.cpu().numpy()
    for i in range(nq):
        _check_topk(oracle_lib, idx, q[i], gi[i], gd[i], oi[i], od[i], True)


@pytest.mark.parametrize("case,kc,k", [("ties", 30000, 25000), ("inner_product", 30000, 25000),
                                       ("ties", 30000, 20000), ("inner_product", 30000, 20000),
                                       ("ties", 12000, 5000), ("ties", 12000, 11500), ("ties", 12000, 1),
                                       ("inner_product", 12000, 3000)])
@pytest.mark.parametrize("fused", [1, 0])
def test_topk_heavy_bins_and_sign_span(bbc, oracle_lib, case, kc, k, fused):
    """Top-k on candidates with thousands of equal distances and on inner
    products whose distances span the sign boundary.  k = 25,000 takes the
    global-scratch form (its kept keys exceed shared memory; one block of ties
    above its shared-memory sort, one within it); k = 20,000 over 30,000
    candidates the shared-memory form with more candidates than it keeps;
    K_c = 12,000 the shared-memory form, where a block of ties holds the k-th
    place (k = 5,000: selected inside the bin) or lies below it (k = 11,500:
    the bin is sorted in place).  fused = 1: re-rank and top-k in one kernel
    where the K_c = 12,000 candidates fit in its shared memory."""
    from synth import build_ivf_pq
    from synth.data import sift_shaped, embedding_shaped
    if case == "ties":
        x, q = sift_shaped(30000, 3, d=128, n_centers=200)
        x[:10000] = x[0]
        x[10000:15000] = x[10000]
        idx = build_ivf_pq(x, 16, 16, 8, "l2", kmeans_iters=3, pq_iters=3, pq_sample=5000)
        q = np.stack([x[0] + 1.0, x[10000], q[0]]).astype(np.float32)
    else:
        x, q = embedding_shaped(30000, 3, d=64)
        idx = build_ivf_pq(x, 16, 16, 8, "ip", kmeans_iters=3, pq_iters=3, pq_sample=5000)
    h = bbc.bbc_index_create(idx, 0)
    try:
        bbc.bbc_set_param(h, "rerank_fused", fused)
        nq = len(q)
        cand = np.tile(np.arange(kc, dtype=np.uint32), (nq, 1))
        cnt = np.full(nq, kc, dtype=np.int64)
        gi = torch.empty((nq, k), dtype=torch.int64, device="cuda")
        gd = torch.empty((nq, k), dtype=torch.float32, device="cuda")
        bbc.bbc_rerank_topk(h, cuda(q), nq, cuda(cand), cuda(cnt), kc, k, gi, gd)
        sync_ok(bbc, h)
        gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
        for i in range(nq):
            d64 = oracle_lib.rerank(q[i], idx.vectors, cand[i].astype(np.int64), idx.metric)
            oi, od = oracle_lib.topk_final(d64, cand[i].astype(np.int64), k)
            _check_topk(oracle_lib, idx, q[i], gi[i], gd[i], oi, od, case == "ties")
    finally:
        bbc.bbc_index_free(h)


@pytest.mark.parametrize("d", [128, 64])
@pytest.mark.parametrize("frac", [0.0, 0.37])
@pytest.mark.parametrize("fused", [1, 0])
def test_rerank_integer_rows_integer_and_fractional_queries(bbc, oracle_lib, d, frac, fused):
    """Re-rank + top-k over the exact u8 copy: integer queries take the integer
    dot-product path (bit-exact), fractional ones the FP32 path (1e-5 of FP64);
    d = 128 runs the fixed-shape kernel, d = 64 the general one."""
    from synth import build_ivf_pq
    from synth.data import sift_shaped
    x, q = sift_shaped(20000, 4, d=d, n_centers=100)
    idx = build_ivf_pq(x, 16, d // 8, 8, "l2", kmeans_iters=3, pq_iters=3, pq_sample=5000)
    h = bbc.bbc_index_create(idx, 0)
    try:
        assert bbc.bbc_index_info(h)["vectors_u8_exact"] == 1
        bbc.bbc_set_param(h, "rerank_fused", fused)
        q = (q + np.float32(frac)).astype(np.float32)
        nq, kc, k = len(q), 12000, 3000
        cand = np.tile(np.arange(kc, dtype=np.uint32), (nq, 1))
        cnt = np.full(nq, kc, dtype=np.int64)
        gi = torch.empty((nq, k), dtype=torch.int64, device="cuda")
        gd = torch.empty((nq, k), dtype=torch.float32, device="cuda")
        bbc.bbc_rerank_topk(h, cuda(q), nq, cuda(cand), cuda(cnt), kc, k, gi, gd)
        sync_ok(bbc, h)
        gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
        for i in range(nq):
            d64 = oracle_lib.rerank(q[i], idx.vectors, cand[i].astype(np.int64), "l2")
            oi, od = oracle_lib.topk_final(d64, cand[i].astype(np.int64), k)
            _check_topk(oracle_lib, idx, q[i], gi[i], gd[i], oi, od, frac == 0.0)
    finally:
        bbc.bbc_index_free(h)


@pytest.mark.parametrize("kind,k,nprobe,ratio,rows", [("tiny", 100, 12, 2.0, "auto"), ("sift", 500, 16, 1.5, "auto"),
                                                      ("sift", 4000, 64, 1.0, "auto"), ("sift", 500, 16, 1.5, "early"),
                                                      ("sift", 500, 16, 1.5, "f32"), ("embed", 200, 10, 1.5, "auto"),
                                                      ("ragged", 50, 40, 1.0, "auto"), ("wide", 300, 6, 2.0, "auto"),
                                                      ("tiny", 1, 3, 1.0, "auto")])
def test_rerank_fused_equals_two_kernels(bbc, oracle_lib, kind, k, nprobe, ratio, rows):
    """The one-kernel re-rank + top-k (each query's distances kept in shared
    memory) returns, bit for bit, what the re-rank kernel followed by the top-k
    kernel returns: integer rows (u8 path), FP32 rows of 512 bytes and of other
    widths (rows = "f32": the FP32 vectors of integer data), and the early
    re-rank's variant (rows = "early").  The stage profile shows which path
    ran (the fused kernel is timed as the re-rank stage, the top-k stage stays
    empty)."""
    h, idx, q = dev_index(bbc, kind)
    bbc.bbc_set_param(h, "kc_ratio", ratio)
    nq = len(q)
    outs = []
    try:
        if rows == "early":
            bbc.bbc_set_param(h, "split", 1)
            bbc.bbc_set_param(h, "early_rerank", 1)
        if rows == "f32":
            bbc.bbc_set_param(h, "rerank", 0)
        bbc.bbc_set_param(h, "profile", 1)
        for fused in (0, 1):
            bbc.bbc_set_param(h, "rerank_fused", fused)
            bbc.bbc_profile_read(h, reset=True)
            gi = torch.empty((nq, k), dtype=torch.int64, device="cuda")
            gd = torch.empty((nq, k), dtype=torch.float32, device="cuda")
            bbc.bbc_search(h, cuda(q), nq, k, nprobe, gi, gd)
            sync_ok(bbc, h)
            stages, _ = bbc.bbc_profile_read(h, reset=True)
            outs.append((gi.cpu().numpy(), gd.cpu().numpy(), stages))
    finally:
        bbc.bbc_set_param(h, "profile", 0)
        bbc.bbc_set_param(h, "rerank_fused", 0)
        if rows == "early":
            bbc.bbc_set_param(h, "early_rerank", 0)
            bbc.bbc_set_param(h, "split", 0)
        if rows == "f32":
            bbc.bbc_set_param(h, "rerank", 1)
    assert outs[0][2]["topk"] > 0.0 and outs[1][2]["topk"] == 0.0 and outs[1][2]["rerank"] > 0.0
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    kc = max(k, int(np.ceil(ratio * k - 1e-9)))
    oi, od = oracle_lib.search(idx, q, k, nprobe, kc, "sort")
    exact = kind in ("sift", "sift4")
    for i in range(nq):
        _check_topk(oracle_lib, idx, q[i], outs[1][0][i], outs[1][1][i], oi[i], od[i], exact)


@pytest.mark.parametrize("kind", ["tiny", "sift", "ragged"])
def test_split_scan_equals_one_cta_per_query(bbc, kind):
    """Several CTAs per query (persistent (query, part) items, global collector
    state) and two queries per CTA (pair form) give exactly the candidates,
    threshold and results of one CTA per query."""
    h, idx, q = dev_index(bbc, kind)
    nq, k, nprobe = len(q), 150, min(idx.nlist, 24)
    bbc.bbc_set_param(h, "kc_ratio", 2.0)
    outs = {}
    try:
        for split in (1, 2, 7, 64, "pair"):
            bbc.bbc_set_param(h, "pair", 1 if split == "pair" else 0)
            bbc.bbc_set_param(h, "split", 1 if split == "pair" else split)
            lists, ids, cnt, state = _collect(bbc, h, idx, q, nprobe, 2 * k)
            ri = torch.empty((nq, k), dtype=torch.int64, device="cuda")
            rd = torch.empty((nq, k), dtype=torch.float32, device="cuda")
            bbc.bbc_search(h, cuda(q), nq, k, nprobe, ri, rd)
            sync_ok(bbc, h)
            cands = [np.sort(ids[i, :cnt[i]]) for i in range(nq)]
            outs[split] = (cands, cnt, state, ri.cpu().numpy(), rd.cpu().numpy())
    finally:
        bbc.bbc_set_param(h, "split", 0)
        bbc.bbc_set_param(h, "pair", 0)
    ref = outs[1]
    for split in (2, 7, 64, "pair"):
        got = outs[split]
        assert np.array_equal(got[1], ref[1])
        for i in range(nq):
            assert np.array_equal(got[0][i], ref[0][i]), (split, i)
        for f in ("d_min", "d_max", "sh", "sample_lists", "sample_size", "scanned", "tau", "below"):
            assert np.array_equal(got[2][f], ref[2][f]), (split, f)
        assert np.array_equal(got[3], ref[3]) and np.array_equal(got[4], ref[4]), split


def test_graph_replay_matches_eager(bbc):
    """With 'graphs' on, the first call captures and the next ones replay; a
    replay reads the current contents of the same query buffer."""
    h, idx, q = dev_index(bbc, "sift")
    bbc.bbc_set_param(h, "kc_ratio", 1.5)
    nq, k, nprobe = len(q), 300, 16
    side = torch.cuda.Stream()
    qd = cuda(q)
    eager_i = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    eager_d = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    bbc.bbc_search(h, qd, nq, k, nprobe, eager_i, eager_d, side)
    qflip = cuda(q[::-1].copy())
    flip_i = torch.empty_like(eager_i)
    flip_d = torch.empty_like(eager_d)
    bbc.bbc_search(h, qflip, nq, k, nprobe, flip_i, flip_d, side)
    side.synchronize()
    bbc.bbc_set_param(h, "graphs", 1)
    try:
        gi = torch.empty_like(eager_i)
        gd = torch.empty_like(eager_d)
        qbuf = qd.clone()
        for rep in range(3):
            bbc.bbc_search(h, qbuf, nq, k, nprobe, gi, gd, side)
            side.synchronize()
            assert torch.equal(gi, eager_i) and torch.equal(gd, eager_d), rep
        qbuf.copy_(qflip)
        torch.cuda.synchronize()
        bbc.bbc_search(h, qbuf, nq, k, nprobe, gi, gd, side)
        side.synchronize()
        assert torch.equal(gi, flip_i) and torch.equal(gd, flip_d)
    finally:
        bbc.bbc_set_param(h, "graphs", 0)
    bbc.bbc_stream_status(h, side)


def test_autotune_picks_and_caches(bbc, tmp_path):
    h, idx, q = dev_index(bbc, "tiny")
    bbc.bbc_set_param(h, "kc_ratio", 2.0)
    nq, k, nprobe = len(q), 100, 12
    qd = cuda(q)
    ref_i = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    ref_d = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    bbc.bbc_search(h, qd, nq, k, nprobe, ref_i, ref_d)
    cache = str(tmp_path / "tune.jsonl")
    try:
        ms = bbc.bbc_autotune(h, qd, nq, k, nprobe, cache)
        assert ms > 0
        chosen = (bbc.bbc_get_param(h, "split"), bbc.bbc_get_param(h, "buckets"), bbc.bbc_get_param(h, "pair"))
        assert open(cache).read().count('"split"') == 1
        bbc.bbc_set_param(h, "split", 0)
        bbc.bbc_set_param(h, "buckets", 64)
        bbc.bbc_set_param(h, "pair", 1 - chosen[2])
        assert bbc.bbc_autotune(h, qd, nq, k, nprobe, cache) == 0.0          # from the cache
        assert (bbc.bbc_get_param(h, "split"), bbc.bbc_get_param(h, "buckets"), bbc.bbc_get_param(h, "pair")) == chosen
        gi = torch.empty_like(ref_i)
        gd = torch.empty_like(ref_d)
        bbc.bbc_search(h, qd, nq, k, nprobe, gi, gd)
        sync_ok(bbc, h)
        assert torch.equal(gi, ref_i) and torch.equal(gd, ref_d)
    finally:
        bbc.bbc_set_param(h, "split", 0)
        bbc.bbc_set_param(h, "buckets", 64)
        bbc.bbc_set_param(h, "pair", 0)


@pytest.mark.parametrize("nq", [2, 3, 5, 33])
def test_pair_form_small_and_degenerate_batches(bbc, oracle_lib, nq):
    """The pair form on tiny batches (an odd query left alone), on duplicated
    queries (a pair at distance 0) and on queries far apart (nearly disjoint
    probe sets): candidates equal the oracle's top-K_c and the one-CTA form's."""
    h, idx, q = dev_index(bbc, "sift")
    rng = np.random.default_rng(nq)
    sel = rng.integers(0, len(q), size=nq)
    qs = q[sel].copy()
    if nq >= 3:
        qs[1] = qs[0]                                     # identical queries
        qs[2] = 255.0 - qs[0]                             # a query far from the others
    nprobe, kc = 20, 700
    outs = []
    try:
        for pair in (0, 1):
            bbc.bbc_set_param(h, "split", 1)
            bbc.bbc_set_param(h, "pair", pair)
            outs.append(_collect(bbc, h, idx, qs, nprobe, kc))
    finally:
        bbc.bbc_set_param(h, "split", 0)
        bbc.bbc_set_param(h, "pair", 0)
    (l0, i0, c0, s0), (l1, i1, c1, s1) = outs
    assert np.array_equal(c0, c1)
    for f in ("d_min", "d_max", "sh", "sample_lists", "sample_size", "scanned", "tau", "below"):
        assert np.array_equal(s0[f], s1[f]), f
    for i in range(nq):
        assert np.array_equal(np.sort(i0[i, :c0[i]]), np.sort(i1[i, :c1[i]])), i
        sel_pos, _ = scanned_set(idx, l1[i])
        t16 = oracle_lib.lut16(qs[i], idx.codebooks, idx.metric)
        e = oracle_lib.adc(t16, idx.codes[sel_pos], idx.pq_m, idx.pq_bits)
        ref_ids, _ = oracle_lib.topkc(e, idx.ids[sel_pos], kc, "sort")
        assert np.array_equal(np.sort(i1[i, :c1[i]].astype(np.int64)), np.sort(ref_ids)), i


def test_pair_form_many_plan_blocks(bbc):
    """More queries than one pairing block (16,384): pairs never cross blocks and
    every query's candidates equal those of the one-CTA form."""
    h, idx, q = dev_index(bbc, "tiny")
    rng = np.random.default_rng(3)
    nq = 16384 + 1001
    qs = (q[rng.integers(0, len(q), size=nq)] + rng.normal(0, 0.05, size=(nq, idx.d))).astype(np.float32)
    nprobe, kc = 6, 200
    outs = []
    try:
        for pair in (0, 1):
            bbc.bbc_set_param(h, "split", 1)
            bbc.bbc_set_param(h, "pair", pair)
            outs.append(_collect(bbc, h, idx, qs, nprobe, kc))
    finally:
        bbc.bbc_set_param(h, "split", 0)
        bbc.bbc_set_param(h, "pair", 0)
    (_, i0, c0, s0), (_, i1, c1, s1) = outs
    assert np.array_equal(c0, c1)
    assert np.array_equal(s0["tau"], s1["tau"]) and np.array_equal(s0["below"], s1["below"])
    a = np.sort(np.where(np.arange(kc)[None, :] < c0[:, None], i0, 0xFFFFFFFF), axis=1)
    b = np.sort(np.where(np.arange(kc)[None, :] < c1[:, None], i1, 0xFFFFFFFF), axis=1)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("collector", [1, 2])
@pytest.mark.parametrize("kind,nprobe,kc", [("tiny", 12, 300), ("sift", 16, 900), ("sift4", 20, 1200),
                                            ("ragged", 40, 300), ("sift", 64, 12000), ("tiny", 5, 1)])
def test_baseline_collectors_same_candidates(bbc, oracle_lib, kind, nprobe, kc, collector):
    """The lazy linear buffer and the binary heap (the collectors the result
    buffer is compared with) collect exactly the oracle's top-K_c by
    (estimated distance, id), and the whole search returns the same results."""
    h, idx, q = dev_index(bbc, kind)
    bbc.bbc_set_param(h, "collector", collector)
    try:
        lists, ids, cnt, state = _collect(bbc, h, idx, q, nprobe, kc)
    finally:
        bbc.bbc_set_param(h, "collector", 0)
    for i in range(len(q)):
        sel, _ = scanned_set(idx, lists[i])
        t16 = oracle_lib.lut16(q[i], idx.codebooks, idx.metric)
        e = oracle_lib.adc(t16, idx.codes[sel], idx.pq_m, idx.pq_bits)
        ref_ids, _ = oracle_lib.topkc(e, idx.ids[sel], kc, "sort")
        n = int(cnt[i])
        assert n == min(kc, len(e))
        assert np.array_equal(np.sort(ids[i, :n].astype(np.int64)), np.sort(ref_ids)), f"query {i}"
        assert state[i]["scanned"] == len(e)
    k = max(1, kc // 2)
    outs = []
    for c in (0, collector):
        bbc.bbc_set_param(h, "collector", c)
        bbc.bbc_set_param(h, "kc_ratio", kc / k)
        gi = torch.empty((len(q), k), dtype=torch.int64, device="cuda")
        gd = torch.empty((len(q), k), dtype=torch.float32, device="cuda")
        bbc.bbc_search(h, cuda(q), len(q), k, nprobe, gi, gd)
        sync_ok(bbc, h)
        outs.append((gi.cpu(), gd.cpu()))
    bbc.bbc_set_param(h, "collector", 0)
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("k,nprobe,ratio", [(500, 16, 1.5), (4000, 64, 1.0), (60, 3, 2.0)])
def test_early_rerank_same_results(bbc, oracle_lib, k, nprobe, ratio):
    """Algorithm 4's early re-rank computes some candidates' exact distances
    during the scan; candidates and results stay the oracle's, bit for bit
    (integer data), and the re-rank uses early distances it was given."""
    h, idx, q = dev_index(bbc, "sift")
    qs = q.copy()
    qs[1] += 0.5                                         # a fractional query: nothing scored early for it
    nq = len(qs)
    bbc.bbc_set_param(h, "kc_ratio", ratio)
    bbc.bbc_set_param(h, "split", 1)
    outs = []
    try:
        for early in (0, 1):
            bbc.bbc_set_param(h, "early_rerank", early)
            bbc.bbc_early_stats(h, reset=True)
            gi = torch.empty((nq, k), dtype=torch.int64, device="cuda")
            gd = torch.empty((nq, k), dtype=torch.float32, device="cuda")
            bbc.bbc_search(h, cuda(qs), nq, k, nprobe, gi, gd)
            sync_ok(bbc, h)
            outs.append((gi.cpu().numpy(), gd.cpu().numpy(), bbc.bbc_early_stats(h, reset=True)))
    finally:
        bbc.bbc_set_param(h, "early_rerank", 0)
        bbc.bbc_set_param(h, "split", 0)
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    st = outs[1][2]
    kc = max(k, int(np.ceil(ratio * k - 1e-9)))
    if nprobe <= 8:
        # the sample (at least 8 lists) covers every probed list: nothing is scanned after the
        # first predicted threshold exists (the oracle's special case of Algorithm 4)
        assert st["scored_early"] == 0 and st["used"] == 0
    else:
        assert 0 < st["used"] <= st["scored_early"] and st["used"] <= nq * kc
    oi, od = oracle_lib.search(idx, qs, k, nprobe, kc, "sort")
    for i in range(nq):
        _check_topk(oracle_lib, idx, qs[i], outs[1][0][i], outs[1][1][i], oi[i], od[i], i != 1)


def test_early_rerank_refused_where_it_does_not_apply(bbc):
    h, idx, q = dev_index(bbc, "tiny")                   # FP32 data: no exact u8 copy
    with pytest.raises(bbc.BBCError) as ei:
        bbc.bbc_set_param(h, "early_rerank", 1)
    assert ei.value.code == -9
