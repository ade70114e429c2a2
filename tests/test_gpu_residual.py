"""Residual IVF-PQ on the device vs the CPU oracle, through the C ABI.

The codes quantise each object's residual o - c_l; the scan's integer keys
are the table sum plus a per-(query, list) base and a per-object term, all
decided in FP32 in a fixed order, so the candidate sets and the result
buffer's state match the oracle's bit for bit.  End-to-end results follow
the tolerance rules of the plain path (bit-exact on integer data).
"""

import numpy as np
import pytest

from conftest import check_topk, scanned_set, small_workload

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
        assert idx.residual
        _IDX[kind] = (bbc.bbc_index_create(idx, 0), idx, q)
    return _IDX[kind]


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def sync_ok(bbc, h):
    torch.cuda.synchronize()
    bbc.bbc_stream_status(h)


def oracle_keys(oracle_lib, idx, qv, lists):
    """The oracle's residual keys of the probed lists' objects, in probe order."""
    t16 = oracle_lib.lut16(qv, idx.codebooks, idx.metric)
    inv, _ = oracle_lib.lut16_scale(qv, idx.codebooks, idx.metric)
    parts = []
    for l in lists:
        a, b = idx.list_offsets[l], idx.list_offsets[l + 1]
        parts.append(oracle_lib.adc_resid(t16, idx.codes[a:b], qv, idx.centroids[l], idx.codebooks, inv,
                                          idx.metric))
    return np.concatenate(parts) if parts else np.zeros(0, np.uint32)


MODES = {"single": (1, 0), "split": (0, 0), "pair": (1, 1)}   # pair: falls back to one query per CTA


def set_mode(bbc, h, mode):
    split, pair = MODES[mode]
    bbc.bbc_set_param(h, "split", split)
    bbc.bbc_set_param(h, "pair", pair)


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("kind,nprobe,kc,m,smin", [
    ("rtiny", 12, 300, 64, 8), ("rtiny", 48, 5000, 32, 8), ("rsift", 16, 900, 64, 8),
    ("rsift4", 20, 1200, 256, 4), ("rembed", 10, 400, 2, 8), ("rragged", 40, 300, 16, 3),
    ("rragged", 2, 1000, 64, 8), ("rsift", 64, 12000, 64, 8), ("rtiny", 5, 1, 64, 8),
    ("rsift", 1, 50, 64, 8)])
def test_residual_candidates_and_state(bbc, oracle_lib, kind, nprobe, kc, m, smin, mode):
    h, idx, q = dev_index(bbc, kind)
    bbc.bbc_set_param(h, "buckets", m)
    bbc.bbc_set_param(h, "sample_lists", smin)
    set_mode(bbc, h, mode)
    nq = len(q)
    try:
        qd = cuda(q)
        lists = torch.empty((nq, nprobe), dtype=torch.int32, device="cuda")
        bbc.bbc_probe(h, qd, nq, nprobe, lists)
        ids = torch.full((nq, kc), -1, dtype=torch.int32, device="cuda")
        cnt = torch.empty(nq, dtype=torch.int64, device="cuda")
        st = torch.empty(nq * bbc.STATE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        bbc.bbc_collect(h, qd, nq, nprobe, lists, kc, ids, cnt, st)
        sync_ok(bbc, h)
    finally:
        bbc.bbc_set_param(h, "buckets", 64)
        bbc.bbc_set_param(h, "sample_lists", 8)
        set_mode(bbc, h, "split")
    lists = lists.cpu().numpy()
    ids = ids.cpu().numpy().view(np.uint32)
    cnt = cnt.cpu().numpy()
    state = st.cpu().numpy().view(bbc.STATE_DTYPE)
    for i in range(nq):
        ol, _ = oracle_lib.probe(q[i], idx.centroids, nprobe, idx.metric)
        assert np.array_equal(lists[i], ol)
        sel, lofs = scanned_set(idx, ol)
        e = oracle_keys(oracle_lib, idx, q[i], ol)
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


@pytest.mark.parametrize("mode", ["single", "split"])
@pytest.mark.parametrize("kind,k,nprobe,ratio", [("rtiny", 100, 12, 2.0), ("rsift", 500, 16, 1.5),
                                                 ("rsift4", 300, 24, 2.0), ("rembed", 200, 10, 1.5),
                                                 ("rragged", 50, 40, 1.0), ("rtiny", 1, 3, 1.0),
                                                 ("rsift", 4000, 64, 1.0)])
def test_residual_search_end_to_end(bbc, oracle_lib, kind, k, nprobe, ratio, mode):
    h, idx, q = dev_index(bbc, kind)
    bbc.bbc_set_param(h, "kc_ratio", ratio)
    set_mode(bbc, h, mode)
    kc = max(k, int(np.ceil(ratio * k - 1e-9)))
    nq = len(q)
    ids = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    dd = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    bbc.bbc_search(h, cuda(q), nq, k, nprobe, ids, dd)
    sync_ok(bbc, h)
    set_mode(bbc, h, "split")
    gi, gd = ids.cpu().numpy(), dd.cpu().numpy()
    oi, od = oracle_lib.search(idx, q, k, nprobe, kc, "sort")
    exact = kind in ("rsift", "rsift4")
    for i in range(nq):
        check_topk(oracle_lib, idx, q[i], gi[i], gd[i], oi[i], od[i], exact)


def test_residual_mixed_batch_vs_oracle(bbc, oracle_lib):
    h, idx, q = dev_index(bbc, "rsift")
    bbc.bbc_set_param(h, "kc_ratio", 1.5)
    nq = len(q)
    rng = np.random.default_rng(11)
    ks = rng.choice([10, 200, 700], size=nq).astype(np.int32)
    nps = rng.choice([1, 8, 24, 64], size=nq).astype(np.int32)
    tot = int(ks.sum())
    ids = torch.empty(tot, dtype=torch.int64, device="cuda")
    dd = torch.empty(tot, dtype=torch.float32, device="cuda")
    bbc.bbc_search_ex(h, cuda(q), nq, ks, nps, ids, dd)
    sync_ok(bbc, h)
    gi, gd = ids.cpu().numpy(), dd.cpu().numpy()
    off = 0
    for i in range(nq):
        k, npb = int(ks[i]), int(nps[i])
        kc = max(k, int(np.ceil(1.5 * k - 1e-9)))
        oi, od = oracle_lib.search(idx, q[i:i + 1], k, npb, kc, "sort")
        check_topk(oracle_lib, idx, q[i], gi[off:off + k], gd[off:off + k], oi[0], od[0], True)
        off += k


def test_residual_static_collect_equals_collect(bbc):
    h, idx, q = dev_index(bbc, "rsift")
    nq, nprobe, kc = len(q), 16, 800
    qd = cuda(q)
    lists = torch.empty((nq, nprobe), dtype=torch.int32, device="cuda")
    bbc.bbc_probe(h, qd, nq, nprobe, lists)
    out = []
    for fn in (bbc.bbc_collect, bbc.bbc_collect_static):
        ids = torch.full((nq, kc), -1, dtype=torch.int32, device="cuda")
        cnt = torch.empty(nq, dtype=torch.int64, device="cuda")
        fn(h, qd, nq, nprobe, lists, kc, ids, cnt, None)
        sync_ok(bbc, h)
        out.append((np.sort(ids.cpu().numpy(), axis=1), cnt.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_residual_refusals(bbc):
    h, idx, q = dev_index(bbc, "rsift")
    with pytest.raises(bbc.BBCError):
        bbc.bbc_set_param(h, "early_rerank", 1)
    bbc.bbc_set_param(h, "collector", 1)
    try:
        ids = torch.empty((2, 10), dtype=torch.int64, device="cuda")
        dd = torch.empty((2, 10), dtype=torch.float32, device="cuda")
        with pytest.raises(bbc.BBCError):
            bbc.bbc_search(h, cuda(q[:2]), 2, 10, 8, ids, dd)
    finally:
        bbc.bbc_set_param(h, "collector", 0)
    assert bbc.bbc_index_info(h)["quantizer"] == 2


def test_residual_index_file_round_trip(bbc, oracle_lib, tmp_path):
    from synth.index import write_index
    h, idx, q = dev_index(bbc, "rtiny")
    path = str(tmp_path / "rtiny.bbcidx")
    write_index(path, idx)
    hl = bbc.bbc_index_load(path, 0)
    try:
        assert bbc.bbc_index_info(hl)["quantizer"] == 2
        nq, k, nprobe = len(q), 50, 12
        res = []
        for hh in (h, hl):
            bbc.bbc_set_param(hh, "kc_ratio", 1.5)           # same parameters on both handles
            set_mode(bbc, hh, "split")
            ids = torch.empty((nq, k), dtype=torch.int64, device="cuda")
            dd = torch.empty((nq, k), dtype=torch.float32, device="cuda")
            bbc.bbc_search(hh, cuda(q), nq, k, nprobe, ids, dd)
            sync_ok(bbc, hh)
            res.append((ids.cpu().numpy(), dd.cpu().numpy()))
        assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    finally:
        bbc.bbc_index_free(hl)
