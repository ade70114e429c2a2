"""Precision form of the re-rank (BF16 / FP8-E4M3 copies) vs the CPU oracle.

* The copies are compared byte for byte with the oracle's, built from the
  formats' definitions; the per-vector error and norm must bound the oracle's.
* Every candidate's low-precision score d^ must lie within its bound rho of
  the FP64 distance: |d^ - d64| <= rho (the bound invariant).
* The final set must equal the oracle's k smallest (d64, id) exactly: the
  bounds only decide what they can prove, FP32 and FP64 decide the rest.
  Reported distances lie within the bound of d64, and the output is sorted by
  them.
"""

import numpy as np
import pytest

from conftest import scanned_set, small_workload

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


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def sync_ok(bbc, h):
    torch.cuda.synchronize()
    bbc.bbc_stream_status(h)


class precision:
    """Sets 'precision' (and 'rerank' 0 for integer data) for a block."""

    def __init__(self, bbc, h, prec, **extra):
        self.bbc, self.h, self.prec, self.extra = bbc, h, prec, extra

    def __enter__(self):
        self.old = {k: self.bbc.bbc_get_param(self.h, k) for k in self.extra}
        for k, v in self.extra.items():
            self.bbc.bbc_set_param(self.h, k, v)
        self.bbc.bbc_set_param(self.h, "precision", self.prec)

    def __exit__(self, *a):
        self.bbc.bbc_set_param(self.h, "precision", 0)
        for k, v in self.old.items():
            self.bbc.bbc_set_param(self.h, k, v)


def oracle_candidates(oracle_lib, idx, q, nprobe, kc):
    """Per query: the K_c smallest (ADC estimate, id) of the probed lists."""
    out = []
    for i in range(len(q)):
        ol, _ = oracle_lib.probe(q[i], idx.centroids, nprobe, idx.metric)
        sel, _ = scanned_set(idx, ol)
        t16 = oracle_lib.lut16(q[i], idx.codebooks, idx.metric)
        e = oracle_lib.adc(t16, idx.codes[sel], idx.pq_m, idx.pq_bits)
        ids, _ = oracle_lib.topkc(e, idx.ids[sel], kc, "sort")
        out.append(np.asarray(ids, dtype=np.int64))
    return out


def pack(cands, kc):
    nq = len(cands)
    a = np.zeros((nq, kc), dtype=np.uint32)
    cnt = np.zeros(nq, dtype=np.int64)
    for i, c in enumerate(cands):
        a[i, :len(c)] = c
        cnt[i] = len(c)
    return a, cnt


def bounds_of(bbc, h, q, ids_list, kc):
    """d^ and rho of the given ids per query (through the bounds entry point)."""
    a, cnt = pack(ids_list, kc)
    dd = torch.zeros((len(q), kc), dtype=torch.float32, device="cuda")
    rr = torch.zeros((len(q), kc), dtype=torch.float32, device="cuda")
    bbc.bbc_rerank_bounds(h, cuda(q), len(q), cuda(a), cuda(cnt), kc, dd, rr)
    sync_ok(bbc, h)
    return dd.cpu().numpy().astype(np.float64), rr.cpu().numpy().astype(np.float64)


def check_result(oracle_lib, bbc, h, idx, q, gi, gd, oi, kc):
    """Set equality with the oracle, padding, sort order and distance bounds."""
    nq, k = gi.shape
    ids_list = []
    for i in range(nq):
        valid = oi[i] >= 0
        assert np.array_equal(gi[i] >= 0, valid), f"query {i}: padding"
        assert np.all(np.isinf(gd[i][~valid]))
        assert set(gi[i][valid].tolist()) == set(oi[i][valid].tolist()), f"query {i}: result set"
        v = gd[i][valid].astype(np.float64)
        assert np.all(np.diff(v) >= 0), f"query {i}: not sorted"
        ids_list.append(gi[i][valid])
    dh, rho = bounds_of(bbc, h, q, ids_list, max(k, 1))
    for i in range(nq):
        g = ids_list[i]
        if len(g) == 0:
            continue
        d64 = oracle_lib.rerank(q[i], idx.vectors, g, idx.metric)
        err = np.abs(gd[i][:len(g)].astype(np.float64) - d64)
        # the reported distance is d^, d32 or d64: each within the copy's bound or FP32 rounding
        lim = np.maximum(rho[i, :len(g)], 2e-6 * np.abs(d64) + 1e-30)
        assert np.all(err <= lim), (i, float((err / lim).max()))


KINDS = [("tiny", 1), ("tiny", 2), ("embed", 1), ("embed", 2), ("pad", 1), ("pad", 2), ("wide", 1), ("wide", 2)]


@pytest.mark.parametrize("kind,prec", KINDS + [("sift", 2)])
def test_copy_matches_oracle(bbc, oracle_lib, kind, prec):
    h, idx, q = dev_index(bbc, kind)
    with precision(bbc, h, prec, **({"rerank": 0} if kind == "sift" else {})):
        dpad = (idx.d + 15) // 16 * 16
        rows = torch.zeros(idx.n * dpad * (2 if prec == 1 else 1), dtype=torch.uint8, device="cuda")
        meta = torch.zeros((idx.n, 4), dtype=torch.float32, device="cuda")
        bbc.bbc_precision_copy(h, rows, meta)
        sync_ok(bbc, h)
    got = rows.cpu().numpy().view(np.uint16 if prec == 1 else np.uint8).reshape(idx.n, dpad)
    gm = meta.cpu().numpy().astype(np.float64)
    ref, rm = oracle_lib.prec_copy(idx.vectors, prec)
    assert np.array_equal(got, ref)
    assert np.array_equal(gm[:, 0], rm[:, 0])
    for col in (1, 2):                       # rounded up, within a few ulps of the FP64 value
        assert np.all(gm[:, col] >= rm[:, col])
        assert np.all(gm[:, col] <= rm[:, col] * (1 + 1e-6) + 1e-37)


@pytest.mark.parametrize("kind,prec", KINDS + [("sift", 1), ("sift", 2)])
def test_bound_invariant(bbc, oracle_lib, kind, prec):
    h, idx, q = dev_index(bbc, kind)
    nprobe, kc = min(16, idx.nlist), 1500
    cands = oracle_candidates(oracle_lib, idx, q, nprobe, kc)
    with precision(bbc, h, prec, **({"rerank": 0} if kind == "sift" else {})):
        dh, rho = bounds_of(bbc, h, q, cands, kc)
    worst = 0.0
    for i, c in enumerate(cands):
        d64 = oracle_lib.rerank(q[i], idx.vectors, c, idx.metric)
        n = len(c)
        err = np.abs(dh[i, :n] - d64)
        assert np.all(np.isfinite(rho[i, :n]))
        assert np.all(err <= rho[i, :n]), (i, float((err / rho[i, :n]).max()))
        worst = max(worst, float((err / rho[i, :n]).max()))
        # not vacuous: the bound is well below the spread of the candidates' distances
        spread = d64.max() - d64.min()
        assert np.median(rho[i, :n]) < 0.25 * spread
    # integers in [0, 255] are exact in BF16: then the copy's scores are exact too
    assert worst == 0.0 if (kind, prec) == ("sift", 1) else worst > 0.0


@pytest.mark.parametrize("kind,prec", KINDS + [("sift", 1), ("sift", 2)])
@pytest.mark.parametrize("k,kc", [(100, 600), (1, 50), (700, 700), (500, 3000)])
def test_rerank_topk_equals_oracle(bbc, oracle_lib, kind, prec, k, kc):
    h, idx, q = dev_index(bbc, kind)
    nprobe = min(12, idx.nlist)
    cands = oracle_candidates(oracle_lib, idx, q, nprobe, kc)
    a, cnt = pack(cands, kc)
    nq = len(q)
    gi = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    gd = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    with precision(bbc, h, prec, **({"rerank": 0} if kind == "sift" else {})):
        bbc.bbc_precision_stats(h, reset=True)
        bbc.bbc_rerank_topk(h, cuda(q), nq, cuda(a), cuda(cnt), kc, k, gi, gd)
        sync_ok(bbc, h)
        st = bbc.bbc_precision_stats(h, reset=True)
        gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
        oi = np.empty((nq, k), dtype=np.int64)
        for i, c in enumerate(cands):
            d64 = oracle_lib.rerank(q[i], idx.vectors, c, idx.metric)
            oi[i], _ = oracle_lib.topk_final(d64, c, k)
        check_result(oracle_lib, bbc, h, idx, q, gi, gd, oi, kc)
    assert st["scored"] == int(cnt.sum())
    assert st["final"] == int(np.minimum(cnt, k).sum())
    assert 0 <= st["fp64_scored"] <= st["fp32_rechecked"] <= st["scored"]


@pytest.mark.parametrize("kind,prec,k,nprobe,ratio", [
    ("tiny", 1, 100, 12, 2.0), ("tiny", 2, 300, 24, 3.0), ("embed", 1, 200, 10, 1.5),
    ("embed", 2, 200, 10, 4.0), ("pad", 2, 150, 8, 2.0), ("pad", 1, 1, 3, 1.0),
    ("sift", 1, 500, 16, 1.5), ("sift", 2, 2000, 32, 1.2), ("ragged", 2, 50, 40, 1.0),
    ("wide", 1, 400, 6, 3.0), ("wide", 2, 400, 6, 3.0)])
def test_search_end_to_end(bbc, oracle_lib, kind, prec, k, nprobe, ratio):
    h, idx, q = dev_index(bbc, kind)
    kc = max(k, int(np.ceil(ratio * k - 1e-9)))
    nq = len(q)
    gi = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    gd = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    extra = {"kc_ratio": ratio}
    if kind == "sift":
        extra["rerank"] = 0
    with precision(bbc, h, prec, **extra):
        bbc.bbc_search(h, cuda(q), nq, k, nprobe, gi, gd)
        sync_ok(bbc, h)
        gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
        oi, _ = oracle_lib.search(idx, q, k, nprobe, kc, "sort")
        check_result(oracle_lib, bbc, h, idx, q, gi, gd, oi, kc)


def test_prefilter_leaves_few_candidates_bf16(bbc):
    """With BF16 the FP32 recheck touches a minority of the candidates."""
    h, idx, q = dev_index(bbc, "embed")
    k, nq = 200, len(q)
    gi = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    gd = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    with precision(bbc, h, 1, kc_ratio=4.0):
        bbc.bbc_precision_stats(h, reset=True)
        bbc.bbc_search(h, cuda(q), nq, k, 16, gi, gd)
        sync_ok(bbc, h)
        st = bbc.bbc_precision_stats(h, reset=True)
    assert st["scored"] == nq * 4 * k
    assert st["fp32_rechecked"] < 0.5 * st["scored"]


@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_batch_equals_alone(bbc, prec):
    h, idx, q = dev_index(bbc, "tiny")
    rng = np.random.default_rng(5)
    nq = len(q)
    ks = rng.integers(1, 400, nq).astype(np.int32)
    nps = rng.integers(1, 30, nq).astype(np.int32)
    with precision(bbc, h, prec, kc_ratio=2.0):
        tot = int(ks.sum())
        oi = torch.empty(tot, dtype=torch.int64, device="cuda")
        od = torch.empty(tot, dtype=torch.float32, device="cuda")
        bbc.bbc_search_ex(h, cuda(q), nq, ks, nps, oi, od)
        sync_ok(bbc, h)
        oi, od = oi.cpu().numpy(), od.cpu().numpy()
        off = 0
        for i in range(nq):
            k = int(ks[i])
            ai = torch.empty((1, k), dtype=torch.int64, device="cuda")
            ad = torch.empty((1, k), dtype=torch.float32, device="cuda")
            bbc.bbc_search(h, cuda(q[i:i + 1]), 1, k, int(nps[i]), ai, ad)
            sync_ok(bbc, h)
            assert np.array_equal(oi[off:off + k], ai.cpu().numpy()[0]), f"query {i}"
            assert np.array_equal(od[off:off + k], ad.cpu().numpy()[0]), f"query {i}"
            off += k


def test_graph_replay_with_precision(bbc):
    h, idx, q = dev_index(bbc, "embed")
    nq, k = len(q), 150
    st = torch.cuda.Stream()
    qd = cuda(q)
    outs = []
    with precision(bbc, h, 2, kc_ratio=2.0):
        for graphs in (0, 1, 1):
            bbc.bbc_set_param(h, "graphs", graphs)
            gi = torch.empty((nq, k), dtype=torch.int64, device="cuda")
            gd = torch.empty((nq, k), dtype=torch.float32, device="cuda")
            with torch.cuda.stream(st):
                bbc.bbc_search(h, qd, nq, k, 10, gi, gd, stream=st)
            st.synchronize()
            sync_ok(bbc, h)
            outs.append((gi.cpu().numpy(), gd.cpu().numpy()))
        bbc.bbc_set_param(h, "graphs", 0)
    for a, b in outs[1:]:
        assert np.array_equal(a, outs[0][0]) and np.array_equal(b, outs[0][1])


def test_large_k_precision(bbc, oracle_lib):
    """k above the shared-memory top-k limit: the final top-k runs on global keys."""
    h, idx, q = dev_index(bbc, "medium")
    q = q[:4]
    k, ratio, nprobe = 17000, 1.25, 64
    kc = int(np.ceil(ratio * k - 1e-9))
    nq = len(q)
    gi = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    gd = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    with precision(bbc, h, 2, kc_ratio=ratio, rerank=0):
        bbc.bbc_search(h, cuda(q), nq, k, nprobe, gi, gd)
        sync_ok(bbc, h)
        gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
        oi, _ = oracle_lib.search(idx, q, k, nprobe, kc, "sort")
        check_result(oracle_lib, bbc, h, idx, q, gi, gd, oi, kc)


def test_precision_param_errors(bbc):
    h, idx, q = dev_index(bbc, "tiny")
    with pytest.raises(bbc.BBCError):
        bbc.bbc_set_param(h, "precision", 3)
    bbc.bbc_set_param(h, "precision", 0)
    dd = torch.zeros(4, dtype=torch.float32, device="cuda")
    with pytest.raises(bbc.BBCError):                       # no copy built
        bbc.bbc_rerank_bounds(h, cuda(q[:1]), 1, cuda(np.zeros(4, np.uint32)),
                              cuda(np.array([4], np.int64)), 4, dd, dd)
    assert bbc.bbc_get_param(h, "precision") == 0
