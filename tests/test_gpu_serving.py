"""Serving: continuous batching of single-query requests (different k and
nprobe per request) with admission by candidate-buffer bytes.  Every result
must equal the oracle's result for that request (its own k, nprobe and K_c)
and searching that query alone, whatever batch it ran in."""

import threading

import numpy as np
import pytest

from conftest import check_topk, small_workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bbc():
    import paper_2604_01960_gb300 as bbc
    bbc.build()
    assert torch.cuda.is_available(), "CUDA device required"
    return bbc


def _alone(bbc, h, qv, k, nprobe):
    qd = torch.from_numpy(np.ascontiguousarray(qv[None, :])).cuda()
    oi = torch.empty((1, k), dtype=torch.int64, device="cuda")
    od = torch.empty((1, k), dtype=torch.float32, device="cuda")
    bbc.bbc_search(h, qd, 1, k, nprobe, oi, od)
    torch.cuda.synchronize()
    return oi.cpu().numpy()[0], od.cpu().numpy()[0]


@pytest.mark.parametrize("kind,budget_mb,streams,max_batch", [("sift", 1, 3, 5), ("tiny", 64, 4, 64),
                                                               ("medium", 4, 2, 8)])
def test_serving_results_equal_alone(bbc, oracle_lib, kind, budget_mb, streams, max_batch):
    idx, q = small_workload(kind)
    h = bbc.bbc_index_create(idx, 0)
    try:
        bbc.bbc_set_param(h, "kc_ratio", 1.5)
        rng = np.random.default_rng(5)
        n = 3 * len(q)
        qs = np.concatenate([q] * 3)
        ks = np.exp(rng.uniform(np.log(10), np.log(3000), size=n)).astype(np.int32)
        ps = rng.choice([1, max(1, idx.nlist // 8), idx.nlist // 2, idx.nlist], size=n).astype(np.int32)
        budget = budget_mb << 20
        sv = bbc.bbc_serve_start(h, max_batch=max_batch, streams=streams, cand_bytes_budget=budget)
        tickets = [None] * n

        def submit(lo, hi):
            for i in range(lo, hi):
                tickets[i] = bbc.bbc_serve_submit(sv, qs[i], int(ks[i]), int(ps[i]))

        th = [threading.Thread(target=submit, args=(j * n // 3, (j + 1) * n // 3)) for j in range(3)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        got = [bbc.bbc_serve_poll(sv, tickets[i], int(ks[i]), 60000) for i in range(n)]
        st = bbc.bbc_serve_stats(sv)
        bbc.bbc_serve_stop(sv)
        assert st["submitted"] == n and st["completed"] == n
        assert st["p99_ms"] >= st["p50_ms"] > 0 and st["batches"] >= 1
        cap = np.sort(np.diff(idx.list_offsets))[::-1].cumsum()
        largest = max(8 * int(cap[p - 1]) + 8 * int(np.ceil(1.5 * k)) for k, p in zip(ks, ps))
        assert st["inflight_bytes_peak"] <= max(budget, largest)
        exact = kind in ("sift", "medium")
        for i in range(n):
            k = int(ks[i])
            kc = max(k, int(np.ceil(1.5 * k - 1e-9)))
            oi, od = oracle_lib.search(idx, qs[i:i + 1], k, int(ps[i]), kc, "sort")
            check_topk(oracle_lib, idx, qs[i], got[i][0], got[i][1], oi[0], od[0], exact)
            ai, ad = _alone(bbc, h, qs[i], int(ks[i]), int(ps[i]))
            assert np.array_equal(got[i][0], ai), i
            assert np.array_equal(got[i][1], ad), i
    finally:
        bbc.bbc_index_free(h)


def test_serving_poll_timeout_and_unknown_ticket(bbc):
    idx, q = small_workload("tiny")
    h = bbc.bbc_index_create(idx, 0)
    try:
        sv = bbc.bbc_serve_start(h, max_batch=4, streams=1, cand_bytes_budget=1 << 30)
        t = bbc.bbc_serve_submit(sv, q[0], 50, 8)
        ids, dd = bbc.bbc_serve_poll(sv, t, 50, -1)
        assert (ids >= 0).all()
        with pytest.raises(bbc.BBCError) as ei:
            bbc.bbc_serve_poll(sv, t, 50, 0)                 # already consumed
        assert ei.value.code == -1
        bbc.bbc_serve_stop(sv)
    finally:
        bbc.bbc_index_free(h)
