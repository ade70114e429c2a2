"""Parity at full size, in the launch configuration the benchmark times.

* 1M x 128 SIFT-shaped IVF-PQ (1,024 lists, PQ 32 x 8), 10,000 queries in one
  bbc_search call, k = 10,000, nprobe = 256, K_c = 1.4 k: sampled queries
  (first, last and spread between) are recomputed one by one by the oracle and
  must match bit for bit (integer data: the FP32 re-rank is exact).
* The same data with PQ 64 x 4 bit and the list-grouped tensor-core scan
  (2047-level tables), K_c = 1.5 k, the benchmark's default configuration:
  sampled queries must match the oracle's search on the same table bit for bit.
* 1M x 960 GIST-shaped sign-code index (4,096 lists), 4,096 queries in one
  call, k = 10,000, nprobe = 256, hard bounds: sampled queries must return the
  oracle's exact top-k of their probed lists.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bbc():
    import paper_2604_01960_gb300 as bbc
    bbc.build()
    assert torch.cuda.is_available(), "CUDA device required"
    return bbc


def _build(kind):
    from synth import WORKLOADS, make_workload, build_ivf_pq, build_ivf_sign
    from synth.index import set_build_device
    w = WORKLOADS[kind]
    x, q = make_workload(w)
    set_build_device("cuda")
    try:
        if w.quantizer == "sign":
            idx = build_ivf_sign(x, w.nlist)
        else:
            idx = build_ivf_pq(x, w.nlist, w.pq_m, w.pq_bits, w.metric)
    finally:
        set_build_device("cpu")
    return w, idx, q


def test_sift_1m_full_batch_sampled_parity(bbc, oracle_lib):
    w, idx, q = _build("sift")
    k, nprobe, ratio = w.k, w.nprobe, 1.4
    kc = int(np.ceil(ratio * k - 1e-9))
    h = bbc.bbc_index_create(idx, 0)
    try:
        bbc.bbc_set_param(h, "kc_ratio", ratio)
        bbc.bbc_set_param(h, "workspace_mb", 64 * 1024)
        nq = len(q)
        ids = torch.empty((nq, k), dtype=torch.int64, device="cuda")
        dd = torch.empty((nq, k), dtype=torch.float32, device="cuda")
        bbc.bbc_search(h, torch.from_numpy(q).cuda(), nq, k, nprobe, ids, dd)
        torch.cuda.synchronize()
        bbc.bbc_stream_status(h)
        for i in (0, 1234, 5001, 7777, nq - 1):
            oi, od = oracle_lib.search(idx, q[i:i + 1], k, nprobe, kc, "sort")
            assert np.array_equal(ids[i].cpu().numpy(), oi[0]), f"query {i}: ids"
            assert np.array_equal(dd[i].cpu().numpy().astype(np.float64), od[0]), f"query {i}: distances"
    finally:
        bbc.bbc_index_free(h)


def test_sift4_1m_tensor_core_scan_full_batch_sampled_parity(bbc, oracle_lib):
    w, idx, q = _build("sift4")
    k, nprobe, ratio = w.k, w.nprobe, 1.5
    kc = int(np.ceil(ratio * k - 1e-9))
    h = bbc.bbc_index_create(idx, 0)
    try:
        bbc.bbc_set_param(h, "kc_ratio", ratio)
        bbc.bbc_set_param(h, "workspace_mb", 64 * 1024)
        bbc.bbc_set_param(h, "scan_tc", 1)
        nq = len(q)
        ids = torch.empty((nq, k), dtype=torch.int64, device="cuda")
        dd = torch.empty((nq, k), dtype=torch.float32, device="cuda")
        bbc.bbc_search(h, torch.from_numpy(q).cuda(), nq, k, nprobe, ids, dd)
        torch.cuda.synchronize()
        bbc.bbc_stream_status(h)
        for i in (0, 2222, 6001, nq - 1):
            oi, od = oracle_lib.search(idx, q[i:i + 1], k, nprobe, kc, "sort", lut_levels=2047)
            assert np.array_equal(ids[i].cpu().numpy(), oi[0]), f"query {i}: ids"
            assert np.array_equal(dd[i].cpu().numpy().astype(np.float64), od[0]), f"query {i}: distances"
    finally:
        bbc.bbc_index_free(h)


def test_gist_1m_sign_full_batch_sampled_parity(bbc, oracle_lib):
    w, idx, q = _build("gist")
    k, nprobe = w.k, 256
    h = bbc.bbc_index_create(idx, 0)
    try:
        bbc.bbc_set_param(h, "workspace_mb", 64 * 1024)
        nq = len(q)
        ids = torch.empty((nq, k), dtype=torch.int64, device="cuda")
        dd = torch.empty((nq, k), dtype=torch.float32, device="cuda")
        bbc.bbc_search(h, torch.from_numpy(q).cuda(), nq, k, nprobe, ids, dd)
        torch.cuda.synchronize()
        bbc.bbc_stream_status(h)
        sample = [0, 2049, nq - 1]
        lists = [oracle_lib.probe(q[i], idx.centroids, nprobe, "l2")[0] for i in sample]
        codes, fac = oracle_lib.sign_encode_lists(idx, np.concatenate(lists))
        eps = oracle_lib.rotation_eps(idx.rotation)
        oi, od, _ = oracle_lib.sign_search(idx, q[sample], k, nprobe, codes=codes, fac=fac, eps=eps)
        for j, i in enumerate(sample):
            g = ids[i].cpu().numpy()
            assert set(g.tolist()) == set(oi[j].tolist()), f"query {i}: result set"
            d64 = oracle_lib.rerank(q[i], idx.vectors, g, "l2")
            gd = dd[i].cpu().numpy().astype(np.float64)
            assert np.all(np.abs(gd - d64) <= 1e-5 * d64)
    finally:
        bbc.bbc_index_free(h)
