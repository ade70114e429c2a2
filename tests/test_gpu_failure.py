"""Failure detection on the device without a GPU fault.

Every append to a query's collector region is bounds-checked by the scan
kernels; an append past the region's capacity is dropped and latches an
overrun bit in the index's status word, which bbc_stream_status reports as
BBC_ERR_CAPACITY after synchronising the stream.  The parameter "region_cap"
lowers the capacity below the number of objects a query scans, so the
overrun happens on ordinary inputs: no access leaves its buffer.  Afterwards
the status word is clear and a search at the automatic capacity returns the
oracle's results again.
"""

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


def _search(bbc, h, q, k, nprobe):
    nq = len(q)
    ids = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    dd = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    bbc.bbc_search(h, torch.from_numpy(q).cuda(), nq, k, nprobe, ids, dd)
    return ids, dd


@pytest.mark.parametrize("split", [1, 4])
def test_region_overrun_reports_capacity(bbc, oracle_lib, split):
    idx, q = small_workload("sift")
    h = bbc.bbc_index_create(idx, 0)
    try:
        k, nprobe, ratio = 200, 16, 1.5
        bbc.bbc_set_param(h, "kc_ratio", ratio)
        bbc.bbc_set_param(h, "split", split)
        # a region far smaller than the objects each query scans (and than K_c)
        bbc.bbc_set_param(h, "region_cap", 64)
        assert bbc.bbc_get_param(h, "region_cap") == 64
        _search(bbc, h, q, k, nprobe)
        torch.cuda.synchronize()
        with pytest.raises(bbc.BBCError) as ei:
            bbc.bbc_stream_status(h)
        assert ei.value.code == -6                         # BBC_ERR_CAPACITY
        bbc.bbc_stream_status(h)                           # read and cleared
        bbc.bbc_set_param(h, "region_cap", 0)
        ids, dd = _search(bbc, h, q, k, nprobe)
        torch.cuda.synchronize()
        bbc.bbc_stream_status(h)
        kc = int(np.ceil(ratio * k))
        oi, od = oracle_lib.search(idx, q, k, nprobe, kc, "sort")
        gi, gd = ids.cpu().numpy(), dd.cpu().numpy()
        for i in range(len(q)):
            check_topk(oracle_lib, idx, q[i], gi[i], gd[i], oi[i], od[i], True)
    finally:
        bbc.bbc_index_free(h)


def test_region_cap_at_scanned_size_is_clean(bbc):
    """A capacity equal to the largest S_q of the batch drops nothing."""
    idx, q = small_workload("tiny")
    h = bbc.bbc_index_create(idx, 0)
    try:
        k, nprobe = 100, 8
        lists = torch.empty((len(q), nprobe), dtype=torch.int32, device="cuda")
        bbc.bbc_probe(h, torch.from_numpy(q).cuda(), len(q), nprobe, lists)
        lens = np.diff(idx.list_offsets)
        sq = lens[lists.cpu().numpy()].sum(1).max()
        ref_i, ref_d = _search(bbc, h, q, k, nprobe)
        bbc.bbc_set_param(h, "region_cap", int(sq))
        gi, gd = _search(bbc, h, q, k, nprobe)
        torch.cuda.synchronize()
        bbc.bbc_stream_status(h)
        assert torch.equal(gi, ref_i) and torch.equal(gd, ref_d)
    finally:
        bbc.bbc_index_free(h)


def test_sign_region_overrun_reports_capacity(bbc):
    from synth import build_ivf_sign
    from synth.data import gist_shaped
    x, q = gist_shaped(6000, 4, d=64, n_centers=40)
    idx = build_ivf_sign(x, 16, kmeans_iters=3)
    h = bbc.bbc_index_create(idx, 0)
    try:
        bbc.bbc_set_param(h, "region_cap", 32)
        _search(bbc, h, q, 50, 4)
        torch.cuda.synchronize()
        with pytest.raises(bbc.BBCError) as ei:
            bbc.bbc_stream_status(h)
        assert ei.value.code == -6
        bbc.bbc_set_param(h, "region_cap", 0)
        _search(bbc, h, q, 50, 4)
        torch.cuda.synchronize()
        bbc.bbc_stream_status(h)
    finally:
        bbc.bbc_index_free(h)


def test_region_cap_argument_checks(bbc):
    idx, q = small_workload("tiny")
    h = bbc.bbc_index_create(idx, 0)
    try:
        for bad in (-1, 2.5):
            with pytest.raises(bbc.BBCError):
                bbc.bbc_set_param(h, "region_cap", bad)
    finally:
        bbc.bbc_index_free(h)
