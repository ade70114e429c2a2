"""bbc_collect_static, the allocation-free collect stage, against bbc_collect.

bbc_collect_static serves callers that cannot call cudaMalloc (programs that
budget all device memory themselves, latency-critical threads).  Its scratch
is one static device array shared by every call, so this test makes two calls
in a row on different queries -- the second must not see anything of the
first -- and checks both against the allocating entry point.  Candidate sets
are integer results, so they must match exactly.  The file is named to run
last; it also passes on its own in a fresh process.
"""

import numpy as np
import pytest

from conftest import small_workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _collect(bbc, fn, h, qd, nq, nprobe, lists, kc, with_state=True):
    ids = torch.full((nq, kc), -1, dtype=torch.int32, device="cuda")
    cnt = torch.full((nq,), -1, dtype=torch.int64, device="cuda")
    st = torch.zeros(nq * bbc.STATE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    fn(h, qd, nq, nprobe, lists, kc, ids, cnt, st if with_state else None)
    torch.cuda.synchronize()
    bbc.bbc_stream_status(h)
    return ids.cpu().numpy().view(np.uint32), cnt.cpu().numpy(), st.cpu().numpy().view(bbc.STATE_DTYPE)


def _same_candidates(got, ref, nq, state=True):
    got_ids, got_cnt, got_st = got
    ref_ids, ref_cnt, ref_st = ref
    assert np.array_equal(got_cnt, ref_cnt)
    for i in range(nq):
        n = int(ref_cnt[i])
        assert np.array_equal(np.sort(got_ids[i, :n]), np.sort(ref_ids[i, :n])), f"query {i}"
    if state:
        for f in ("d_min", "d_max", "sh", "tau", "below", "scanned"):
            assert np.array_equal(got_st[f], ref_st[f]), f


def test_static_scratch_collect_matches_allocating_collect():
    import paper_2604_01960_gb300 as bbc
    bbc.build()
    assert torch.cuda.is_available(), "CUDA device required"
    idx, q = small_workload("sift")
    h = bbc.bbc_index_create(idx, 0)
    try:
        # consecutive calls whose scratch layouts differ (query count, probe
        # count, K_c, and the collector state inside or outside the array), so
        # the lookup tables, state and region move inside the static array
        calls = [(q[:12], 16, 900, True), (q[12:24], 16, 900, True), (q[:20], 24, 400, False),
                 (q[3:9], 8, 1300, False), (q[5:21], 32, 700, True)]
        for qs, nprobe, kc, with_state in calls:
            nq = len(qs)
            qd = torch.from_numpy(np.ascontiguousarray(qs)).cuda()
            lists = torch.empty((nq, nprobe), dtype=torch.int32, device="cuda")
            bbc.bbc_probe(h, qd, nq, nprobe, lists)
            ref = _collect(bbc, bbc.bbc_collect, h, qd, nq, nprobe, lists, kc)
            got = _collect(bbc, bbc.bbc_collect_static, h, qd, nq, nprobe, lists, kc, with_state)
            _same_candidates(got, ref, nq, with_state)
        # more queries than the static scratch can hold: refused before any launch
        big = 200_000
        nprobe, kc = 16, 900
        qd = torch.zeros((big, idx.d), dtype=torch.float32, device="cuda")
        lists = torch.zeros((big, nprobe), dtype=torch.int32, device="cuda")
        ids = torch.empty((1,), dtype=torch.int32, device="cuda")
        cnt = torch.empty((big,), dtype=torch.int64, device="cuda")
        with pytest.raises(bbc.BBCError) as ei:
            bbc.bbc_collect_static(h, qd, big, nprobe, lists, kc, ids, cnt)
        assert ei.value.code == -1 and "static scratch" in str(ei.value)
    finally:
        bbc.bbc_index_free(h)


def test_static_scratch_collect_allocates_nothing():
    """On an index that has never searched, bbc_collect_static leaves the
    device's free memory unchanged, while bbc_collect's first call grows that
    index's workspace."""
    import paper_2604_01960_gb300 as bbc
    bbc.build()
    idx, q = small_workload("sift")
    nq, nprobe, kc = len(q), 16, 900
    qd = torch.from_numpy(np.ascontiguousarray(q)).cuda()
    lists = torch.empty((nq, nprobe), dtype=torch.int32, device="cuda")
    ids = torch.full((nq, kc), -1, dtype=torch.int32, device="cuda")
    cnt = torch.full((nq,), -1, dtype=torch.int64, device="cuda")
    warm = bbc.bbc_index_create(idx, 0)                  # loads every kernel of the path once
    try:
        bbc.bbc_probe(warm, qd, nq, nprobe, lists)
        bbc.bbc_collect_static(warm, qd, nq, nprobe, lists, kc, ids, cnt)
        torch.cuda.synchronize()
    finally:
        bbc.bbc_index_free(warm)
    h = bbc.bbc_index_create(idx, 0)
    try:
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        bbc.bbc_collect_static(h, qd, nq, nprobe, lists, kc, ids, cnt)
        torch.cuda.synchronize()
        bbc.bbc_stream_status(h)
        assert torch.cuda.mem_get_info()[0] == free0
        bbc.bbc_collect(h, qd, nq, nprobe, lists, kc, ids, cnt)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] < free0
    finally:
        bbc.bbc_index_free(h)
