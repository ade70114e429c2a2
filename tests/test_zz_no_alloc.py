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


def _collect(bbc, fn, h, qd, nq, nprobe, lists, kc):
    ids = torch.full((nq, kc), -1, dtype=torch.int32, device="cuda")
    cnt = torch.full((nq,), -1, dtype=torch.int64, device="cuda")
    st = torch.zeros(nq * bbc.STATE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    fn(h, qd, nq, nprobe, lists, kc, ids, cnt, st)
    torch.cuda.synchronize()
    bbc.bbc_stream_status(h)
    return ids.cpu().numpy().view(np.uint32), cnt.cpu().numpy(), st.cpu().numpy().view(bbc.STATE_DTYPE)


def test_static_scratch_collect_matches_allocating_collect():
    import paper_2604_01960_gb300 as bbc
    bbc.build()
    assert torch.cuda.is_available(), "CUDA device required"
    idx, q = small_workload("sift")
    h = bbc.bbc_index_create(idx, 0)
    try:
        nprobe, kc = 16, 900
        for qs in (q[:12], q[12:24]):                    # two calls in a row, different queries
            nq = len(qs)
            qd = torch.from_numpy(np.ascontiguousarray(qs)).cuda()
            lists = torch.empty((nq, nprobe), dtype=torch.int32, device="cuda")
            bbc.bbc_probe(h, qd, nq, nprobe, lists)
            ref_ids, ref_cnt, ref_st = _collect(bbc, bbc.bbc_collect, h, qd, nq, nprobe, lists, kc)
            got_ids, got_cnt, got_st = _collect(bbc, bbc.bbc_collect_static, h, qd, nq, nprobe, lists, kc)
            assert np.array_equal(got_cnt, ref_cnt)
            for i in range(nq):
                n = int(ref_cnt[i])
                assert np.array_equal(np.sort(got_ids[i, :n]), np.sort(ref_ids[i, :n])), f"query {i}"
            for f in ("d_min", "d_max", "sh", "tau", "below", "scanned"):
                assert np.array_equal(got_st[f], ref_st[f]), f
        # more queries than the static scratch can hold: refused before any launch
        big = 200_000
        qd = torch.zeros((big, idx.d), dtype=torch.float32, device="cuda")
        lists = torch.zeros((big, nprobe), dtype=torch.int32, device="cuda")
        ids = torch.empty((1,), dtype=torch.int32, device="cuda")
        cnt = torch.empty((big,), dtype=torch.int64, device="cuda")
        with pytest.raises(bbc.BBCError) as ei:
            bbc.bbc_collect_static(h, qd, big, nprobe, lists, kc, ids, cnt)
        assert ei.value.code == -1 and "static scratch" in str(ei.value)
    finally:
        bbc.bbc_index_free(h)
