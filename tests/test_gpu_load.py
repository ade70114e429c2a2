"""bbc_index_load: an index written to disk by the offline builder, loaded on
the device and searched, gives the same results as the same index created
from host arrays, and the oracle's results (the indexing phase of Section 2
done offline, the querying phase on the loaded structure)."""

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
    torch.cuda.synchronize()
    bbc.bbc_stream_status(h)
    return ids.cpu().numpy(), dd.cpu().numpy()


@pytest.mark.parametrize("kind,k,nprobe", [("sift", 300, 16), ("sift4", 200, 24), ("embed", 150, 10)])
def test_loaded_pq_index_matches_created_and_oracle(bbc, oracle_lib, tmp_path, kind, k, nprobe):
    from synth.index import write_index
    idx, q = small_workload(kind)
    path = str(tmp_path / f"{kind}.bbcidx")
    write_index(path, idx)
    hl = bbc.bbc_index_load(path, 0)
    hc = bbc.bbc_index_create(idx, 0)
    try:
        il, ic = bbc.bbc_index_info(hl), bbc.bbc_index_info(hc)
        for f in ("n", "d", "nlist", "metric", "pq_m", "pq_bits", "max_list_len", "vectors_u8_exact", "quantizer"):
            assert il[f] == ic[f], f
        for h in (hl, hc):
            bbc.bbc_set_param(h, "kc_ratio", 1.5)
        li, ld = _search(bbc, hl, q, k, nprobe)
        ci, cd = _search(bbc, hc, q, k, nprobe)
        assert np.array_equal(li, ci) and np.array_equal(ld, cd)
        kc = int(np.ceil(1.5 * k))
        oi, od = oracle_lib.search(idx, q, k, nprobe, kc, "sort")
        for i in range(len(q)):
            check_topk(oracle_lib, idx, q[i], li[i], ld[i], oi[i], od[i], kind in ("sift", "sift4"))
    finally:
        bbc.bbc_index_free(hl)
        bbc.bbc_index_free(hc)


def test_loaded_sign_index_matches_created_and_oracle(bbc, oracle_lib, tmp_path):
    from synth import build_ivf_sign
    from synth.data import gist_shaped
    from synth.index import write_sign_index
    x, q = gist_shaped(8000, 6, d=128, n_centers=80)
    idx = build_ivf_sign(x, 32, kmeans_iters=4)
    path = str(tmp_path / "sign.bbcidx")
    write_sign_index(path, idx)
    hl = bbc.bbc_index_load(path, 0)
    hc = bbc.bbc_index_create(idx, 0)
    try:
        assert bbc.bbc_index_info(hl)["quantizer"] == 1
        k, nprobe = 120, 8
        li, ld = _search(bbc, hl, q, k, nprobe)
        ci, cd = _search(bbc, hc, q, k, nprobe)
        assert np.array_equal(li, ci) and np.array_equal(ld, cd)
        oi, _, _ = oracle_lib.sign_search(idx, q, k, nprobe)
        for i in range(len(q)):
            assert set(li[i].tolist()) == set(oi[i].tolist()), f"query {i}"
    finally:
        bbc.bbc_index_free(hl)
        bbc.bbc_index_free(hc)


def test_load_rejects_truncated_file(bbc, tmp_path):
    from synth.index import write_index
    idx, _ = small_workload("tiny")
    path = tmp_path / "t.bbcidx"
    write_index(str(path), idx)
    data = path.read_bytes()
    path.write_bytes(data[:len(data) // 2])
    with pytest.raises(bbc.BBCError) as ei:
        bbc.bbc_index_load(str(path), 0)
    assert ei.value.code == -3
