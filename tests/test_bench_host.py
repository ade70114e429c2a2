"""Host-side logic of the benchmark on the CPU: the tie-aware recall that
decides whether a line clears recall@k >= 0.95, the exact k-th distance it
compares against, and the scaling of a recorded ncu capture to the bench's
launch (reported as unknown once the kernel's source no longer matches)."""

import hashlib
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _bench():
    import bench
    return bench


def _np_dist(x, q, metric):
    x = x.astype(np.float64)
    q = q.astype(np.float64)
    if metric == "ip":
        return -(q @ x.T)
    return ((q[:, None, :] - x[None, :, :]) ** 2).sum(-1)


@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_exact_kth_is_the_sorted_kth_distance(metric):
    rng = np.random.default_rng(11)
    x = rng.integers(0, 256, size=(700, 32)).astype(np.float32)
    q = rng.integers(0, 256, size=(9, 32)).astype(np.float32)
    k = 37
    got = _bench().exact_kth(torch.from_numpy(x), torch.from_numpy(q), k, metric).numpy()
    want = np.sort(_np_dist(x, q, metric), axis=1)[:, k - 1]
    assert np.array_equal(got.astype(np.float64), want)        # integer data: exact in FP32


def test_recall_counts_ties_at_the_kth_distance_and_ignores_padding():
    """Points at equal distance from the query: any k of the tied ones are a
    correct answer (recall 1); ids past the k-th distance and -1 padding do not
    count."""
    d = 16
    x = np.zeros((40, d), dtype=np.float32)
    x[:10, 0] = 1.0           # distance 1 from the origin query: ten-way tie
    x[10:, 0] = 5.0           # distance 25
    q = np.zeros((3, d), dtype=np.float32)
    k = 4
    ids = torch.tensor([[9, 8, 7, 6],          # four of the ten tied nearest: all correct
                        [0, 1, 20, 21],        # two correct, two beyond the k-th distance
                        [0, 1, 2, -1]],        # three correct and one padding slot
                       dtype=torch.int64)
    mean, mn, dk = _bench().recall_at_k(torch.from_numpy(x), torch.from_numpy(q), ids, k)
    assert dk.tolist() == [1.0, 1.0, 1.0]
    assert mn == pytest.approx(0.5)
    assert mean == pytest.approx((1.0 + 0.5 + 0.75) / 3)


@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_recall_matches_a_direct_count(metric):
    rng = np.random.default_rng(12)
    x = rng.integers(0, 256, size=(900, 24)).astype(np.float32)
    q = rng.integers(0, 256, size=(7, 24)).astype(np.float32)
    k = 50
    dist = _np_dist(x, q, metric)
    order = np.argsort(dist, axis=1, kind="stable")
    # a result list that keeps the true first 40 and then takes ranks 100..109
    ids = np.concatenate([order[:, :40], order[:, 100:110]], axis=1)
    kth = np.sort(dist, axis=1)[:, k - 1]
    want = [(dist[i, ids[i]] <= kth[i]).sum() / k for i in range(len(q))]
    mean, mn, _ = _bench().recall_at_k(torch.from_numpy(x), torch.from_numpy(q), torch.from_numpy(ids), k, metric)
    assert mean == pytest.approx(float(np.mean(want)))
    assert mn == pytest.approx(float(np.min(want)))


def _capture_table(root, src_rel, src_bytes, sha):
    os.makedirs(os.path.join(root, "profiles"), exist_ok=True)
    os.makedirs(os.path.dirname(os.path.join(root, src_rel)), exist_ok=True)
    with open(os.path.join(root, src_rel), "wb") as f:
        f.write(src_bytes)
    table = {"captures": [{"stage": "scan", "kernel": "k", "workload": "w", "nprobe": 256, "kc": 15000,
                           "pair": False, "queries": 2000, "dram_bytes": 489286912, "source": src_rel,
                           "source_sha256": sha, "file": "profiles/x.md"}]}
    with open(os.path.join(root, "profiles", "traffic.json"), "w") as f:
        json.dump(table, f)


def test_captured_traffic_scales_by_queries_and_goes_null_on_a_changed_source(tmp_path, monkeypatch):
    bench = _bench()
    src = b"__global__ void k() {}\n"
    _capture_table(str(tmp_path), "csrc/k.cu", src, hashlib.sha256(src).hexdigest())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    t, why = bench.captured_traffic("scan", "w", 256, 15000, 10000, False)
    assert t == pytest.approx(489286912 / 2000 * 10000)
    assert "2000 queries" in why
    # another workload, nprobe, K_c or schedule: no capture
    for args in (("scan", "v", 256, 15000), ("scan", "w", 128, 15000), ("scan", "w", 256, 14000),
                 ("rerank", "w", 256, 15000)):
        assert bench.captured_traffic(*args, 10000, False)[0] is None
    assert bench.captured_traffic("scan", "w", 256, 15000, 10000, True)[0] is None
    # the kernel source changed after the capture: the figure is withdrawn
    with open(os.path.join(str(tmp_path), "csrc/k.cu"), "ab") as f:
        f.write(b"// edited\n")
    t, why = bench.captured_traffic("scan", "w", 256, 15000, 10000, False)
    assert t is None and "source changed" in why


def test_committed_captures_name_existing_sources_and_profiles():
    """Every recorded capture points at a kernel source and a summary that exist
    in the repository, and carries the fields the scaling needs."""
    bench = _bench()
    table = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    assert table["captures"]
    for e in table["captures"]:
        assert os.path.isfile(os.path.join(bench.ROOT, e["source"]))
        assert os.path.isfile(os.path.join(bench.ROOT, e["file"]))
        assert e["queries"] > 0 and e["dram_bytes"] == e["dram_read_bytes"] + e["dram_write_bytes"]
        assert len(e["source_sha256"]) == 64
