"""Pins of the oracle's residual IVF-PQ keys (Section 2 "Quantization", with
PQ codes of each object's residual o - c_l to its list centroid).

The oracle splits the estimated distance into the query's table, a
per-(query, list) term A_ql and a per-object term V_o, and expresses their sum
in the uint16 table's integer units.  These tests check it against what does
not share that split: the FP64 distance from the query to the object's
reconstruction c_l + y_o, computed here with numpy; the reduction to plain PQ
when every centroid is zero; the rounding and clamping rules on hand values;
brute force when every list is probed and every object re-ranked.
"""

import numpy as np
import pytest

from conftest import small_workload

BIAS = 1 << 30


def _recon(idx, rows):
    """FP64 reconstruction y of the residual for the given list positions."""
    from synth.index import unpack_codes
    un = unpack_codes(idx.codes[rows], idx.pq_m, idx.pq_bits)
    b = idx.codebooks.astype(np.float64)
    return np.concatenate([b[m][un[:, m]] for m in range(idx.pq_m)], axis=1)


def _list_of_positions(idx):
    return np.repeat(np.arange(idx.nlist), np.diff(idx.list_offsets))


@pytest.mark.parametrize("kind", ["rtiny", "rsift", "rsift4", "rembed"])
def test_residual_key_is_distance_to_reconstruction(oracle_lib, kind):
    """(key - 2^30) / inv + sum_m lo_m equals the FP64 estimated distance
    ||q - c_l - y||^2 (L2) or -<q, c_l + y> (IP) within the integer rounding
    (M/2 table entries, base and w each half a unit) plus FP32 error."""
    idx, q = small_workload(kind)
    assert idx.residual
    for qi in range(3):
        t16 = oracle_lib.lut16(q[qi], idx.codebooks, idx.metric)
        inv, lo_sum = oracle_lib.lut16_scale(q[qi], idx.codebooks, idx.metric)
        assert inv > 0
        qq = q[qi].astype(np.float64)
        for l in (0, idx.nlist // 2, idx.nlist - 1):
            a, b = idx.list_offsets[l], idx.list_offsets[l + 1]
            if b == a:
                continue
            rows = np.arange(a, b)
            c = idx.centroids[l].astype(np.float64)
            key = oracle_lib.adc_resid(t16, idx.codes[rows], q[qi], idx.centroids[l], idx.codebooks, inv,
                                       idx.metric).astype(np.float64)
            rec = c[None, :] + _recon(idx, rows)
            if idx.metric == "l2":
                ref = ((rec - qq[None, :]) ** 2).sum(axis=1)
                mag = (qq ** 2).sum() + (rec ** 2).sum(axis=1) + 2 * np.abs(rec) @ np.abs(qq)
            else:
                ref = -(rec @ qq)
                mag = np.abs(rec) @ np.abs(qq)
            est = (key - BIAS) / inv + lo_sum
            tol = (idx.pq_m / 2 + 1.5) / inv + 4e-6 * mag
            assert np.all(np.abs(est - ref) <= tol), (kind, qi, l, np.abs(est - ref).max(), tol.max())


@pytest.mark.parametrize("kind", ["rtiny", "rembed"])
def test_zero_centroids_reduce_to_plain_pq(oracle_lib, kind):
    """With every centroid at the origin the residual is the vector itself:
    A_ql = 0 and V_o = 0, so each key is the plain table sum plus 2^30."""
    import dataclasses
    idx, q = small_workload(kind)
    z = dataclasses.replace(idx, centroids=np.zeros_like(idx.centroids))
    for qi in range(2):
        t16 = oracle_lib.lut16(q[qi], z.codebooks, z.metric)
        inv, _ = oracle_lib.lut16_scale(q[qi], z.codebooks, z.metric)
        rows = np.arange(0, 700)
        plain = oracle_lib.adc(t16, z.codes[rows], z.pq_m, z.pq_bits).astype(np.int64)
        res = oracle_lib.adc_resid(t16, z.codes[rows], q[qi], z.centroids[0], z.codebooks, inv, z.metric)
        assert np.array_equal(res.astype(np.int64), plain + BIAS)


def test_per_list_and_per_object_terms_closed_form(oracle_lib):
    idx, q = small_workload("rsift")
    qq = q[0].astype(np.float64)
    for l in range(0, idx.nlist, 9):
        c = idx.centroids[l].astype(np.float64)
        a_l2 = oracle_lib.resid_a(q[0], idx.centroids[l], "l2")
        assert abs(a_l2 - ((c ** 2).sum() - 2 * c @ qq)) <= 1e-6 * ((c ** 2).sum() + 2 * np.abs(c) @ np.abs(qq))
        a_ip = oracle_lib.resid_a(q[0], idx.centroids[l], "ip")
        assert abs(a_ip + c @ qq) <= 1e-6 * (np.abs(c) @ np.abs(qq))
        a, b = idx.list_offsets[l], min(idx.list_offsets[l + 1], idx.list_offsets[l] + 50)
        rows = np.arange(a, b)
        v = oracle_lib.resid_v(idx.centroids[l], idx.codes[rows], idx.codebooks, "l2").astype(np.float64)
        y = _recon(idx, rows)
        np.testing.assert_allclose(v, 2 * y @ c, rtol=0, atol=1e-6 * 2 * (np.abs(y) @ np.abs(c)).max())
        assert np.all(oracle_lib.resid_v(idx.centroids[l], idx.codes[rows], idx.codebooks, "ip") == 0)


def test_rounding_and_clamps():
    import oracle
    oracle.build()
    w = oracle.resid_w
    assert [w(x, 1.0) for x in (2.5, 3.5, -2.5, -0.5, 0.5, 1.49)] == [2, 4, -2, 0, 0, 1]      # ties to even
    assert w(1e30, 1.0) == 1 << 28 and w(-1e30, 1.0) == -(1 << 28)
    assert w(3.0, 0.0) == 0
    base = oracle.resid_base
    assert base(0.0, 5.0) == BIAS
    assert base(-10.25, 2.0) == BIAS - 20 and base(10.75, 2.0) == BIAS + 22
    assert base(1e30, 1.0) == BIAS + (1 << 29) and base(-1e30, 1.0) == BIAS - (1 << 29)


@pytest.mark.parametrize("kind", ["rtiny", "rembed"])
def test_full_probe_full_candidates_is_exact_knn(oracle_lib, kind):
    """Every list probed and every object a candidate: the exact re-rank makes
    the result the exact kNN whatever the keys are."""
    idx, q = small_workload(kind)
    qs = q[:3]
    oi, od = oracle_lib.search(idx, qs, 20, idx.nlist, idx.n, collector="bucket")
    bi, bd = oracle_lib.bruteforce(qs, idx.vectors, 20, idx.metric)
    np.testing.assert_array_equal(oi, bi)
    np.testing.assert_allclose(od, bd, rtol=1e-12, atol=0)


def test_residual_estimates_are_closer_than_plain(oracle_lib):
    """The residual code spends its codewords on o - c_l, which is smaller
    than o: on clustered data its estimated distances are nearer the exact
    ones than plain PQ's (measured as the mean absolute error over the
    probed objects, both in the same units)."""
    ridx, q = small_workload("rsift")
    pidx, _ = small_workload("sift")
    err = {}
    for name, idx in (("plain", pidx), ("residual", ridx)):
        tot, cnt = 0.0, 0
        for qi in range(4):
            qq = q[qi].astype(np.float64)
            lists, _ = oracle_lib.probe(q[qi], idx.centroids, 4, idx.metric)
            t16 = oracle_lib.lut16(q[qi], idx.codebooks, idx.metric)
            inv, lo_sum = oracle_lib.lut16_scale(q[qi], idx.codebooks, idx.metric)
            for l in lists:
                rows = np.arange(idx.list_offsets[l], idx.list_offsets[l + 1])
                if idx.residual:
                    key = oracle_lib.adc_resid(t16, idx.codes[rows], q[qi], idx.centroids[l], idx.codebooks,
                                               inv, idx.metric).astype(np.float64) - BIAS
                else:
                    key = oracle_lib.adc(t16, idx.codes[rows], idx.pq_m, idx.pq_bits).astype(np.float64)
                est = key / inv + lo_sum
                ex = ((idx.vectors[idx.ids[rows]].astype(np.float64) - qq[None, :]) ** 2).sum(axis=1)
                tot += np.abs(est - ex).sum()
                cnt += len(rows)
        err[name] = tot / cnt
    assert err["residual"] < 0.95 * err["plain"], err
