#!/usr/bin/env python3
"""Benchmark: QPS at recall@k >= 0.95 of the large-k IVF-PQ search path.

Workload (default): 1,000,000 SIFT-shaped vectors (d = 128, integer components
in [0, 255]), 1,024 IVF lists, PQ 64 x 4 bit (the 4-bit variant of the
configuration), 10,000 queries, k = 10,000, nprobe = 256, K_c = 1.5 k
candidates re-ranked, the list-grouped scan on the tensor cores with
2047-level tables (recall 0.958; K_c = 1.4 k gives 0.947).  --workload sift
runs PQ 32 x 8 bit with the one-query scan (K_c = 1.4 k, recall 0.959).  A
step is one bbc_search over the whole 10,000-query batch (probe, LUT, scan +
bucket-based result buffer, selection, re-rank, top-k) with queries and index
resident in HBM; L2 is flushed between timed steps.  Recall@k is measured in the same run against
exact kNN over the whole data set (tie-aware: a returned id counts when its
exact distance is <= the k-th exact distance).

Printed: one JSON line (rank 0).  --impl reference times the CPU oracle on the
same workload instead (bounded query sample per step).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "QPS at recall@k>=0.95 (k=10k, 1Mx128 IVF-PQ)"
METRICS = {"sift": METRIC, "sift4": "QPS at recall@k>=0.95 (k=10k, 1Mx128 IVF-PQ 64x4)",
           "sift4m32": "QPS at recall@k>=0.95 (k=10k, 1Mx128 IVF-PQ 32x4)",
           "sift_iid": "QPS at recall@k>=0.95 (k=10k, 1Mx128 IVF-PQ, i.i.d. mixture)",
           "gist": "QPS at recall@k>=0.95 (k=10k, 1Mx960 IVF + 1-bit sign codes, bounded re-rank)",
           "embed": "QPS at recall@k>=0.95 (k=50k, 10Mx768 IVF-PQ, inner product)",
           "tiny": "QPS at recall@k>=0.95 (k=1k, 100kx128 IVF-PQ)"}
UNIT = "queries/s"
SMS = 152
LOOKUPS_PER_SM_CLK = 32          # one 4-byte shared-memory word per lane per clock


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference", "plain"],
                   help="gb300: the batched path; reference: the CPU oracle; plain: the FP32 single-query GPU "
                        "form (one bbc_search per query, FP32 rows)")
    p.add_argument("--workload", default="sift4")
    p.add_argument("--n", type=int, default=None, help="override data size (testing only)")
    p.add_argument("--nq", type=int, default=None)
    p.add_argument("--k", type=int, default=None)
    p.add_argument("--nprobe", default=None, help="lists probed; a comma list prints one line per value")
    p.add_argument("--kc-ratio", default=None,
                   help="K_c / k (default: the smallest tenth that reaches recall 0.95 on the workload); "
                        "a comma list prints one line per value")
    p.add_argument("--buckets", default="64", help="bucket count m; a comma list prints one line per value")
    p.add_argument("--collector", default="0",
                   help="top-K_c collector: 0 the result buffer, 1 lazy linear buffer, 2 binary heap; a comma list "
                        "prints one line per value")
    p.add_argument("--early-rerank", default="0",
                   help="Algorithm 4's early re-rank: 1 on, 0 off; a comma list prints one line per value")
    p.add_argument("--residual", action="store_true",
                   help="residual IVF-PQ: the PQ codes quantise each vector's residual to its list centroid")
    p.add_argument("--scan-tc", default=None,
                   help="1 = list-grouped scan on the tensor cores (4-bit codes, 2047-level tables; the default "
                        "for 4-bit workloads); a comma list prints one line per value")
    p.add_argument("--pair", default="0",
                   help="scan schedule: 1 two queries per CTA (pair form), 0 one; a comma list prints one line per value")
    p.add_argument("--cpu-queries", type=int, default=200, help="oracle sample for cpu_baseline")
    p.add_argument("--cpu-mt-queries", type=int, default=None,
                   help="oracle sample for the all-cores baseline (default: 64 per host core)")
    p.add_argument("--plain-queries", type=int, default=1000, help="--impl plain: queries per step")
    p.add_argument("--mixed-k", default=None,
                   help="mixed batch: per-query k drawn uniformly (seed 7) from this comma list; the step is one "
                        "bbc_search_ex call")
    p.add_argument("--mixed-nprobe", default=None, help="mixed batch: per-query nprobe drawn from this comma list")
    p.add_argument("--ref-queries", type=int, default=24, help="oracle queries per reference step")
    p.add_argument("--e2e-steps", type=int, default=10)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--mode", default="batch", choices=["batch", "serve"],
                   help="batch: the headline batched search; serve: continuous-batching server")
    p.add_argument("--requests", type=int, default=100_000, help="serve mode: requests per rate")
    p.add_argument("--rates", default="20000,50000,100000", help="serve mode: Poisson arrival rates (req/s)")
    p.add_argument("--serve-nprobe", default="32,128,512", help="serve mode: nprobe drawn uniformly from this list")
    p.add_argument("--precision", default=None,
                   help="re-rank precision: 0 FP32 rows (or the exact u8 copy), 1 BF16 prefilter, 2 FP8-E4M3 "
                        "prefilter; a comma list prints one line per value (default: 0, or 2 for float data)")
    p.add_argument("--bound-scale", default="1",
                   help="sign-code indexes: factor on the worst-case bound terms (1 = hard bounds); a comma list "
                        "prints one line per value")
    p.add_argument("--estimator", default="0",
                   help="sign-code indexes: 0 hard bounds, 1 the RaBitQ estimator's probabilistic bounds; a comma "
                        "list prints one line per value")
    p.add_argument("--epsilon0", type=float, default=1.9, help="epsilon_0 of the estimator bounds")
    p.add_argument("--recall-queries", type=int, default=None,
                   help="queries whose recall is measured against exact kNN (default: all, at most 1,000)")
    a = p.parse_args()
    if a.kc_ratio is None:
        a.kc_ratio = DEFAULT_KC.get(a.workload, "1.5")
    if a.scan_tc is None:
        a.scan_tc = "1" if a.workload in ("sift4", "sift4m32") and not a.residual else "0"
    return a


# K_c / k per workload: the smallest tenth whose recall@k reaches 0.95
DEFAULT_KC = {"sift": "1.4", "sift4": "1.5"}


def pq_desc(idx) -> str:
    """The quantizer of an index as the bench line's config names it."""
    if hasattr(idx, "rotation"):
        return "sign 1-bit"
    return f"{idx.pq_m}x{idx.pq_bits}" + (" residual" if getattr(idx, "residual", False) else "")


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if _cuda() else "gloo")
    return ws, rank, local


def _cuda():
    import torch
    return torch.cuda.is_available()


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v: float) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if _cuda() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_rows(n_total: int, rank: int, ws: int):
    """Contiguous shard [lo, hi) of n_total rows for rank of ws (the last may be shorter)."""
    per = (n_total + ws - 1) // ws
    lo = min(n_total, rank * per)
    return lo, min(n_total, lo + per)


def make_inputs(args, device, rank: int = 0, ws: int = 1):
    """Data, index and this rank's queries: with ws ranks the batch is a disjoint shard of a
    ws x nq query set (weak scaling: nq queries per rank, no data-path collective)."""
    from synth import WORKLOADS, make_workload, build_ivf_pq
    from synth.index import set_build_device
    w = WORKLOADS[args.workload]
    n = args.n or w.n
    nq = args.nq or w.nq
    k = args.k or w.k
    nprobe = int(str(args.nprobe).split(",")[0]) if args.nprobe else w.nprobe
    x, q = make_workload(w, n=n, nq=nq * ws)
    lo, hi = shard_rows(len(q), rank, ws)
    q = np.ascontiguousarray(q[lo:hi])
    set_build_device(device)
    t0 = time.time()
    nlist = w.nlist if n >= 100 * w.nlist else max(8, n // 200)
    if w.quantizer == "sign":
        from synth import build_ivf_sign
        idx = build_ivf_sign(x, nlist)
    else:
        idx = build_ivf_pq(x, nlist, w.pq_m, w.pq_bits, w.metric, residual=bool(getattr(args, "residual", False)))
    return w, idx, q, k, nprobe, time.time() - t0


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# recall
# ---------------------------------------------------------------------------
def _dist_block(x_t, xn, qs, metric):
    if metric == "ip":
        return -(qs @ x_t.T)
    return xn[None, :] + (qs * qs).sum(1)[:, None] - 2.0 * (qs @ x_t.T)


def exact_kth(x_t, q_t, k, metric="l2"):
    """k-th smallest exact distance per query (torch on the GPU, FP32).

    For integer components in [0, 255] and d = 128 every partial sum of the
    FP32 evaluation is an integer below 2^24, so these distances are exact."""
    import torch
    xn = (x_t * x_t).sum(1)
    chunk = max(1, min(500, int(4e9 // (4 * x_t.shape[0]))))
    out = []
    for s in range(0, q_t.shape[0], chunk):
        out.append(torch.kthvalue(_dist_block(x_t, xn, q_t[s:s + chunk], metric), k, dim=1).values)
    return torch.cat(out)


def recall_at_k(x_t, q_t, ids, k, metric="l2"):
    """Mean and minimum recall@k, tie-aware: a returned id counts when its exact
    distance is <= the k-th exact distance."""
    import torch
    dk = exact_kth(x_t, q_t, k, metric)
    chunk = max(1, min(500, int(2e9 // (4 * k * x_t.shape[1]))))
    rec = []
    for s in range(0, q_t.shape[0], chunk):
        i = ids[s:s + chunk]
        valid = i >= 0
        v = x_t[i.clamp(min=0)]
        qs = q_t[s:s + chunk, None, :]
        d = -(v * qs).sum(-1) if metric == "ip" else ((v - qs) ** 2).sum(-1)
        ok = (d <= dk[s:s + chunk, None]) & valid
        rec.append(torch.clamp(ok.sum(1), max=k).double() / k)
    r = torch.cat(rec)
    return float(r.mean()), float(r.min()), dk


# ---------------------------------------------------------------------------
def run_reference(args, ws, rank):
    """The oracle (single-threaded C on the host) as the reference arm."""
    import oracle
    if rank != 0:
        return
    oracle.build()
    device = "cuda" if _cuda() else "cpu"
    w, idx, q, k, nprobe, _ = make_inputs(args, device)
    kc = max(k, int(math.ceil(float(str(args.kc_ratio).split(",")[0]) * k - 1e-9)))
    nqs = min(args.ref_queries, len(q))
    # the table the measured arm uses (2047 levels with the tensor-core scan)
    levels = 2047 if str(args.scan_tc).split(",")[0] == "1" else 65535
    for s in range(args.warmup):
        oracle.search(idx, q[:1], k, nprobe, kc, "sort", lut_levels=levels)
    t = []
    for s in range(args.steps):
        sel = q[(s * nqs) % len(q):][:nqs]
        t0 = time.perf_counter()
        oracle.search(idx, sel, k, nprobe, kc, "sort", lut_levels=levels)
        t.append(time.perf_counter() - t0)
    qps = nqs * len(t) / sum(t)
    sample = f"{nqs} queries per step of the {len(q)}-query batch, full {idx.n}-vector index"
    print(json.dumps({
        "impl": "reference", "metric": METRICS.get(args.workload, METRIC), "value": qps, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sum(t) / len(t), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n": idx.n, "d": idx.d, "nlist": idx.nlist, "pq": pq_desc(idx),
                   "nq_per_step": nqs, "k": k, "nprobe": nprobe, "kc": kc, "lut_levels": levels},
        "cpu_baseline": {"value": qps, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": qps, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_serve(args, ws, rank, local):
    """Serving workload: index of the 1M x 128 IVF-PQ configuration, Poisson
    arrivals at swept rates, k log-uniform in [100, 50,000], nprobe from
    {32, 128, 512}; p50 / p99 latency and completed requests per second."""
    import threading
    import torch
    import paper_2604_01960_gb300 as bbc
    from synth.requests import request_stream
    torch.cuda.set_device(local)
    bbc.build()
    w, idx, q, _, _, t_build = make_inputs(args, f"cuda:{local}")
    index = bbc.Index(idx, device=local)
    index.set(kc_ratio=float(str(args.kc_ratio).split(",")[0]), workspace_mb=64 * 1024)
    h = index.handle
    rates = [float(r) for r in args.rates.split(",")]
    pset = tuple(int(v) for v in args.serve_nprobe.split(","))
    nrec = min(args.requests, args.recall_queries or 2000)
    every = max(1, args.requests // nrec)
    lines = []
    for rate in rates:
        arr, ks, ps, qi = request_stream(args.requests, rate, len(q), seed=6, nprobes=pset)
        sv = bbc.bbc_serve_start(h, max_batch=1024, streams=4, cand_bytes_budget=16 << 30)
        # warm-up: one request of each nprobe, largest k
        for p_ in pset:
            t = bbc.bbc_serve_submit(sv, q[0], 50000, p_)
            bbc.bbc_serve_poll(sv, t, 50000, -1)
        bbc.bbc_serve_stop(sv)
        sv = bbc.bbc_serve_start(h, max_batch=1024, streams=4, cand_bytes_budget=16 << 30)
        tickets = [0] * len(arr)
        results = {}
        done = threading.Event()

        def poller():
            for i in range(len(arr)):
                while tickets[i] == 0:
                    time.sleep(0.0001)
                r = bbc.bbc_serve_poll(sv, tickets[i], int(ks[i]), -1)
                if i % every == 0:
                    results[i] = r
            done.set()

        th = threading.Thread(target=poller, daemon=True)
        th.start()
        t0 = time.perf_counter()
        for i in range(len(arr)):
            while time.perf_counter() - t0 < arr[i]:
                pass
            tickets[i] = bbc.bbc_serve_submit(sv, q[qi[i]], int(ks[i]), int(ps[i]))
        done.wait()
        wall = time.perf_counter() - t0
        st = bbc.bbc_serve_stats(sv)
        bbc.bbc_serve_stop(sv)
        # recall on every (requests / recall sample)-th request (tie-aware, exact kNN on the GPU)
        xt = torch.from_numpy(idx.vectors).cuda()
        recs = []
        for i, (ri, rd) in results.items():
            qv = torch.from_numpy(q[qi[i]][None, :]).cuda()
            dk = exact_kth(xt, qv, int(ks[i]))[0]
            v = xt[torch.from_numpy(ri).cuda().clamp(min=0)]
            d = ((v - qv) ** 2).sum(-1)
            ok = (d <= dk) & (torch.from_numpy(ri).cuda() >= 0)
            recs.append((int(ps[i]), min(int(ks[i]), int(ok.sum())) / int(ks[i])))
        by_p = {p_: float(np.mean([r for pp, r in recs if pp == p_])) for p_ in pset
                if any(pp == p_ for pp, _ in recs)}
        # requests served at recall@k >= 0.95: those whose nprobe reaches it on the sample
        ok_p = [p_ for p_, r in by_p.items() if r >= 0.95]
        frac_ok = float(np.mean(np.isin(ps, ok_p))) if ok_p else 0.0
        lines.append({"offered_rps": rate, "completed_rps": len(arr) / wall, "p50_ms": st["p50_ms"],
                      "p99_ms": st["p99_ms"], "mean_batch": st["mean_batch"], "batches": st["batches"],
                      "inflight_bytes_peak": st["inflight_bytes_peak"], "recall_by_nprobe": by_p,
                      "recall_sample": len(recs), "nprobe_at_recall_0.95": ok_p,
                      "completed_rps_at_recall_0.95": frac_ok * len(arr) / wall, "wall_s": wall})
    if rank == 0:
        best = max(lines, key=lambda r: r["completed_rps"])
        print(json.dumps({
            "metric": "serving: completed requests/s and p50/p99 latency (1Mx128 IVF-PQ, k in [100,50000])",
            "value": best["completed_rps"], "unit": "requests/s", "n_gpus": ws, "higher_is_better": True,
            "p50_ms": best["p50_ms"], "p99_ms": best["p99_ms"], "data": "synthetic", "dtype": "u16/u32 ADC, f32 re-rank",
            "config": {"workload": "serve-" + w.name, "requests_per_rate": args.requests, "k": "log-uniform [100, 50000]",
                       "nprobe": f"uniform {list(pset)}", "kc_ratio": float(str(args.kc_ratio).split(",")[0]), "streams": 4,
                       "max_batch": 1024, "cand_bytes_budget": 16 << 30, "index_build_s": round(t_build, 1)},
            "rates": lines}), flush=True)
    index.close()


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.mode == "serve":
        run_serve(args, ws, rank, local)
        return
    if args.impl == "plain":
        run_plain(args, ws, rank, local)
        return
    import torch
    import paper_2604_01960_gb300 as bbc
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    bbc.build()
    w, idx, q, k, nprobe, t_build = make_inputs(args, f"cuda:{local}", rank, ws)
    torch.cuda.empty_cache()
    index = bbc.Index(idx, device=local)
    index.set(workspace_mb=64 * 1024)
    float_data = not index.info["vectors_u8_exact"]
    precs = [int(v) for v in args.precision.split(",")] if args.precision else [2 if float_data else 0]
    if index.info["quantizer"] == 1 and not args.precision:
        precs = [0]                                      # sign codes: FP32 rounds unless a copy is asked for
    xt = torch.from_numpy(idx.vectors).to(dev)
    nprobes = [int(v) for v in args.nprobe.split(",")] if args.nprobe else [nprobe]
    ratios = [float(v) for v in str(args.kc_ratio).split(",")]
    scales = [float(v) for v in str(args.bound_scale).split(",")] if index.info["quantizer"] == 1 else [None]
    ests = [int(v) for v in str(args.estimator).split(",")] if index.info["quantizer"] == 1 else [None]
    if ests[0] is not None:
        index.set(epsilon0=args.epsilon0)
    buckets = [int(v) for v in str(args.buckets).split(",")]
    pairs = [int(v) for v in str(args.pair).split(",")]
    collectors = [int(v) for v in str(args.collector).split(",")]
    earlys = [int(v) for v in str(args.early_rerank).split(",")]
    tcs = [int(v) for v in str(args.scan_tc).split(",")]
    if args.mixed_k:
        index.set(kc_ratio=ratios[0], buckets=buckets[0], pair=pairs[0])
        if tcs[0]:
            index.set(scan_tc=1)
        if scales[0] is not None:
            index.set(bound_scale=scales[0], estimator=ests[0])
        measure_mixed(args, ws, rank, local, bbc, index, w, idx, q, t_build, xt, precs[0], ratios[0])
        index.close()
        return
    for prec in precs:
        for npb in nprobes:
            for ratio in ratios:
                for m in buckets:
                    for scale in scales:
                        for est in ests:
                            for pair in pairs:
                                for coll in collectors:
                                    for early in earlys:
                                        for tc in tcs:
                                            index.set(kc_ratio=ratio, buckets=m, pair=pair, collector=coll)
                                            if early != index.get("early_rerank"):
                                                index.set(early_rerank=early)
                                            if scale is not None:
                                                index.set(bound_scale=scale, estimator=est)
                                            index.set(scan_tc=tc)
                                            if not tc:
                                                index.set(lut_levels=65535)
                                            measure(args, ws, rank, local, bbc, index, w, idx, q, k, npb, t_build,
                                                    xt, prec, ratio, m)
    index.close()


def run_plain(args, ws, rank, local):
    """The plain FP32 single-query GPU form: one bbc_search per query (probe,
    table, scan, selection, re-rank from the FP32 rows, top-k), the queries one
    after another on one stream: no batching across queries, no CUDA graphs, no
    u8 or low-precision copy.  A step is --plain-queries such searches."""
    import torch
    import paper_2604_01960_gb300 as bbc
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    bbc.build()
    w, idx, q, k, nprobe, t_build = make_inputs(args, f"cuda:{local}", rank, ws)
    torch.cuda.empty_cache()
    index = bbc.Index(idx, device=local)
    ratio = float(str(args.kc_ratio).split(",")[0])
    index.set(workspace_mb=64 * 1024, kc_ratio=ratio, graphs=0, pair=0, split=0, buckets=int(str(args.buckets).split(",")[0]))
    if index.info["vectors_u8_exact"]:
        index.set(rerank=0)
    if index.get("precision"):
        index.set(precision=0)
    h = index.handle
    nsel = min(args.plain_queries, len(q))
    qd = torch.from_numpy(np.ascontiguousarray(q[:nsel])).to(dev)
    ids = torch.empty((nsel, k), dtype=torch.int64, device=dev)
    dists = torch.empty((nsel, k), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    L = bbc.lib()
    qp, ip, dp, sp, d = qd.data_ptr(), ids.data_ptr(), dists.data_ptr(), stream.cuda_stream, idx.d

    def step():
        for i in range(nsel):
            rc = L.bbc_search(h, qp + 4 * d * i, 1, k, nprobe, ip + 8 * k * i, dp + 4 * k * i, sp)
            if rc:
                raise bbc.BBCError(rc, L.bbc_last_error().decode())

    step()
    torch.cuda.synchronize()
    bbc.bbc_stream_status(h)
    xt = torch.from_numpy(idx.vectors).to(dev)
    nrec = min(nsel, args.recall_queries or 1000)
    rec_mean, rec_min, _ = recall_at_k(xt, qd[:nrec], ids[:nrec], k, idx.metric)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    barrier(ws)
    evs = []
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    barrier(ws)
    clocks = sampler.stop()
    t = max_over_ranks(ws, sum(a.elapsed_time(b) for a, b in evs) / 1e3)
    if rank == 0:
        print(json.dumps({
            "impl": "plain", "metric": METRICS.get(args.workload, METRIC), "value": ws * nsel * args.steps / t,
            "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u16/u32 ADC, f32 re-rank from the FP32 rows", "data": "synthetic",
            "config": {"workload": w.name, "n": idx.n, "d": idx.d, "nlist": idx.nlist,
                       "pq": pq_desc(idx),
                       "queries_per_step": nsel, "k": k, "nprobe": nprobe, "kc_ratio": ratio,
                       "form": "one bbc_search per query, FP32 rows, no graphs",
                       "recall_at_k": rec_mean, "recall_at_k_min": rec_min, "recall_queries": nrec,
                       "l2_flush_between_steps": True, "index_build_s": round(t_build, 1)},
            "clocks": clocks}), flush=True)
    index.close()


def measure_mixed(args, ws, rank, local, bbc, index, w, idx, q, t_build, xt, prec, ratio):
    """One bbc_search_ex call over the whole batch with per-query k and nprobe
    drawn uniformly (seed 7) from --mixed-k and --mixed-nprobe."""
    import torch
    dev = torch.device("cuda", local)
    if index.get("precision") != prec:
        index.set(precision=prec)
    rng = np.random.default_rng(7)
    kset = [int(v) for v in args.mixed_k.split(",")]
    pset = [int(v) for v in (args.mixed_nprobe or str(w.nprobe)).split(",")]
    nq = len(q)
    ks = rng.choice(np.asarray(kset, dtype=np.int32), nq)
    ps = rng.choice(np.asarray(pset, dtype=np.int32), nq)
    off = np.concatenate([[0], np.cumsum(ks.astype(np.int64))])
    tot = int(off[-1])
    h = index.handle
    qd = torch.from_numpy(q).to(dev)
    ids = torch.empty(tot, dtype=torch.int64, device=dev)
    dists = torch.empty(tot, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    is_sign = hasattr(idx, "rotation")

    def step(qsrc=None):
        bbc.bbc_search_ex(h, qd if qsrc is None else qsrc, nq, ks, ps, ids, dists, stream)

    bbc.bbc_bounded_stats(h, reset=True)
    step()
    torch.cuda.synchronize()
    bbc.bbc_stream_status(h)
    bstats = bbc.bbc_bounded_stats(h, reset=True) if is_sign else None
    # recall per k value, on up to --recall-queries queries of each
    nrec_each = args.recall_queries or 250
    rec_by_k, rec_by_p, rec_all = {}, {}, []
    for kv in kset:
        sel = np.nonzero(ks == kv)[0][:nrec_each]
        if len(sel) == 0:
            continue
        rows = torch.stack([ids[off[i]:off[i] + kv] for i in sel])
        dk = exact_kth(xt, qd[sel], kv, idx.metric)
        v = xt[rows.clamp(min=0)]
        qs = qd[sel][:, None, :]
        dd = -(v * qs).sum(-1) if idx.metric == "ip" else ((v - qs) ** 2).sum(-1)
        r = (torch.clamp(((dd <= dk[:, None]) & (rows >= 0)).sum(1), max=kv).double() / kv).cpu().numpy()
        rec_by_k[kv] = float(r.mean())
        for i, ri in zip(sel, r):
            rec_all.append(ri)
            rec_by_p.setdefault(int(ps[i]), []).append(ri)
        del v, dd
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    bbc.bbc_set_param(h, "profile", 1)
    bbc.bbc_profile_read(h, reset=True)
    sampler = ClockSampler(local)
    sampler.start()
    barrier(ws)
    torch.cuda.synchronize()
    evs = []
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    barrier(ws)
    clocks = sampler.stop()
    stage_ms, launches = bbc.bbc_profile_read(h, reset=True)
    bbc.bbc_set_param(h, "profile", 0)
    t_dev = max_over_ranks(ws, sum(a.elapsed_time(b) for a, b in evs) / 1e3)
    # end to end: pinned host queries copied in, results copied out, every step
    hq = torch.from_numpy(q).pin_memory()
    hi = torch.empty(tot, dtype=torch.int64).pin_memory()
    hd = torch.empty(tot, dtype=torch.float32).pin_memory()
    qbuf = torch.empty_like(qd)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        qbuf.copy_(hq, non_blocking=True)
        step(qbuf)
        hi.copy_(ids, non_blocking=True)
        hd.copy_(dists, non_blocking=True)
        torch.cuda.synchronize()
    t_e2e = max_over_ranks(ws, time.perf_counter() - t0)
    cpu, cpu_mt = None, None
    if rank == 0 and not args.no_cpu_baseline:
        cpu, cpu_mt = cpu_baselines(args, idx, q, ks, ps, kc_ratio=ratio,
                                    scale=index.get("bound_scale") if is_sign else None,
                                    estimator=int(index.get("estimator")) if is_sign else 0,
                                    eps0=index.get("epsilon0") if is_sign else 1.9,
                                    lut_levels=65535 if is_sign else int(index.get("lut_levels")))
    if rank == 0:
        per = {s_: stage_ms[s_] / args.steps for s_ in stage_ms}
        out = {
            "metric": METRICS.get(args.workload, METRIC) + ", mixed k and nprobe",
            "value": ws * nq * args.steps / t_dev, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": ("1-bit codes x 4-bit query planes (AND+POPC), f32 bounds, f32 re-rank (f64 at ties)" if is_sign
                      else "u16/u32 ADC, f32 re-rank"), "data": "synthetic",
            "config": {"workload": w.name, "n": idx.n, "d": idx.d, "nlist": idx.nlist, "nq": nq,
                       "k": f"uniform over {kset} (seed 7)", "nprobe": f"uniform over {pset} (seed 7)",
                       "one_call": "bbc_search_ex", "kc_ratio": None if is_sign else ratio,
                       "recall_at_k": float(np.mean(rec_all)), "recall_by_k": rec_by_k,
                       "recall_by_nprobe": {p_: float(np.mean(v)) for p_, v in sorted(rec_by_p.items())},
                       "recall_queries_per_k": nrec_each, "recall_tie_aware": True,
                       "l2_flush_between_steps": True, "index_build_s": round(t_build, 1)},
            "stage_ms_per_step": per,
            "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_mt,
            "e2e": {"value": ws * nq * args.e2e_steps / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(q.nbytes),
                    "d2h_bytes_per_step": int(tot * 12)},
            "gpu_launches": int(launches), "clocks": clocks}
        if is_sign:
            out["bounded"] = {"per_step": bstats, "in_S_per_query": bstats["in_S"] / nq,
                              "exact_per_query": bstats["exact"] / nq, "scanned_per_query": bstats["scanned"] / nq,
                              "bounds": "RaBitQ estimator, probabilistic" if index.get("estimator") else "hard",
                              "epsilon0": index.get("epsilon0") if index.get("estimator") else None}
        print(json.dumps(out), flush=True)
    del ids, dists, flush, qd


def measure(args, ws, rank, local, bbc, index, w, idx, q, k, nprobe, t_build, xt, prec, ratio, m):
    """Time one configuration and print its JSON line (rank 0)."""
    import torch
    dev = torch.device("cuda", local)
    if index.get("precision") != prec:
        index.set(precision=prec)
    kc = max(k, int(math.ceil(ratio * k - 1e-9)))
    nq = len(q)
    h = index.handle
    qd = torch.from_numpy(q).to(dev)
    ids = torch.empty((nq, k), dtype=torch.int64, device=dev)
    dists = torch.empty((nq, k), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        bbc.bbc_search(h, qd, nq, k, nprobe, ids, dists, stream)

    # correctness of the operating point: recall against exact kNN
    is_sign = hasattr(idx, "rotation")
    bbc.bbc_precision_stats(h, reset=True)
    bbc.bbc_bounded_stats(h, reset=True)
    bbc.bbc_early_stats(h, reset=True)
    step()
    torch.cuda.synchronize()
    bbc.bbc_stream_status(h)
    pstats = bbc.bbc_precision_stats(h, reset=True) if prec else None
    estats = bbc.bbc_early_stats(h, reset=True) if index.get("early_rerank") else None
    bstats = bbc.bbc_bounded_stats(h, reset=True) if is_sign else None
    nrec = min(nq, args.recall_queries or 1000)
    rec_mean, rec_min, dk = recall_at_k(xt, qd[:nrec], ids[:nrec], k, idx.metric)
    gt_check, err = None, None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        if idx.n * idx.d <= (1 << 28):
            bi, bd = oracle.bruteforce(q[:2], idx.vectors, k, idx.metric)
            gt_check = bool(np.allclose(bd[:, -1], dk[:2].double().cpu().numpy(), rtol=0, atol=0))
        # reported distances against FP64 on a few queries
        gi, gd = ids[:4].cpu().numpy(), dists[:4].cpu().numpy().astype(np.float64)
        rel = []
        for i in range(len(gi)):
            v = gi[i] >= 0
            d64 = oracle.rerank(q[i], idx.vectors, gi[i][v], idx.metric)
            rel.append(float(np.max(np.abs(gd[i][v] - d64) / np.maximum(np.abs(d64), 1e-30))))
        err = {"max_rel_err_vs_fp64": max(rel), "queries": len(gi)}
    # collector statistics for the algorithmic work per launch (outside the timed region)
    lists = torch.empty((nq, nprobe), dtype=torch.int32, device=dev)
    bbc.bbc_probe(h, qd, nq, nprobe, lists)
    sizes = torch.from_numpy(np.diff(idx.list_offsets)).to(dev)
    s_q = sizes[lists.long()].sum(1)
    stats = {"S_q_mean": float(s_q.double().mean())}
    del lists
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    bbc.bbc_set_param(h, "profile", 1)
    bbc.bbc_profile_read(h, reset=True)
    sampler = ClockSampler(local)
    sampler.start()
    barrier(ws)
    torch.cuda.synchronize()
    evs = []
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    barrier(ws)
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    stage_ms, launches = bbc.bbc_profile_read(h, reset=True)
    bbc.bbc_set_param(h, "profile", 0)
    bbc.bbc_stream_status(h)
    t_dev = sum(step_ms) / 1e3
    t_max = max_over_ranks(ws, t_dev)
    value = ws * nq * args.steps / t_max

    # end to end through the host entry point: pinned host queries in, host results out
    hq = torch.from_numpy(q).pin_memory()
    hi = torch.empty((nq, k), dtype=torch.int64).pin_memory()
    hd = torch.empty((nq, k), dtype=torch.float32).pin_memory()
    bbc.bbc_search_host(h, hq, nq, k, nprobe, hi, hd, stream)
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        bbc.bbc_search_host(h, hq, nq, k, nprobe, hi, hd, stream)
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(ws, time.perf_counter() - t0)
    e2e = {"value": ws * nq * args.e2e_steps / t_e2e, "unit": UNIT,
           "h2d_bytes_per_step": int(q.nbytes), "d2h_bytes_per_step": int(nq * k * (8 + 4))}
    assert torch.equal(hi, ids.cpu()), "host entry point disagrees with the device entry point"
    del hi, hd, hq

    # roofline of the dominant stage
    per = {s: stage_ms[s] / args.steps for s in stage_ms}
    peaks = _peaks()
    # the lookup peak at the SM clock sampled during the timed region (maximum clock if none was sampled)
    sm_clk = clocks.get("sm_mhz") or 2070.0
    lookups = float(s_q.double().sum()) * (idx.pq_m if not is_sign else 0)
    dpad = (idx.d + 15) // 16 * 16
    u8 = bool(index.get("rerank"))
    if prec:
        rr_bytes = nq * kc * (dpad * (2 if prec == 1 else 1) + 16 + 4 + 8)
    elif per.get("topk", 0.0) <= 0.0:
        # re-rank and top-k in one kernel: rows and ids in, the k results out (distances stay on chip)
        rr_bytes = nq * kc * (idx.d * (1 if u8 else 4) + 4) + nq * k * 12
    else:
        rr_bytes = nq * kc * (idx.d * (1 if u8 else 4) + 4 + 4)
    unc = (pstats["fp32_rechecked"] if pstats else 0) * args.steps / max(1, args.steps)
    work = {
        "scan": ("alu", lookups / 1e9, "Glookup/s", SMS * LOOKUPS_PER_SM_CLK * sm_clk * 1e6 / 1e9),
        "rerank": ("hbm", rr_bytes / 1e9, "GB/s", peaks["hbm_gbs"]),
        "topk": ("hbm", nq * ((k if prec else kc) * 8 + k * 12) / 1e9, "GB/s", peaks["hbm_gbs"]),
        "select": ("hbm", nq * kc * 8 * 2 / 1e9, "GB/s", peaks["hbm_gbs"]),
        "probe_scores": ("tensor", 2.0 * nq * idx.nlist * idx.d / 1e12, "TFLOP/s", peaks["bf16_tflops"]),
        "probe_select": ("hbm", nq * idx.nlist * 4 / 1e9, "GB/s", peaks["hbm_gbs"]),
        "lut": ("hbm", nq * getattr(idx, "pq_m", 0) * (1 << getattr(idx, "pq_bits", 0)) * 2 / 1e9, "GB/s",
                peaks["hbm_gbs"]),
        "prec_classify": ("hbm", nq * kc * 8 * 5 / 1e9, "GB/s", peaks["hbm_gbs"]),
        "prec_recheck": ("hbm", unc * (idx.d * 4 + 16) / 1e9, "GB/s", peaks["hbm_gbs"]),
    }
    tc = bool(index.get("scan_tc")) if not is_sign else False
    if tc:
        # the one-hot contraction: 2 x 16 M flops per (query, scanned object) pair (K = 16 M table
        # entries), FP16 operands, FP32 accumulation; FP16 and BF16 share the dense tensor rate
        work["scan"] = ("tensor", float(s_q.double().sum()) * 2.0 * 16 * idx.pq_m / 1e12, "TFLOP/s",
                        peaks["bf16_tflops"])
    if is_sign:
        # codes (d/8 bytes) + factors (16 bytes) per scanned object; rows of the exact re-rank
        work["scan"] = ("hbm", float(s_q.double().sum()) * (idx.d // 8 + 16) / 1e9, "GB/s", peaks["hbm_gbs"])
        if prec:
            work["rerank"] = ("hbm", bstats["exact"] * (dpad * (2 if prec == 1 else 1) + 28) / 1e9, "GB/s",
                              peaks["hbm_gbs"])
            work["prec_recheck"] = ("hbm", (unc + nq * k) * (idx.d * 4 + 8) / 1e9, "GB/s", peaks["hbm_gbs"])
        else:
            work["prec_recheck"] = ("hbm", bstats["exact"] * (idx.d * 4 + 8) / 1e9, "GB/s", peaks["hbm_gbs"])
        work["select"] = ("hbm", bstats["scanned"] * 16 * 3 / 1e9, "GB/s", peaks["hbm_gbs"])
        work["prec_classify"] = ("hbm", bstats["exact"] * 12 * 5 / 1e9, "GB/s", peaks["hbm_gbs"])
        work["topk"] = ("hbm", nq * k * 20 / 1e9, "GB/s", peaks["hbm_gbs"])
        work["lut"] = ("hbm", nq * idx.d * 12 / 1e9, "GB/s", peaks["hbm_gbs"])
    dom = max(per, key=lambda s: per[s])
    bound, amount, unit, peak = work[dom]
    achieved = amount / (per[dom] / 1e3)
    traffic, traffic_src = captured_traffic(dom, w.name, nprobe, kc, nq, bool(index.get("pair")))
    roof = {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_src,
            "peak_source": (f"152 SMs x 32 four-byte shared-memory lookups per clock x {sm_clk:.0f} MHz "
                            "(median SM clock sampled during the timed region)") if dom == "scan" and not tc
            else "MEASURED_PEAKS.json (measured copy / cuBLAS BF16 burst)"}
    if tc and "scan" in per:
        # the same scan as table lookups per second, beside the SIMT scan's shared-memory lookup peak
        roof["scan_lookup_rate"] = {"achieved": lookups / 1e9 / (per["scan"] / 1e3), "unit": "Glookup/s",
                                    "simt_lookup_peak": SMS * LOOKUPS_PER_SM_CLK * sm_clk * 1e6 / 1e9}

    cpu, cpu_mt = None, None
    if rank == 0 and not args.no_cpu_baseline:
        cpu, cpu_mt = cpu_baselines(args, idx, q, [k] * nq, [nprobe] * nq, kc_ratio=ratio,
                                    scale=index.get("bound_scale") if is_sign else None,
                                    estimator=int(index.get("estimator")) if is_sign else 0,
                                    eps0=index.get("epsilon0") if is_sign else 1.9,
                                    lut_levels=65535 if is_sign else int(index.get("lut_levels")))

    if rank == 0:
        rerank = ["u8-exact" if u8 else "f32", "bf16-prefilter", "fp8e4m3-prefilter"][prec]
        if is_sign:
            rerank = "bounded, two rounds, " + ["f32", "bf16 prefilter + f32", "e4m3 prefilter + f32"][prec] + \
                " (f64 at ties)"
        out = {
            "metric": METRICS.get(args.workload, METRIC), "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ("1-bit codes x 4-bit query planes (AND+POPC), f32 bounds, f32 re-rank (f64 at ties)" if is_sign
                      else ("f16 one-hot x f16 table (integers <= 2047) -> f32 ADC, " if tc else "u16/u32 ADC, ") +
                      {0: "f32 re-rank", 1: "bf16+f32 re-rank (f64 at ties)",
                       2: "e4m3+f32 re-rank (f64 at ties)"}[prec]),
            "data": "synthetic",
            "config": {"workload": w.name, "n": idx.n, "d": idx.d, "nlist": idx.nlist, "metric_space": idx.metric,
                       "pq": pq_desc(idx), "nq": nq, "k": k,
                       "nprobe": nprobe, "kc": None if is_sign else kc,
                       "kc_ratio": ratio, "buckets": m, "rerank": rerank,
                       "scan_schedule": ("list-grouped, tensor cores" if tc else
                                         "pair" if index.get("pair") else "one query per CTA"),
                       "lut_levels": int(index.get("lut_levels")),
                       "collector": ["result buffer", "lazy linear buffer", "binary heap"][int(index.get("collector"))],
                       "early_rerank": bool(index.get("early_rerank")),
                       "recall_at_k": rec_mean, "recall_at_k_min": rec_min, "recall_queries": nrec,
                       "recall_tie_aware": True, "ground_truth_cpu_spotcheck": gt_check,
                       "l2_flush_between_steps": True, "parallelism": f"replicas x{ws}",
                       "S_q_mean": stats["S_q_mean"], "index_build_s": round(t_build, 1), "wall_s_timed": wall},
            "stage_ms_per_step": per,
            "roofline": roof,
            "cpu_baseline": cpu,
            "cpu_baseline_all_cores": cpu_mt,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks,
        }
        if is_sign:
            out["bounded"] = {"per_step": bstats, "in_S_per_query": bstats["in_S"] / nq,
                              "exact_per_query": bstats["exact"] / nq,
                              "bound_scale": index.get("bound_scale"),
                              "bounds": "RaBitQ estimator, probabilistic" if index.get("estimator") else "hard",
                              "epsilon0": index.get("epsilon0") if index.get("estimator") else None}
        if estats:
            out["early_rerank"] = {"scored_early_per_query": estats["scored_early"] / nq,
                                   "used_per_query": estats["used"] / nq, "kc": kc}
        if prec:
            out["precision"] = {"per_step": pstats, "fp32_recheck_frac": pstats["fp32_rechecked"] / max(1, pstats["scored"]),
                                "fp64_frac": pstats["fp64_scored"] / max(1, pstats["scored"])}
        if err:
            out["error_vs_fp64"] = err
        if rec_mean < 0.95:
            out["warning"] = "recall below 0.95 at this operating point"
        print(json.dumps(out), flush=True)
    del ids, dists, flush, qd
    torch.cuda.empty_cache()


def cpu_baselines(args, idx, q, ks, ps, kc_ratio=None, scale=None, estimator=0, eps0=1.9, lut_levels=65535):
    """The oracle, as it stands, timed on the host: single-threaded on the first
    --cpu-queries queries, and on all host cores over a larger sample split
    across threads (ctypes releases the interpreter lock during the C call, so
    each thread runs one oracle call on its own query shard).  ks / ps: k and
    nprobe of every query."""
    import concurrent.futures as cf
    import oracle
    oracle.build()
    is_sign = hasattr(idx, "rotation")
    nq = len(q)
    cores = os.cpu_count() or 1
    seps = oracle.rotation_eps(idx.rotation) if is_sign else None

    def kc_of(k):
        return max(k, int(math.ceil(kc_ratio * k - 1e-9)))

    def prepare(sel):
        # index preparation outside the timed region: sign codes of the probed lists
        if not is_sign:
            return None
        probed = [oracle.probe(q[i], idx.centroids, int(ps[i]), idx.metric)[0] for i in sel]
        return oracle.sign_encode_lists(idx, np.concatenate(probed))

    def run(sel, prep):
        # queries of equal (k, nprobe) go through one oracle call
        groups = {}
        for i in sel:
            groups.setdefault((int(ks[i]), int(ps[i])), []).append(i)
        for (k, p), ii in groups.items():
            if is_sign:
                oracle.sign_search(idx, q[ii], k, p, scale=scale, codes=prep[0], fac=prep[1], eps=seps,
                                   estimator=estimator, eps0=eps0)
            else:
                oracle.search(idx, q[ii], k, p, kc_of(k), "sort", lut_levels=lut_levels)

    n1 = min(args.cpu_queries, nq)
    sel1 = list(range(n1))
    prep1 = prepare(sel1)
    t0 = time.perf_counter()
    run(sel1, prep1)
    t1 = time.perf_counter() - t0
    single = {"value": n1 / t1, "unit": UNIT, "cores": 1, "kind": "oracle",
              "sample": f"first {n1} of the {nq} queries on the full index, single-threaded C"}
    nm = min(args.cpu_mt_queries or 64 * cores, nq)
    shards = [list(range(nm))[c::cores] for c in range(cores)]
    shards = [sh for sh in shards if sh]
    prep_all = prepare(list(range(nm)))                 # one encoding of all probed lists, shared
    preps = [prep_all] * len(shards)
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=len(shards)) as ex:
        list(ex.map(lambda a: run(*a), zip(shards, preps)))
    tm = time.perf_counter() - t0
    allc = {"value": nm / tm, "unit": UNIT, "cores": len(shards), "kind": "oracle, threaded over queries",
            "sample": f"first {nm} of the {nq} queries on the full index, one oracle call per thread and shard"}
    return single, allc


def _source_sha(rel):
    import hashlib
    try:
        return hashlib.sha256(open(os.path.join(ROOT, rel), "rb").read()).hexdigest()
    except OSError:
        return None


def captured_traffic(kernel, workload, nprobe, kc, nq, pair):
    """DRAM bytes per launch of the dominant kernel from the ncu capture recorded in
    profiles/traffic.json, scaled to this launch by queries, or None when no capture
    matches this workload or the kernel's source has changed since the capture."""
    try:
        table = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except (OSError, ValueError):
        return None, "no capture"
    for e in table.get("captures", []):
        if (e.get("stage") == kernel and e.get("workload") == workload and e.get("nprobe") == nprobe
                and e.get("kc") == kc and bool(e.get("pair", False)) == pair):
            if _source_sha(e["source"]) != e.get("source_sha256"):
                return None, f"{e['kernel']}: source changed since the capture"
            return e["dram_bytes"] / e["queries"] * nq, (f"{e['kernel']}, ncu capture of {e['queries']} queries "
                                                        f"scaled by queries ({e['file']})")
    return None, "no capture of this kernel and workload"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"])}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


if __name__ == "__main__":
    main()
