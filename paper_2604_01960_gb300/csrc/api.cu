// Host side of libbbc: the C ABI declared in include/bbc.h.
//
// Owns the device-resident index (layout described in bbc_internal.cuh), the
// per-(index, stream) workspaces, argument checking and the launch sequence
// of the search path:
//   S1 probe scores -> S2 exact probe selection -> S3 uint16 LUT ->
//   S4-S6 scan + bucket-based result buffer -> S7 final selection ->
//   S8 exact re-rank -> S9 final top-k.
// Queries are processed in chunks whose workspace fits the budget.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "bbc_internal.cuh"

namespace bbc {
bool scan_supported(int M, int bits);

cudaError_t smem_attr_once(const void* kernel, int bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static std::mutex mu;
    static std::set<std::tuple<const void*, int, int>> done;
    const auto key = std::make_tuple(kernel, dev, bytes);
    std::lock_guard<std::mutex> lk(mu);
    if (done.count(key)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.insert(key);
    return e;
}
}

using namespace bbc;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CUDA_TRY(expr)                                                                  \
    do {                                                                                \
        cudaError_t _e = (expr);                                                        \
        if (_e != cudaSuccess)                                                          \
            return fail(BBC_ERR_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(_e),  \
                        __FILE__, __LINE__);                                            \
    } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

struct Workspace {
    char* base = nullptr;
    size_t bytes = 0;
};

size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }
constexpr int BBC_ERR_STATE_CAPTURE = BBC_ERR_BUSY;

// FP32 -> BF16, round to nearest even (NaN kept quiet).
uint16_t f32_to_bf16(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7FFFFFFFu) > 0x7F800000u) return 0x7FC0;
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
float bf16_to_f32(uint16_t h) {
    uint32_t u = (uint32_t)h << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

}  // namespace

struct bbc_index {
    int device = 0;
    bbc_index_info_t info{};
    DevIndex dev{};
    std::vector<void*> owned;
    std::vector<int64_t> cap_prefix;     // cap_prefix[p] = sum of the p longest lists
    int64_t region_cap = 0;              // entries of a query's collector region; 0 = cap_prefix[nprobe]
    // Capacity of the collector region of a query probing nprobe lists: every
    // scanned object fits unless "region_cap" lowers it (appends past the
    // capacity are dropped and latch a region overrun).
    int64_t cap_for(int nprobe) const {
        const int64_t c = cap_prefix[nprobe];
        return region_cap > 0 && region_cap < c ? region_cap : c;
    }
    // parameters
    double kc_ratio = 1.5;
    int buckets = 64;
    int sample_lists = 8;
    int rerank_u8 = 1;
    int probe_gemm = 1;
    void* lp_rows = nullptr;               // low-precision copy (precision re-rank)
    float4* lp_meta = nullptr;
    unsigned long long* prec_totals = nullptr;   // [4] device counters of the precision re-rank
    unsigned long long* sign_totals = nullptr;   // [4] device counters of the bounded re-rank
    float bound_scale = 1.f;                     // sign codes: factor on the residual term
    int estimator = 0;                           // sign codes: 0 hard bounds, 1 RaBitQ estimator
    float eps0 = 1.9f;                           // its confidence parameter epsilon_0
    float first_round = 2.f;                     // sign codes: first re-rank round, a multiple of k
    int split = 0;            // 0 automatic, 1 one CTA per query, G >= 2 CTAs per query
    int pair = 0;             // 1: two queries per CTA (pair form) where supported, 0: one
    int collector = 0;        // 0 the bucket-based result buffer; 1 lazy linear buffer, 2 binary heap (baselines)
    int early_rerank = 0;     // 1: Algorithm 4's early re-rank in the scan (exact u8 re-rank, one CTA per query)
    int64_t nslots = 0;       // code-block slots (32 per block)
    uint8_t* lo_rows = nullptr;                 // early re-rank: u8 rows in slot order
    uint32_t* lo_norms = nullptr;               // and their squared norms
    unsigned long long* early_totals = nullptr; // [2] objects scored early, early distances used
    int graphs = 0;           // 1: capture each bbc_search shape into a CUDA graph and replay it
    int lut_levels = 65535;   // top level of the integer lookup tables
    int scan_tc = 0;          // 1: list-grouped scan on the tensor cores (4-bit codes; tables <= 2047)
    int rerank_fused = 0;     // 1: re-rank and top-k in one kernel where the candidates fit in shared memory
    bool capturing = false;
    struct GraphKey {
        const void* q; int64_t nq; int k; int nprobe; void* oi; void* od; cudaStream_t st;
        double kc_ratio; int buckets, sample_lists, split, probe_gemm, rerank, prec;
        int64_t rcap;
        int pair, collector, early, lut_levels, scan_tc, rerank_fused;
        bool operator<(const GraphKey& o) const {
            return std::tie(q, nq, k, nprobe, oi, od, st, kc_ratio, buckets, sample_lists, split, probe_gemm, rerank,
                            prec, rcap, pair, collector, early, lut_levels, scan_tc, rerank_fused) <
                   std::tie(o.q, o.nq, o.k, o.nprobe, o.oi, o.od, o.st, o.kc_ratio, o.buckets, o.sample_lists, o.split,
                            o.probe_gemm, o.rerank, o.prec, o.rcap, o.pair, o.collector, o.early, o.lut_levels,
                            o.scan_tc, o.rerank_fused);
        }
    };
    struct GraphEntry { cudaGraphExec_t exec; int64_t launches; };
    std::map<GraphKey, GraphEntry> graph_cache;
    std::mutex graph_mu;
    double workspace_mb = 8192.0;
    int profile = 0;
    std::mutex mu;
    // tracing
    std::mutex prof_mu;
    struct Rec { int stage; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    int64_t launches = 0;
    std::map<cudaStream_t, Workspace> ws;
    cudaStream_t copy_stream = nullptr;   // host entry points: results copied out while the next part computes

    ~bbc_index() {
        int prev = -1;
        cudaGetDevice(&prev);
        cudaSetDevice(device);
        for (auto& kv : graph_cache) cudaGraphExecDestroy(kv.second.exec);
        for (auto& kv : ws) cudaFree(kv.second.base);
        if (copy_stream) cudaStreamDestroy(copy_stream);
        for (auto& r : recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
        for (void* p : owned) cudaFree(p);
        cudaFree(lp_rows);
        cudaFree(lp_meta);
        cudaFree(prec_totals);
        cudaFree(sign_totals);
        cudaFree(lo_rows);
        cudaFree(lo_norms);
        cudaFree(early_totals);
        if (prev >= 0) cudaSetDevice(prev);
    }
};

namespace {

template <typename T>
int upload(bbc_index* ix, const T* h, size_t count, T** out) {
    void* p = nullptr;
    size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return fail(BBC_ERR_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    ix->owned.push_back(p);
    ix->info.device_bytes += (int64_t)bytes;
    if (count) {
        e = cudaMemcpy(p, h, count * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(BBC_ERR_CUDA, "cudaMemcpy: %s", cudaGetErrorString(e));
    }
    *out = static_cast<T*>(p);
    return BBC_OK;
}

// Workspace arena for one chunk of queries.  Sizes come from per-chunk sums so
// that uniform and mixed (per-query k / nprobe) batches share one layout.
struct ChunkShape {
    int64_t nq = 0;
    int64_t sum_probe = 0, sum_cap = 0, sum_kc = 0, sum_k = 0;
    int max_probe = 0;
    int64_t max_kc = 0;
    bool host_io = false;
    bool mixed = false;
};

struct Plan {
    int64_t chunk;        // queries per chunk (uniform batches)
    int64_t chunk_slots;  // candidate slots of a mixed chunk (sum of K_c)
    int64_t chunk_probe;  // probe lists of a mixed chunk (sum of nprobe)
    int nprobe;
    int64_t kc;
    int k;
    int64_t cap;
    size_t off_scores, off_probe, off_lut, off_state, off_region, off_cand, off_count, off_cdist,
        off_q, off_ids, off_dists, off_abf, off_keys, off_params, off_counters, off_prec, off_pair, off_rdist,
        off_cearly, off_qinv, off_lbase, off_lutf16, off_tcplan, total;
};

// The precision re-rank runs when a low-precision copy exists and the exact u8
// re-rank (already exact at one byte per component) is not in use.
bool prec_active(const bbc_index* ix) {
    return ix->dev.prec > 0 && ix->dev.vec_lp && !(ix->rerank_u8 && ix->dev.vec_u8);
}

// Algorithm 4's early re-rank runs with the exact u8 re-rank, one CTA per
// query and the result buffer (not the precision form, the pair or split
// scan, or a baseline collector).
bool early_active(const bbc_index* ix);

// Scratch of the precision re-rank inside a workspace: per candidate slot
// rho, uncertain ids, final ids / distances, band ids (4 B each) and band
// FP64 distances (8 B); per query n_fin, n_unc, item offsets and ||q||.
size_t prec_bytes(int64_t nq, int64_t slots) {
    size_t o = 0;
    for (int i = 0; i < 5; ++i) o = align_up(o + (size_t)slots * 4);
    o = align_up(o + (size_t)slots * 8);
    o = align_up(o + (size_t)nq * 8 * 2 + (size_t)(nq + 1) * 8 + (size_t)nq * 4);
    return o;
}
PrecArgs prec_args(const bbc_index* ix, char* base, int64_t nq, int64_t slots) {
    PrecArgs a{};
    size_t o = 0;
    auto take = [&](size_t bytes) { char* p = base + o; o = align_up(o + bytes); return p; };
    a.rho = reinterpret_cast<float*>(take((size_t)slots * 4));
    a.unc = reinterpret_cast<uint32_t*>(take((size_t)slots * 4));
    a.fin_id = reinterpret_cast<uint32_t*>(take((size_t)slots * 4));
    a.fin_d = reinterpret_cast<float*>(take((size_t)slots * 4));
    a.band_id = reinterpret_cast<uint32_t*>(take((size_t)slots * 4));
    a.band_d = reinterpret_cast<double*>(take((size_t)slots * 8));
    char* pq = take((size_t)nq * 8 * 2 + (size_t)(nq + 1) * 8 + (size_t)nq * 4);
    a.n_fin = reinterpret_cast<int64_t*>(pq);
    a.n_unc = a.n_fin + nq;
    a.item_off = a.n_unc + nq;
    a.qnorm = reinterpret_cast<float*>(a.item_off + nq + 1);
    a.totals = ix->prec_totals;
    return a;
}
// The precision path: the recheck reads the uncertain list and writes over the
// dead pass-1 scores, which the finalize then reads.
PrecArgs prec_args_rerank(const bbc_index* ix, char* base, int64_t nq, int64_t slots, float* cdist) {
    PrecArgs a = prec_args(ix, base, nq, slots);
    a.unc_d = cdist;
    a.unc_r = a.rho;
    a.copy_unc = 0;
    a.rc_ids = a.unc;
    a.rc_from = nullptr;
    a.rc_count = a.n_unc;
    a.rc_d = cdist;
    a.rc_r = a.rho;
    return a;
}

bool early_active(const bbc_index* ix) {
    return ix->early_rerank && ix->dev.vec_lo && ix->rerank_u8 && ix->dev.vec_u8 && !prec_active(ix) &&
           ix->collector == 0;
}

// The tensor-core list-grouped scan runs when asked for, on plain 4-bit PQ
// codes with the result buffer (not a baseline collector or the early
// re-rank); the tables then have top level lut_levels <= 2047.
bool tc_active(const bbc_index* ix) { return ix->scan_tc && ix->collector == 0 && !early_active(ix); }

// K_c (or k) above which the workspace holds 64-bit keys for the global-scratch
// top-k.  That form runs only when k - 1 + 1,024 kept keys exceed shared memory
// (k above 23,552); since K_c >= k the bound is conservative: it may reserve
// keys the shared-memory top-k then does not use.
constexpr int64_t kTopkSmemMax = 16384;
constexpr int64_t kMaxChunkQueries = 65535;  // queries per launch (some grids index queries in y)

size_t layout(const bbc_index* ix, const ChunkShape& c, Plan& p) {
    const DevIndex& d = ix->dev;
    size_t o = 0;
    p.off_scores = o; o = align_up(o + (size_t)c.nq * d.nlist * 4);
    p.off_probe = o; o = align_up(o + (size_t)c.sum_probe * 4);
    p.off_lut = o; o = align_up(o + (size_t)c.nq * d.M * d.K * 2);
    p.off_state = o; o = align_up(o + (size_t)c.nq * sizeof(bbc_collector_state));
    p.off_region = o; o = align_up(o + (size_t)c.sum_cap * 8);
    p.off_cand = o; o = align_up(o + (size_t)c.sum_kc * 4);
    p.off_count = o; o = align_up(o + (size_t)c.nq * 8);
    p.off_cdist = o; o = align_up(o + (size_t)c.sum_kc * 4);
    p.off_q = o; o = align_up(o + (c.host_io ? (size_t)c.nq * d.d * 4 : 0));
    p.off_ids = o; o = align_up(o + (c.host_io ? (size_t)c.sum_k * 8 : 0));
    p.off_dists = o; o = align_up(o + (c.host_io ? (size_t)c.sum_k * 4 : 0));
    p.off_abf = o; o = align_up(o + (ix->probe_gemm ? probe_tc_workspace(d, c.nq) : 0));
    p.off_keys = o; o = align_up(o + (c.max_kc > kTopkSmemMax ? (size_t)c.sum_kc * 8 : 0));
    p.off_params = o; o = align_up(o + (c.mixed ? (size_t)(c.nq + 1) * 8 * 7 : 0));
    p.off_counters = o; o = align_up(o + 16);
    p.off_prec = o; o = align_up(o + (prec_active(ix) ? prec_bytes(c.nq, c.sum_kc) : 0));
    p.off_pair = o; o = align_up(o + (ix->pair ? pair_plan_bytes(c.nq) : 0));
    const bool early = ix->early_rerank && ix->dev.vec_lo;
    p.off_rdist = o; o = align_up(o + (early ? (size_t)c.sum_cap * 4 : 0));
    p.off_cearly = o; o = align_up(o + (early ? (size_t)c.sum_kc * 4 : 0));
    p.off_qinv = o; o = align_up(o + (d.resid ? (size_t)c.nq * 4 : 0));
    p.off_lbase = o; o = align_up(o + (d.resid ? (size_t)c.sum_probe * 4 : 0));
    const bool tc = tc_active(ix);
    p.off_lutf16 = o; o = align_up(o + (tc ? (size_t)c.nq * d.M * d.K * 2 : 0));
    p.off_tcplan = o; o = align_up(o + (tc ? scan_tc_plan_bytes(d, c.sum_probe) : 0));
    p.total = o;
    return o;
}

Plan make_plan(const bbc_index* ix, int64_t nq, int nprobe, int64_t kc, int k, bool host_io) {
    Plan p{};
    p.nprobe = nprobe;
    p.kc = kc;
    p.k = k;
    p.cap = ix->cap_for(nprobe);
    auto shape = [&](int64_t c) {
        ChunkShape s;
        s.nq = c; s.sum_probe = c * nprobe; s.sum_cap = c * p.cap; s.sum_kc = c * kc; s.sum_k = c * k;
        s.max_probe = nprobe; s.max_kc = kc; s.host_io = host_io;
        return s;
    };
    const size_t budget = (size_t)(ix->workspace_mb * 1024.0 * 1024.0);
    int64_t c = std::max<int64_t>(1, std::min<int64_t>(nq, kMaxChunkQueries));
    Plan tmp = p;
    while (c > 1 && layout(ix, shape(c), tmp) > budget) c = (c + 1) / 2;
    p.chunk = c;
    layout(ix, shape(c), p);
    return p;
}

int get_workspace(bbc_index* ix, cudaStream_t st, size_t bytes, char** base) {
    std::lock_guard<std::mutex> lk(ix->mu);
    Workspace& w = ix->ws[st];
    if (w.bytes < bytes) {
        if (w.base) {
            cudaError_t e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return fail(BBC_ERR_CUDA, "sync before workspace growth: %s", cudaGetErrorString(e));
            cudaFree(w.base);
            w.base = nullptr;
            w.bytes = 0;
        }
        if (ix->capturing) return fail(BBC_ERR_STATE_CAPTURE, "workspace growth during graph capture");
        for (auto& kv : ix->graph_cache) cudaGraphExecDestroy(kv.second.exec);
        ix->graph_cache.clear();
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) return fail(BBC_ERR_OOM, "workspace cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
        w.base = static_cast<char*>(p);
        w.bytes = bytes;
    }
    *base = w.base;
    return BBC_OK;
}

int64_t kc_for(const bbc_index* ix, int k) {
    int64_t kc = (int64_t)std::ceil(ix->kc_ratio * (double)k - 1e-9);
    return std::max<int64_t>(kc, k);
}

int check_search_args(const bbc_index* ix, const void* queries, int64_t nq, int k, int nprobe,
                      const void* out_ids, const void* out_dists) {
    if (!ix) return fail(BBC_ERR_ARG, "null index");
    if (nq < 0) return fail(BBC_ERR_ARG, "nq < 0");
    if (nq > 0 && (!queries || !out_ids || !out_dists)) return fail(BBC_ERR_ARG, "null buffer");
    if (k <= 0) return fail(BBC_ERR_ARG, "k must be >= 1 (got %d)", k);
    if (nprobe < 1 || nprobe > ix->dev.nlist) return fail(BBC_ERR_ARG, "nprobe %d outside [1, %d]", nprobe, ix->dev.nlist);
    if (nprobe > 2048) return fail(BBC_ERR_UNSUPPORTED, "nprobe %d > 2048", nprobe);
    return BBC_OK;
}

// Launch one stage, counting it and (when profiling) bracketing it with events.
template <typename F>
cudaError_t stage(bbc_index* ix, int id, cudaStream_t st, F&& launch) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (ix->profile && !ix->capturing) {
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return cudaErrorMemoryAllocation;
        cudaEventRecord(a, st);
    }
    cudaError_t e = launch();
    {
        std::lock_guard<std::mutex> lk(ix->prof_mu);
        ix->launches += 1;
        if (ix->profile && !ix->capturing) {
            cudaEventRecord(b, st);
            ix->recs.push_back({id, a, b});
        }
    }
    return e;
}

// S8 + S9 for a chunk: the plain re-rank and top-k, or the precision form
// (low-precision scores, classification, FP32 recheck, FP64 decision, top-k
// of the final members).  maxk: the largest k of the chunk.
int run_rerank(bbc_index* ix, int64_t nc, const RerankArgs& ra, const PrecArgs* pa, int maxk, cudaStream_t st) {
    const DevIndex& d = ix->dev;
    if (!pa) {
        if (ix->rerank_fused && rerank_topk_fits(d, ra)) {
            // both steps in one kernel: recorded as the re-rank stage
            CUDA_TRY(stage(ix, 5, st, [&] { return launch_rerank_topk(d, nc, ra, st); }));
            return BBC_OK;
        }
        CUDA_TRY(stage(ix, 5, st, [&] { return launch_rerank(d, nc, ra, st); }));
        CUDA_TRY(stage(ix, 6, st, [&] { return launch_topk(d, nc, ra, st); }));
        return BBC_OK;
    }
    CUDA_TRY(stage(ix, 5, st, [&] { return launch_prec_score(d, nc, ra, *pa, st); }));
    CUDA_TRY(stage(ix, 7, st, [&] { return launch_prec_classify(d, nc, ra, *pa, st); }));
    CUDA_TRY(stage(ix, 7, st, [&] { return launch_prec_plan(nc, *pa, st); }));
    CUDA_TRY(stage(ix, 8, st, [&] { return launch_prec_recheck(d, nc, ra, *pa, st); }));
    CUDA_TRY(stage(ix, 7, st, [&] { return launch_prec_finalize(d, nc, ra, *pa, st); }));
    RerankArgs rb = ra;
    rb.cand = pa->fin_id;
    rb.cdist = pa->fin_d;
    rb.cand_count = pa->n_fin;
    rb.kc = maxk;
    CUDA_TRY(stage(ix, 6, st, [&] { return launch_topk(d, nc, rb, st); }));
    return BBC_OK;
}

// The launch sequence for one chunk.
int run_chunk(bbc_index* ix, const Plan& p, char* ws, const float* q, int64_t nc, int64_t* out_ids,
              float* out_dists, cudaStream_t st, int stop_after /* 9 = all */,
              int32_t* probe_out = nullptr, const int32_t* probe_in = nullptr, uint32_t* cand_out = nullptr,
              int64_t* count_out = nullptr, bbc_collector_state* state_out = nullptr,
              const QueryParams* qp_in = nullptr) {
    const DevIndex& d = ix->dev;
    const QueryParams qp = qp_in ? *qp_in : uniform_params(p.nprobe, p.kc, p.k, p.cap);
    float* scores = reinterpret_cast<float*>(ws + p.off_scores);
    int32_t* probe = probe_out ? probe_out : reinterpret_cast<int32_t*>(ws + p.off_probe);
    uint16_t* lut = reinterpret_cast<uint16_t*>(ws + p.off_lut);
    bbc_collector_state* state = state_out ? state_out : reinterpret_cast<bbc_collector_state*>(ws + p.off_state);
    uint2* region = reinterpret_cast<uint2*>(ws + p.off_region);
    uint32_t* cand = cand_out ? cand_out : reinterpret_cast<uint32_t*>(ws + p.off_cand);
    int64_t* count = count_out ? count_out : reinterpret_cast<int64_t*>(ws + p.off_count);
    float* cdist = reinterpret_cast<float*>(ws + p.off_cdist);
    if (!probe_in) {
        if (ix->probe_gemm)
            CUDA_TRY(stage(ix, 0, st, [&] { return launch_probe_scores_tc(d, q, nc, scores, ws + p.off_abf, st); }));
        else
            CUDA_TRY(stage(ix, 0, st, [&] { return launch_probe_scores(d, q, nc, scores, st); }));
        CUDA_TRY(stage(ix, 1, st, [&] {
            return launch_probe_select(d, q, nc, qp, p.nprobe, scores, probe, ix->probe_gemm, st);
        }));
    }
    if (stop_after <= 2) return BBC_OK;
    float* qinv = d.resid ? reinterpret_cast<float*>(ws + p.off_qinv) : nullptr;
    const bool tc = tc_active(ix);
    uint16_t* lutf16 = tc ? reinterpret_cast<uint16_t*>(ws + p.off_lutf16) : nullptr;
    CUDA_TRY(stage(ix, 2, st, [&] { return launch_lut16(d, q, nc, lut, st, qinv, ix->lut_levels, lutf16); }));
    ScanArgs sa{lut, probe_in ? probe_in : probe, p.nprobe, p.kc, ix->buckets, ix->sample_lists,
                region, p.cap, state, qp, 0, SelectArgs{}};
    if (d.resid) {
        // residual IVF-PQ: each (query, probed list)'s base in the table's units
        int32_t* lbase = reinterpret_cast<int32_t*>(ws + p.off_lbase);
        CUDA_TRY(stage(ix, 2, st, [&] { return launch_resid_base(d, q, nc, qp, p.nprobe, sa.lists, qinv, lbase, st); }));
        sa.qinv = qinv;
        sa.lbase = lbase;
    }
    // one CTA per query when the batch fills the GPU, else G CTAs per query
    int G = ix->split >= 2 ? ix->split : 1;
    if (ix->split == 0) {
        const int64_t slots = 4ll * 2 * d.num_sms;
        if (nc < slots) G = (int)std::min<int64_t>((slots + nc - 1) / nc, std::max(1, p.nprobe));
    }
    if (tc) {
        // list-grouped form on the tensor cores: pairs grouped by list, sample pass,
        // codebooks, main pass; the selection follows as its own kernel
        if (!scan_tc_supported(d, ix->buckets) || ix->lut_levels > 2047)
            return fail(BBC_ERR_UNSUPPORTED, "scan_tc: needs plain 4-bit PQ codes (M = 32, 64 or 128), "
                        "buckets <= 64 and lut_levels <= 2047");
        const int64_t sum_probe = qp.probe_off ? p.chunk_probe : nc * (int64_t)p.nprobe;
        CUDA_TRY(cudaMemsetAsync(state, 0, (size_t)nc * sizeof(bbc_collector_state), st));
        CUDA_TRY(stage(ix, 3, st, [&] {
            return launch_scan_tc(d, nc, sa, lutf16, ws + p.off_tcplan, sum_probe, st);
        }));
    } else if (ix->collector) {
        // a baseline collector in place of the result buffer: it writes the candidates itself
        const uint32_t stage_cap = (uint32_t)((ix->info.max_list_len + 31) / 32 * 32);
        if (!scan_collect_supported(d, ix->collector, p.nprobe, p.kc, stage_cap))
            return fail(BBC_ERR_UNSUPPORTED, "collector %d: table shape, K_c %lld or residual codes not supported",
                        ix->collector, (long long)p.kc);
        sa.fuse_select = 1;
        sa.sel = SelectArgs{region, p.cap, state, p.kc, cand, count, nullptr, qp};
        CUDA_TRY(stage(ix, 3, st, [&] { return launch_scan_collect(d, nc, sa, ix->collector, stage_cap, st); }));
    } else if (G >= 2) {
        unsigned int* counters = reinterpret_cast<unsigned int*>(ws + p.off_counters);
        CUDA_TRY(cudaMemsetAsync(state, 0, (size_t)nc * sizeof(bbc_collector_state), st));
        CUDA_TRY(stage(ix, 3, st, [&] { return launch_scan_split(d, nc, sa, G, counters, st); }));
    } else if (ix->pair && nc >= 2 && scan_pair_supported(d, p.nprobe)) {
        // two queries per CTA: the pairing plan, then the pair form of the scan
        int32_t* perm = reinterpret_cast<int32_t*>(ws + p.off_pair) + 3 * nc;
        CUDA_TRY(stage(ix, 3, st, [&] {
            return launch_pair_plan(q, d.d, nc, qp, sa.lists, ws + p.off_pair, perm, st);
        }));
        CUDA_TRY(stage(ix, 3, st, [&] { return launch_scan_pair(d, nc, sa, perm, st); }));
    } else {
        // one CTA per query: the selection (S7) runs in the scan's tail
        sa.fuse_select = 1;
        sa.sel = SelectArgs{region, p.cap, state, p.kc, cand, count, nullptr, qp};
        if (early_active(ix)) {
            // Algorithm 4: exact distances of the objects below the predicted threshold bucket
            // are computed in the scan and carried to their candidates
            sa.early = 1;
            sa.q = q;
            sa.rdist = reinterpret_cast<float*>(ws + p.off_rdist);
            sa.early_totals = ix->early_totals;
            sa.sel.rdist = sa.rdist;
            sa.sel.cand_early = reinterpret_cast<float*>(ws + p.off_cearly);
        }
        CUDA_TRY(stage(ix, 3, st, [&] { return launch_scan(d, nc, sa, st); }));
    }
    if (!sa.fuse_select) {
        SelectArgs se{region, p.cap, state, p.kc, cand, count, nullptr, qp};
        CUDA_TRY(stage(ix, 4, st, [&] { return launch_select(d, nc, se, st); }));
    }
    if (stop_after <= 7) return BBC_OK;
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(ws + p.off_keys);
    RerankArgs ra{q, cand, count, p.kc, ix->rerank_u8 && d.vec_u8 != nullptr, cdist, p.k, out_ids,
                  out_dists, p.kc > kTopkSmemMax ? keys : nullptr, qp};
    if (sa.early) {
        ra.early = sa.sel.cand_early;
        ra.early_totals = ix->early_totals;
    }
    if (prec_active(ix)) {
        // slots of this chunk: sum of K_c (the per-query offsets index into them)
        const int64_t slots = qp.cand_off ? p.chunk_slots : nc * p.kc;
        const PrecArgs pa = prec_args_rerank(ix, ws + p.off_prec, nc, slots, cdist);
        return run_rerank(ix, nc, ra, &pa, p.k, st);
    }
    return run_rerank(ix, nc, ra, nullptr, p.k, st);
}

// ---------------------------------------------------------------------------
// Bounded re-rank on a sign-code index (S9b): probe, rotate, scan with the
// result buffer on the upper bound, two re-rank rounds, exact final order.
// ---------------------------------------------------------------------------
struct SignShape {
    int64_t nq = 0, sum_probe = 0, sum_cap = 0, sum_k = 0;
    int max_probe = 0, max_k = 0;
    bool host_io = false, mixed = false;
};

struct SignPlan {
    size_t off_scores, off_abf, off_probe, off_qrot, off_prep, off_region, off_small, off_clist, off_rkey, off_rid,
        off_cd, off_cr, off_ud, off_ur, off_keys, off_prec, off_params, off_q, off_ids, off_dists, total;
};

size_t sign_layout(const bbc_index* ix, const SignShape& c, SignPlan& p) {
    const DevIndex& d = ix->dev;
    const size_t slots = (size_t)c.sum_cap;
    size_t o = 0;
    p.off_scores = o; o = align_up(o + (size_t)c.nq * d.nlist * 4);
    p.off_abf = o; o = align_up(o + (ix->probe_gemm ? probe_tc_workspace(d, c.nq) : 0));
    p.off_probe = o; o = align_up(o + (size_t)c.sum_probe * 4);
    p.off_qrot = o; o = align_up(o + (size_t)c.nq * d.d * 8);
    p.off_prep = o; o = align_up(o + sign_prep_bytes(d, c.sum_probe));
    p.off_region = o; o = align_up(o + slots * 16);
    p.off_small = o; o = align_up(o + (size_t)c.nq * 8 * 5);         // pushed, scanned, n_b, n_c, n_rest
    p.off_clist = o; o = align_up(o + slots * 4);
    p.off_rkey = o; o = align_up(o + slots * 4);
    p.off_rid = o; o = align_up(o + slots * 4);
    p.off_cd = o; o = align_up(o + slots * 4);
    p.off_cr = o; o = align_up(o + slots * 4);
    p.off_ud = o; o = align_up(o + slots * 4);
    p.off_ur = o; o = align_up(o + slots * 4);
    p.off_keys = o; o = align_up(o + (c.max_k > kTopkSmemMax ? slots * 8 : 0));
    p.off_prec = o; o = align_up(o + prec_bytes(c.nq, (int64_t)slots));
    p.off_params = o; o = align_up(o + (c.mixed ? (size_t)(c.nq + 1) * 8 * 7 : 0));
    p.off_q = o; o = align_up(o + (c.host_io ? (size_t)c.nq * d.d * 4 : 0));
    p.off_ids = o; o = align_up(o + (c.host_io ? (size_t)c.sum_k * 8 : 0));
    p.off_dists = o; o = align_up(o + (c.host_io ? (size_t)c.sum_k * 4 : 0));
    p.total = o;
    return o;
}

SignShape sign_uniform_shape(const bbc_index* ix, int64_t nc, int nprobe, int k, bool host_io) {
    SignShape c;
    c.nq = nc;
    c.sum_probe = nc * nprobe;
    c.sum_cap = nc * ix->cap_for(nprobe);
    c.sum_k = nc * k;
    c.max_probe = nprobe;
    c.max_k = k;
    c.host_io = host_io;
    return c;
}

// One chunk of the bounded re-rank; qp gives each query's nprobe, k, region
// (capacity = its scanned objects at most) and result offsets.
int run_sign_chunk(bbc_index* ix, const SignPlan& p, const SignShape& c, char* ws, const float* q, int64_t nc,
                   const QueryParams& qp, int64_t* out_ids, float* out_dists, cudaStream_t st) {
    const DevIndex& d = ix->dev;
    float* scores = reinterpret_cast<float*>(ws + p.off_scores);
    int32_t* probe = reinterpret_cast<int32_t*>(ws + p.off_probe);
    double* qrot = reinterpret_cast<double*>(ws + p.off_qrot);
    int64_t* small = reinterpret_cast<int64_t*>(ws + p.off_small);
    int64_t *pushed = small, *scanned = small + nc, *n_b = small + 2 * nc, *n_c = small + 3 * nc,
            *n_rest = small + 4 * nc;
    uint32_t* clist = reinterpret_cast<uint32_t*>(ws + p.off_clist);
    float* cd = reinterpret_cast<float*>(ws + p.off_cd);
    float* cr = reinterpret_cast<float*>(ws + p.off_cr);
    if (ix->probe_gemm)
        CUDA_TRY(stage(ix, 0, st, [&] { return launch_probe_scores_tc(d, q, nc, scores, ws + p.off_abf, st); }));
    else
        CUDA_TRY(stage(ix, 0, st, [&] { return launch_probe_scores(d, q, nc, scores, st); }));
    CUDA_TRY(stage(ix, 1, st, [&] {
        return launch_probe_select(d, q, nc, qp, c.max_probe, scores, probe, ix->probe_gemm, st);
    }));
    CUDA_TRY(stage(ix, 2, st, [&] { return launch_rotate_f64(q, nullptr, nullptr, nullptr, d.rot, nc, d.d, qrot, st); }));
    SignArgs sa{};
    sa.qrot = qrot; sa.q = q; sa.lists = probe; sa.nprobe = c.max_probe; sa.k = c.max_k; sa.m = ix->buckets;
    sa.sample_min = ix->sample_lists; sa.scale = ix->bound_scale; sa.est = ix->estimator; sa.eps0 = ix->eps0;
    sa.region = reinterpret_cast<uint4*>(ws + p.off_region); sa.cap = qp.cap; sa.pushed = pushed; sa.scanned = scanned;
    sa.prep = reinterpret_cast<uint32_t*>(ws + p.off_prep);
    sa.qp = qp;
    CUDA_TRY(stage(ix, 3, st, [&] { return launch_sign_scan(d, nc, sa, st); }));
    SignSelectArgs ss{};
    ss.region = sa.region; ss.pushed = pushed; ss.scanned = scanned; ss.clist = clist; ss.n_b = n_b; ss.n_c = n_c;
    ss.rest_key = reinterpret_cast<uint32_t*>(ws + p.off_rkey); ss.rest_id = reinterpret_cast<uint32_t*>(ws + p.off_rid);
    ss.n_rest = n_rest; ss.cd = cd; ss.cr = cr; ss.totals = ix->sign_totals; ss.qp = qp; ss.first = ix->first_round;
    CUDA_TRY(stage(ix, 4, st, [&] { return launch_sign_select(d, nc, ss, st); }));
    PrecArgs pa = prec_args(ix, ws + p.off_prec, nc, c.sum_cap);
    pa.rho = cr;
    pa.unc_d = reinterpret_cast<float*>(ws + p.off_ud);
    pa.unc_r = reinterpret_cast<float*>(ws + p.off_ur);
    pa.copy_unc = 1;
    pa.rc_ids = clist;
    pa.rc_d = cd;
    pa.rc_r = cr;
    CUDA_TRY(cudaMemsetAsync(pa.qnorm, 0, (size_t)nc * sizeof(float), st));
    unsigned long long* keys = c.max_k > kTopkSmemMax ? reinterpret_cast<unsigned long long*>(ws + p.off_keys) : nullptr;
    RerankArgs ra{q, clist, n_c, qp.kc, 0, cd, c.max_k, out_ids, out_dists, keys, qp};
    if (d.prec > 0 && d.vec_lp) {
        // both rounds scored from the low-precision copy with its bound; then the
        // precision form's classification, FP32 recheck and FP64 decision
        RerankArgs r1 = ra;
        r1.cand_count = n_b;
        // grid sizing: the first round holds up to ceil(first_round * k) objects
        r1.kc = std::min<int64_t>(qp.kc, (int64_t)std::ceil((double)ix->first_round * c.max_k));
        pa.sc_from = nullptr;
        CUDA_TRY(stage(ix, 5, st, [&] { return launch_prec_score(d, nc, r1, pa, st); }));
        CUDA_TRY(stage(ix, 4, st, [&] { return launch_sign_filter(d, nc, ss, st); }));
        pa.sc_from = n_b;
        CUDA_TRY(stage(ix, 5, st, [&] { return launch_prec_score(d, nc, ra, pa, st); }));
        pa.sc_from = nullptr;
        pa.copy_unc = 0;
        pa.rc_ids = pa.unc;
        pa.rc_from = nullptr;
        pa.rc_count = pa.n_unc;
        pa.rc_d = pa.unc_d;
        pa.rc_r = pa.unc_r;
        CUDA_TRY(stage(ix, 7, st, [&] { return launch_prec_classify(d, nc, ra, pa, st); }));
        CUDA_TRY(stage(ix, 8, st, [&] { return launch_prec_plan(nc, pa, st); }));
        CUDA_TRY(stage(ix, 8, st, [&] { return launch_prec_recheck(d, nc, ra, pa, st); }));
        CUDA_TRY(stage(ix, 7, st, [&] { return launch_prec_finalize(d, nc, ra, pa, st); }));
        // exact returned distances: the final members re-scored from the FP32 rows
        RerankArgs rf = ra;
        rf.cand = pa.fin_id;
        rf.cand_count = pa.n_fin;
        rf.cdist = pa.fin_d;
        rf.kc = c.max_k;
        CUDA_TRY(stage(ix, 8, st, [&] { return launch_rerank(d, nc, rf, st); }));
    } else {
        // round 1: the first_round * k smallest interval centres of S
        pa.rc_from = nullptr;
        pa.rc_count = n_b;
        CUDA_TRY(stage(ix, 8, st, [&] { return launch_prec_plan(nc, pa, st); }));
        CUDA_TRY(stage(ix, 8, st, [&] { return launch_prec_recheck(d, nc, ra, pa, st); }));
        // round 2: the rest of S whose lower bound reaches the k-th smallest upper bound of round 1
        CUDA_TRY(stage(ix, 4, st, [&] { return launch_sign_filter(d, nc, ss, st); }));
        pa.rc_from = n_b;
        pa.rc_count = n_c;
        CUDA_TRY(stage(ix, 8, st, [&] { return launch_prec_plan(nc, pa, st); }));
        CUDA_TRY(stage(ix, 8, st, [&] { return launch_prec_recheck(d, nc, ra, pa, st); }));
        // exact order: FP32 with its bound, FP64 where the bound cannot decide
        CUDA_TRY(stage(ix, 7, st, [&] { return launch_prec_classify(d, nc, ra, pa, st); }));
        CUDA_TRY(stage(ix, 7, st, [&] { return launch_prec_finalize(d, nc, ra, pa, st); }));
    }
    RerankArgs rb = ra;
    rb.cand = pa.fin_id;
    rb.cdist = pa.fin_d;
    rb.cand_count = pa.n_fin;
    rb.kc = c.max_k;
    CUDA_TRY(stage(ix, 6, st, [&] { return launch_topk(d, nc, rb, st); }));
    return BBC_OK;
}

int search_sign(bbc_index* ix, const float* queries, int64_t nq, int k, int nprobe, int64_t* out_ids,
                float* out_dists, cudaStream_t st, bool host_io) {
    const size_t budget = (size_t)(ix->workspace_mb * 1024.0 * 1024.0);
    SignPlan p{};
    int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(nq, kMaxChunkQueries));
    while (chunk > 1 && sign_layout(ix, sign_uniform_shape(ix, chunk, nprobe, k, host_io), p) > budget)
        chunk = (chunk + 1) / 2;
    const SignShape c = sign_uniform_shape(ix, chunk, nprobe, k, host_io);
    sign_layout(ix, c, p);
    char* ws;
    int rc = get_workspace(ix, st, p.total, &ws);
    if (rc) return rc;
    const int d = ix->dev.d;
    const int64_t cap = ix->cap_for(nprobe);
    const QueryParams qp = uniform_params(nprobe, cap, k, cap);
    for (int64_t q0 = 0; q0 < nq; q0 += chunk) {
        const int64_t nc = std::min(chunk, nq - q0);
        if (host_io) {
            float* dq = reinterpret_cast<float*>(ws + p.off_q);
            int64_t* di = reinterpret_cast<int64_t*>(ws + p.off_ids);
            float* dd = reinterpret_cast<float*>(ws + p.off_dists);
            CUDA_TRY(cudaMemcpyAsync(dq, queries + q0 * d, (size_t)nc * d * 4, cudaMemcpyHostToDevice, st));
            if ((rc = run_sign_chunk(ix, p, c, ws, dq, nc, qp, di, dd, st))) return rc;
            CUDA_TRY(cudaMemcpyAsync(out_ids + q0 * k, di, (size_t)nc * k * 8, cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaMemcpyAsync(out_dists + q0 * k, dd, (size_t)nc * k * 4, cudaMemcpyDeviceToHost, st));
        } else {
            if ((rc = run_sign_chunk(ix, p, c, ws, queries + q0 * d, nc, qp, out_ids + q0 * k, out_dists + q0 * k, st)))
                return rc;
        }
    }
    if (host_io) CUDA_TRY(cudaStreamSynchronize(st));
    return BBC_OK;
}

// Mixed batch (per-query k and nprobe) on a sign-code index: greedy chunks
// that fit the workspace, per-query tables as in the PQ mixed batch.
int search_sign_ex(bbc_index* ix, const float* queries, int64_t nq, const int32_t* k, const int32_t* nprobe,
                   int64_t* out_ids, float* out_dists, cudaStream_t st) {
    const size_t budget = (size_t)(ix->workspace_mb * 1024.0 * 1024.0);
    int64_t out_base = 0;
    for (int64_t q0 = 0; q0 < nq;) {
        SignShape c;
        c.mixed = true;
        int64_t q1 = q0;
        while (q1 < nq) {
            SignShape t = c;
            t.nq += 1; t.sum_probe += nprobe[q1]; t.sum_cap += ix->cap_for(nprobe[q1]); t.sum_k += k[q1];
            t.max_probe = std::max(t.max_probe, nprobe[q1]); t.max_k = std::max(t.max_k, k[q1]);
            SignPlan tp{};
            if (q1 > q0 && (sign_layout(ix, t, tp) > budget || t.nq > kMaxChunkQueries)) break;
            c = t;
            ++q1;
        }
        const int64_t nc = q1 - q0;
        SignPlan p{};
        sign_layout(ix, c, p);
        const size_t n8 = (size_t)nc + 1;
        std::vector<int64_t> tab(n8 * 7, 0);
        int32_t* t_np = reinterpret_cast<int32_t*>(tab.data());
        int32_t* t_k = reinterpret_cast<int32_t*>(tab.data() + n8);
        int64_t* t_kc = tab.data() + 2 * n8;
        int64_t* t_po = tab.data() + 3 * n8;
        int64_t* t_ro = tab.data() + 4 * n8;
        int64_t* t_co = tab.data() + 5 * n8;
        int64_t* t_oo = tab.data() + 6 * n8;
        int64_t maxcap = 0;
        for (int64_t i = 0; i < nc; ++i) {
            const int64_t qq = q0 + i;
            const int64_t cap = ix->cap_for(nprobe[qq]);
            t_np[i] = nprobe[qq];
            t_k[i] = k[qq];
            t_kc[i] = cap;
            t_po[i + 1] = t_po[i] + nprobe[qq];
            t_ro[i + 1] = t_ro[i] + cap;
            t_co[i + 1] = t_co[i] + cap;
            t_oo[i + 1] = t_oo[i] + k[qq];
            maxcap = std::max(maxcap, cap);
        }
        char* ws;
        int rc = get_workspace(ix, st, p.total, &ws);
        if (rc) return rc;
        int64_t* dtab = reinterpret_cast<int64_t*>(ws + p.off_params);
        CUDA_TRY(cudaMemcpyAsync(dtab, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice, st));
        QueryParams qp{};
        qp.nprobe = c.max_probe; qp.kc = maxcap; qp.k = c.max_k; qp.cap = maxcap;
        qp.nprobe_q = reinterpret_cast<const int32_t*>(dtab);
        qp.k_q = reinterpret_cast<const int32_t*>(dtab + n8);
        qp.kc_q = dtab + 2 * n8;
        qp.probe_off = dtab + 3 * n8;
        qp.region_off = dtab + 4 * n8;
        qp.cand_off = dtab + 5 * n8;
        qp.out_off = dtab + 6 * n8;
        rc = run_sign_chunk(ix, p, c, ws, queries + q0 * ix->dev.d, nc, qp, out_ids + out_base, out_dists + out_base, st);
        if (rc) return rc;
        out_base += t_oo[nc];
        q0 = q1;
    }
    return BBC_OK;
}

// Switches Algorithm 4's early re-rank on (building the slot-ordered u8 copy
// and its norms on the device, after waiting for all work on it) or off
// (freeing them).  Cached graphs hold the index's pointers and are dropped.
int set_early_rerank(bbc_index* ix, int on) {
    DeviceGuard g(ix->device);
    const DevIndex& d = ix->dev;
    if (on) {
        if (d.quant != BBC_QUANT_PQ || d.resid || !d.vec_u8 || d.metric != BBC_METRIC_L2 || d.d % 16 || d.d > 256)
            return fail(BBC_ERR_UNSUPPORTED,
                        "early_rerank needs a plain (not residual) L2 PQ index with the exact u8 copy and d a "
                        "multiple of 16 up to 256");
        if (d.bits == 8 ? d.M > 32 : d.M > 64)
            return fail(BBC_ERR_UNSUPPORTED, "early_rerank needs a table of at most 64 KB (pq_m <= 32 at 8 bits)");
    }
    CUDA_TRY(cudaDeviceSynchronize());
    {
        std::lock_guard<std::mutex> lk(ix->graph_mu);
        for (auto& kv : ix->graph_cache) cudaGraphExecDestroy(kv.second.exec);
        ix->graph_cache.clear();
    }
    if (ix->lo_rows) ix->info.device_bytes -= (int64_t)((size_t)ix->nslots * (d.d + 4));
    cudaFree(ix->lo_rows);
    cudaFree(ix->lo_norms);
    ix->lo_rows = nullptr;
    ix->lo_norms = nullptr;
    ix->dev.vec_lo = nullptr;
    ix->dev.vnorm2 = nullptr;
    ix->early_rerank = 0;
    if (!on) return BBC_OK;
    void* r = nullptr;
    void* nrm = nullptr;
    if (cudaMalloc(&r, (size_t)ix->nslots * d.d) != cudaSuccess || cudaMalloc(&nrm, (size_t)ix->nslots * 4) != cudaSuccess) {
        cudaFree(r);
        return fail(BBC_ERR_OOM, "early_rerank copy");
    }
    if (!ix->early_totals) {
        void* t = nullptr;
        if (cudaMalloc(&t, 2 * sizeof(unsigned long long)) != cudaSuccess) {
            cudaFree(r);
            cudaFree(nrm);
            return fail(BBC_ERR_OOM, "early_rerank counters");
        }
        CUDA_TRY(cudaMemset(t, 0, 2 * sizeof(unsigned long long)));
        ix->early_totals = static_cast<unsigned long long*>(t);
    }
    ix->lo_rows = static_cast<uint8_t*>(r);
    ix->lo_norms = static_cast<uint32_t*>(nrm);
    CUDA_TRY(launch_early_copy(d, ix->nslots, ix->lo_rows, ix->lo_norms, 0));
    CUDA_TRY(cudaDeviceSynchronize());
    ix->dev.vec_lo = ix->lo_rows;
    ix->dev.vnorm2 = ix->lo_norms;
    ix->info.device_bytes += (int64_t)((size_t)ix->nslots * (d.d + 4));
    ix->early_rerank = 1;
    return BBC_OK;
}

int pq_only(const bbc_index* ix, const char* what) {
    if (ix && ix->dev.quant != 0) return fail(BBC_ERR_UNSUPPORTED, "%s: not available on a sign-code index", what);
    return BBC_OK;
}

// (Re)builds the low-precision copy for the precision re-rank; 0 drops it.
// Waits for all work on the device first and drops cached graphs, which hold
// the index's device pointers.
int build_precision(bbc_index* ix, int prec) {
    DeviceGuard g(ix->device);
    CUDA_TRY(cudaDeviceSynchronize());
    {
        std::lock_guard<std::mutex> lk(ix->graph_mu);
        for (auto& kv : ix->graph_cache) cudaGraphExecDestroy(kv.second.exec);
        ix->graph_cache.clear();
    }
    const size_t old_es = ix->dev.prec == 1 ? 2 : 1;
    if (ix->lp_rows) ix->info.device_bytes -= (int64_t)((size_t)ix->dev.n * ix->dev.dpad * old_es + (size_t)ix->dev.n * 16);
    cudaFree(ix->lp_rows);
    cudaFree(ix->lp_meta);
    ix->lp_rows = nullptr;
    ix->lp_meta = nullptr;
    ix->dev.vec_lp = nullptr;
    ix->dev.vec_meta = nullptr;
    ix->dev.prec = 0;
    if (prec == 0) return BBC_OK;
    if (!ix->prec_totals) {
        void* t = nullptr;
        cudaError_t e = cudaMalloc(&t, 32);
        if (e != cudaSuccess) return fail(BBC_ERR_OOM, "cudaMalloc(32): %s", cudaGetErrorString(e));
        ix->prec_totals = static_cast<unsigned long long*>(t);
        CUDA_TRY(cudaMemset(t, 0, 32));
    }
    const size_t es = prec == 1 ? 2 : 1;
    const size_t rb = (size_t)ix->dev.n * ix->dev.dpad * es, mb = (size_t)ix->dev.n * sizeof(float4);
    void* rows = nullptr;
    void* meta = nullptr;
    cudaError_t e = cudaMalloc(&rows, rb);
    if (e != cudaSuccess) return fail(BBC_ERR_OOM, "cudaMalloc(%zu) for the low-precision copy: %s", rb, cudaGetErrorString(e));
    e = cudaMalloc(&meta, mb);
    if (e != cudaSuccess) {
        cudaFree(rows);
        return fail(BBC_ERR_OOM, "cudaMalloc(%zu) for the copy metadata: %s", mb, cudaGetErrorString(e));
    }
    ix->lp_rows = rows;
    ix->lp_meta = static_cast<float4*>(meta);
    CUDA_TRY(launch_prec_copy(ix->dev, prec, rows, ix->lp_meta, nullptr));
    CUDA_TRY(cudaDeviceSynchronize());
    ix->dev.vec_lp = rows;
    ix->dev.vec_meta = ix->lp_meta;
    ix->dev.prec = prec;
    ix->info.device_bytes += (int64_t)(rb + mb);
    return BBC_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* bbc_last_error(void) { return g_err.c_str(); }

const char* bbc_version(void) { return "bbc-gb300 0.1 (sm_103a)"; }

int bbc_index_create(const bbc_index_host* h, int device, bbc_index** out) {
    if (!h || !out) return fail(BBC_ERR_ARG, "null argument");
    *out = nullptr;
    if (h->n < 1 || h->n >= (int64_t)0xFFFFFFFFll) return fail(BBC_ERR_ARG, "n=%lld outside [1, 2^32-1)", (long long)h->n);
    if (h->d < 4 || h->d % 4) return fail(BBC_ERR_ARG, "d=%d must be a positive multiple of 4", h->d);
    if (h->nlist < 1) return fail(BBC_ERR_ARG, "nlist must be >= 1");
    if (h->metric != BBC_METRIC_L2 && h->metric != BBC_METRIC_IP) return fail(BBC_ERR_ARG, "bad metric %d", h->metric);
    if (h->pq_m < 1 || h->d % h->pq_m) return fail(BBC_ERR_ARG, "pq_m=%d must divide d=%d", h->pq_m, h->d);
    if (h->residual != 0 && h->residual != 1) return fail(BBC_ERR_ARG, "residual must be 0 or 1");
    if (!scan_supported(h->pq_m, h->pq_bits))
        return fail(BBC_ERR_UNSUPPORTED, "pq_m=%d x %d bits not supported", h->pq_m, h->pq_bits);
    if (!h->centroids || !h->list_offsets || !h->ids || !h->codes || !h->codebooks || !h->vectors)
        return fail(BBC_ERR_ARG, "null array");
    const int64_t n = h->n;
    const int L = h->nlist, d = h->d, M = h->pq_m, bits = h->pq_bits, K = 1 << bits;
    if (h->list_offsets[0] != 0 || h->list_offsets[L] != n) return fail(BBC_ERR_FORMAT, "list_offsets must run from 0 to n");
    int32_t maxlen = 0;
    for (int l = 0; l < L; ++l) {
        int64_t len = h->list_offsets[l + 1] - h->list_offsets[l];
        if (len < 0 || len > (1ll << 30)) return fail(BBC_ERR_FORMAT, "list %d has bad length %lld", l, (long long)len);
        maxlen = std::max<int32_t>(maxlen, (int32_t)len);
    }
    {
        std::vector<uint8_t> seen((size_t)n, 0);
        for (int64_t i = 0; i < n; ++i) {
            int64_t id = h->ids[i];
            if (id < 0 || id >= n || seen[(size_t)id]) return fail(BBC_ERR_FORMAT, "ids are not a permutation of [0, n)");
            seen[(size_t)id] = 1;
        }
    }
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) return fail(BBC_ERR_CUDA, "no CUDA device");
    DeviceGuard g(device);
    if (!g.ok) return fail(BBC_ERR_ARG, "cannot select device %d", device);

    std::unique_ptr<bbc_index> ix(new bbc_index());
    ix->device = device;
    DevIndex& D = ix->dev;
    D.d = d; D.nlist = L; D.metric = h->metric; D.M = M; D.bits = bits; D.K = K; D.dsub = d / M;
    D.code_bytes = M * bits / 8;
    D.cbp = (D.code_bytes + 15) / 16 * 16;
    D.W = lut_row_words(M);
    D.n = n;
    D.dpad = (d + 15) / 16 * 16;
    {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0) sms = 1;
        D.num_sms = sms;
    }

    // block layout
    std::vector<int32_t> list_blk(L), list_len(L);
    int64_t nblocks = 0;
    for (int l = 0; l < L; ++l) {
        list_len[l] = (int32_t)(h->list_offsets[l + 1] - h->list_offsets[l]);
        list_blk[l] = (int32_t)nblocks;
        nblocks += (list_len[l] + 31) / 32;
    }
    if (nblocks >= (1ll << 31) / 32) return fail(BBC_ERR_UNSUPPORTED, "too many blocks");
    ix->nslots = nblocks * 32;
    std::vector<uint8_t> codes((size_t)nblocks * 32 * D.cbp, 0);
    std::vector<uint32_t> ids((size_t)nblocks * 32, kPadId);
    const int cb = D.code_bytes;
    std::vector<uint8_t> row(D.cbp);
    for (int l = 0; l < L; ++l) {
        const int64_t off = h->list_offsets[l];
        for (int32_t p = 0; p < list_len[l]; ++p) {
            const int64_t gb = list_blk[l] + p / 32;
            const int t = p % 32;
            const uint8_t* src = h->codes + (size_t)(off + p) * cb;
            std::fill(row.begin(), row.end(), 0);
            for (int s = 0; s < M; ++s) {
                const int m = (s + t) % M;                       // rotated slot
                int code;
                if (bits == 8) code = src[m];
                else code = (m & 1) ? (src[m >> 1] >> 4) : (src[m >> 1] & 0xF);
                if (bits == 8) row[s] = (uint8_t)code;
                else row[s >> 1] |= (uint8_t)((code & 0xF) << (4 * (s & 1)));
            }
            uint8_t* blk = codes.data() + (size_t)gb * 32 * D.cbp;
            for (int b = 0; b < D.cbp; ++b) blk[(b / 16) * 512 + t * 16 + (b % 16)] = row[b];
            ids[(size_t)gb * 32 + t] = (uint32_t)h->ids[off + p];
        }
    }
    // centroid norms
    std::vector<float> cnorm(L);
    double cmax = 0.0;
    for (int l = 0; l < L; ++l) {
        double s = 0.0;
        for (int i = 0; i < d; ++i) s += (double)h->centroids[(size_t)l * d + i] * h->centroids[(size_t)l * d + i];
        cnorm[l] = (float)s;
        cmax = std::max(cmax, std::sqrt(s));
    }
    D.cmax = (float)(cmax * (1.0 + 1e-6));
    // exact u8 copy
    bool u8 = (d % 16) == 0;
    for (int64_t i = 0; u8 && i < n * (int64_t)d; ++i) {
        float v = h->vectors[i];
        if (!(v >= 0.f && v <= 255.f) || v != std::floor(v)) u8 = false;
    }
    int rc;
    float* dc; float* dcn; int32_t* dlb; int32_t* dll; uint8_t* dcode; uint32_t* did; float* dbook; float* dvec;
    unsigned int* dstat;
    if ((rc = upload(ix.get(), h->centroids, (size_t)L * d, &dc))) return rc;
    if ((rc = upload(ix.get(), cnorm.data(), (size_t)L, &dcn))) return rc;
    if ((rc = upload(ix.get(), list_blk.data(), (size_t)L, &dlb))) return rc;
    if ((rc = upload(ix.get(), list_len.data(), (size_t)L, &dll))) return rc;
    if ((rc = upload(ix.get(), codes.data(), codes.size(), &dcode))) return rc;
    if ((rc = upload(ix.get(), ids.data(), ids.size(), &did))) return rc;
    if ((rc = upload(ix.get(), h->codebooks, (size_t)M * K * (d / M), &dbook))) return rc;
    if ((rc = upload(ix.get(), h->vectors, (size_t)n * d, &dvec))) return rc;
    unsigned int zero = 0;
    if ((rc = upload(ix.get(), &zero, 1, &dstat))) return rc;
    // tensor-core probe operand: [c_hi | c_lo | c_hi | 0-pad] in BF16, K padded to 64
    D.kp = (3 * d + 63) / 64 * 64;
    {
        std::vector<uint16_t> b3((size_t)L * D.kp, 0);
        for (int l = 0; l < L; ++l) {
            uint16_t* r = b3.data() + (size_t)l * D.kp;
            for (int i = 0; i < d; ++i) {
                const float x = h->centroids[(size_t)l * d + i];
                const uint16_t hi = f32_to_bf16(x);
                const uint16_t lo = f32_to_bf16(x - bf16_to_f32(hi));
                r[i] = hi;
                r[d + i] = lo;
                r[2 * d + i] = hi;
            }
        }
        uint16_t* db3;
        if ((rc = upload(ix.get(), b3.data(), b3.size(), &db3))) return rc;
        D.cent_b3 = db3;
    }
    D.centroids = dc; D.cnorm = dcn; D.list_blk = dlb; D.list_len = dll; D.codes = dcode; D.ids = did;
    D.books = dbook; D.vectors = dvec; D.status = dstat; D.vec_u8 = nullptr;
    if (h->residual) {
        // residual IVF-PQ: V_o per code slot and ||c_l||^2 in FP32, computed on the device from the
        // canonical code rows (uploaded for the build only)
        std::vector<float> zs((size_t)ix->nslots, 0.f), zl((size_t)L, 0.f);
        float* drv;
        float* dcn2;
        if ((rc = upload(ix.get(), zs.data(), zs.size(), &drv))) return rc;
        if ((rc = upload(ix.get(), zl.data(), zl.size(), &dcn2))) return rc;
        D.resid = 1;
        D.rv = drv;
        D.rcn2 = dcn2;
        void* canon = nullptr;
        void* offs = nullptr;
        if (cudaMalloc(&canon, std::max<size_t>((size_t)n * cb, 16)) != cudaSuccess ||
            cudaMalloc(&offs, (size_t)(L + 1) * 8) != cudaSuccess) {
            cudaFree(canon);
            return fail(BBC_ERR_OOM, "residual build scratch");
        }
        std::unique_ptr<void, cudaError_t (*)(void*)> fc(canon, cudaFree), fo(offs, cudaFree);
        CUDA_TRY(cudaMemcpy(canon, h->codes, (size_t)n * cb, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(offs, h->list_offsets, (size_t)(L + 1) * 8, cudaMemcpyHostToDevice));
        CUDA_TRY(launch_resid_v(D, static_cast<const uint8_t*>(canon), static_cast<const int64_t*>(offs), drv, dcn2,
                                ix->nslots, 0));
        CUDA_TRY(cudaDeviceSynchronize());
    }
    if (u8) {
        std::vector<uint8_t> v8((size_t)n * d);
        for (size_t i = 0; i < v8.size(); ++i) v8[i] = (uint8_t)h->vectors[i];
        uint8_t* dv8;
        if ((rc = upload(ix.get(), v8.data(), v8.size(), &dv8))) return rc;
        D.vec_u8 = dv8;
    }
    // region capacity per query: the nprobe longest lists
    std::vector<int64_t> lens(list_len.begin(), list_len.end());
    std::sort(lens.begin(), lens.end(), std::greater<int64_t>());
    ix->cap_prefix.assign(L + 1, 0);
    for (int l = 0; l < L; ++l) ix->cap_prefix[l + 1] = ix->cap_prefix[l] + lens[l];

    bbc_index_info_t& I = ix->info;
    I.n = n; I.d = d; I.nlist = L; I.metric = h->metric; I.pq_m = M; I.pq_bits = bits;
    I.max_list_len = maxlen; I.vectors_u8_exact = u8 ? 1 : 0; I.device = device;
    I.quantizer = h->residual ? BBC_QUANT_PQ_RESIDUAL : BBC_QUANT_PQ;
    *out = ix.release();
    return BBC_OK;
}

int bbc_index_create_sign(const bbc_sign_host* h, int device, bbc_index** out) {
    if (!h || !out) return fail(BBC_ERR_ARG, "null argument");
    *out = nullptr;
    if (h->n < 1 || h->n >= (int64_t)0xFFFFFFFFll) return fail(BBC_ERR_ARG, "n=%lld outside [1, 2^32-1)", (long long)h->n);
    if (h->metric != BBC_METRIC_L2) return fail(BBC_ERR_UNSUPPORTED, "sign codes: only the L2 metric is supported");
    if (h->d < 32 || h->d % 32 || h->d > 2048) return fail(BBC_ERR_UNSUPPORTED, "sign codes: d=%d must be a multiple of 32 in [32, 2048]", h->d);
    if (h->nlist < 1) return fail(BBC_ERR_ARG, "nlist must be >= 1");
    if (!h->centroids || !h->list_offsets || !h->ids || !h->rotation || !h->vectors) return fail(BBC_ERR_ARG, "null array");
    const int64_t n = h->n;
    const int L = h->nlist, d = h->d, W = d / 32;
    if (h->list_offsets[0] != 0 || h->list_offsets[L] != n) return fail(BBC_ERR_FORMAT, "list_offsets must run from 0 to n");
    int32_t maxlen = 0;
    for (int l = 0; l < L; ++l) {
        const int64_t len = h->list_offsets[l + 1] - h->list_offsets[l];
        if (len < 0 || len > (1ll << 30)) return fail(BBC_ERR_FORMAT, "list %d has bad length %lld", l, (long long)len);
        maxlen = std::max<int32_t>(maxlen, (int32_t)len);
    }
    {
        std::vector<uint8_t> seen((size_t)n, 0);
        for (int64_t i = 0; i < n; ++i) {
            const int64_t id = h->ids[i];
            if (id < 0 || id >= n || seen[(size_t)id]) return fail(BBC_ERR_FORMAT, "ids are not a permutation of [0, n)");
            seen[(size_t)id] = 1;
        }
    }
    DeviceGuard g(device);
    if (!g.ok) return fail(BBC_ERR_ARG, "cannot select device %d", device);
    std::unique_ptr<bbc_index> ix(new bbc_index());
    ix->device = device;
    DevIndex& D = ix->dev;
    D.d = d; D.nlist = L; D.metric = BBC_METRIC_L2; D.M = 0; D.bits = 0; D.K = 0; D.dsub = 0;
    D.n = n; D.dpad = (d + 15) / 16 * 16; D.quant = BBC_QUANT_SIGN;
    {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0) sms = 1;
        D.num_sms = sms;
    }
    // 32-slot block layout shared with the PQ codes
    std::vector<int32_t> list_blk(L), list_len(L);
    int64_t nblocks = 0;
    for (int l = 0; l < L; ++l) {
        list_len[l] = (int32_t)(h->list_offsets[l + 1] - h->list_offsets[l]);
        list_blk[l] = (int32_t)nblocks;
        nblocks += (list_len[l] + 31) / 32;
    }
    if (nblocks >= (1ll << 31) / 32) return fail(BBC_ERR_UNSUPPORTED, "too many blocks");
    const int64_t nslots = nblocks * 32;
    std::vector<uint32_t> ids((size_t)nslots, kPadId);
    std::vector<int64_t> rows((size_t)nslots, -1);
    std::vector<int32_t> slot_list((size_t)nslots, 0);
    for (int l = 0; l < L; ++l) {
        for (int32_t p = 0; p < list_len[l]; ++p) {
            const int64_t slot = (int64_t)list_blk[l] * 32 + p;
            const int64_t id = h->ids[h->list_offsets[l] + p];
            ids[(size_t)slot] = (uint32_t)id;
            rows[(size_t)slot] = id;
            slot_list[(size_t)slot] = l;
        }
    }
    std::vector<float> cnorm(L);
    double cmax = 0.0;
    for (int l = 0; l < L; ++l) {
        double s2 = 0.0;
        for (int i = 0; i < d; ++i) s2 += (double)h->centroids[(size_t)l * d + i] * h->centroids[(size_t)l * d + i];
        cnorm[l] = (float)s2;
        cmax = std::max(cmax, std::sqrt(s2));
    }
    D.cmax = (float)(cmax * (1.0 + 1e-6));
    int rc;
    float *dc, *dcn, *dvec, *drot;
    int32_t *dlb, *dll, *dsl;
    uint32_t* did;
    int64_t* drows;
    unsigned int* dstat;
    if ((rc = upload(ix.get(), h->centroids, (size_t)L * d, &dc))) return rc;
    if ((rc = upload(ix.get(), cnorm.data(), (size_t)L, &dcn))) return rc;
    if ((rc = upload(ix.get(), list_blk.data(), (size_t)L, &dlb))) return rc;
    if ((rc = upload(ix.get(), list_len.data(), (size_t)L, &dll))) return rc;
    if ((rc = upload(ix.get(), ids.data(), ids.size(), &did))) return rc;
    if ((rc = upload(ix.get(), h->vectors, (size_t)n * d, &dvec))) return rc;
    if ((rc = upload(ix.get(), h->rotation, (size_t)d * d, &drot))) return rc;
    unsigned int zero = 0;
    if ((rc = upload(ix.get(), &zero, 1, &dstat))) return rc;
    D.kp = (3 * d + 63) / 64 * 64;
    {
        std::vector<uint16_t> b3((size_t)L * D.kp, 0);
        for (int l = 0; l < L; ++l) {
            uint16_t* r = b3.data() + (size_t)l * D.kp;
            for (int i = 0; i < d; ++i) {
                const float x = h->centroids[(size_t)l * d + i];
                const uint16_t hi = f32_to_bf16(x);
                r[i] = hi;
                r[d + i] = f32_to_bf16(x - bf16_to_f32(hi));
                r[2 * d + i] = hi;
            }
        }
        uint16_t* db3;
        if ((rc = upload(ix.get(), b3.data(), b3.size(), &db3))) return rc;
        D.cent_b3 = db3;
    }
    D.centroids = dc; D.cnorm = dcn; D.list_blk = dlb; D.list_len = dll; D.ids = did; D.vectors = dvec;
    D.status = dstat; D.rot = drot; D.codes = nullptr; D.books = nullptr; D.vec_u8 = nullptr;
    // P c_l (FP64) and ||P P^T - I||_F (equal to ||P^T P - I||_F for a square P)
    double* dcrot;
    {
        void* t = nullptr;
        if (cudaMalloc(&t, (size_t)L * d * 8) != cudaSuccess) return fail(BBC_ERR_OOM, "cudaMalloc for P c_l");
        ix->owned.push_back(t);
        ix->info.device_bytes += (int64_t)L * d * 8;
        dcrot = static_cast<double*>(t);
    }
    CUDA_TRY(launch_rotate_f64(dc, nullptr, nullptr, nullptr, drot, L, d, dcrot, nullptr));
    {
        double* dpp = nullptr;
        if (cudaMalloc(&dpp, (size_t)d * d * 8) != cudaSuccess) return fail(BBC_ERR_OOM, "cudaMalloc for P P^T");
        cudaError_t e = launch_rotate_f64(drot, nullptr, nullptr, nullptr, drot, d, d, dpp, nullptr);
        std::vector<double> pp((size_t)d * d);
        if (e == cudaSuccess) e = cudaMemcpy(pp.data(), dpp, pp.size() * 8, cudaMemcpyDeviceToHost);
        cudaFree(dpp);
        if (e != cudaSuccess) return fail(BBC_ERR_CUDA, "P P^T: %s", cudaGetErrorString(e));
        double f = 0.0;
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                const double v = pp[(size_t)i * d + j] - (i == j ? 1.0 : 0.0);
                f += v * v;
            }
        D.eps_p = std::sqrt(f) * (1.0 + 1e-6) + 1e-15;
    }
    // codes and factors, a chunk of slots at a time through the FP64 rotation
    uint32_t* dsgn;
    float4* dfac;
    {
        void* t = nullptr;
        if (cudaMalloc(&t, (size_t)nslots * W * 4) != cudaSuccess) return fail(BBC_ERR_OOM, "cudaMalloc for sign codes");
        ix->owned.push_back(t);
        dsgn = static_cast<uint32_t*>(t);
        if (cudaMalloc(&t, (size_t)nslots * 16) != cudaSuccess) return fail(BBC_ERR_OOM, "cudaMalloc for factors");
        ix->owned.push_back(t);
        dfac = static_cast<float4*>(t);
        ix->info.device_bytes += (int64_t)nslots * (W * 4 + 16);
    }
    {
        void *t1 = nullptr, *t2 = nullptr, *t3 = nullptr;
        const int64_t chunk = 65536;
        if (cudaMalloc(&t1, (size_t)nslots * 8) != cudaSuccess || cudaMalloc(&t2, (size_t)nslots * 4) != cudaSuccess ||
            cudaMalloc(&t3, (size_t)chunk * d * 8) != cudaSuccess) {
            cudaFree(t1); cudaFree(t2); cudaFree(t3);
            return fail(BBC_ERR_OOM, "cudaMalloc for the sign encoding scratch");
        }
        drows = static_cast<int64_t*>(t1);
        dsl = static_cast<int32_t*>(t2);
        double* R = static_cast<double*>(t3);
        cudaError_t e = cudaMemcpy(drows, rows.data(), (size_t)nslots * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(dsl, slot_list.data(), (size_t)nslots * 4, cudaMemcpyHostToDevice);
        for (int64_t s0 = 0; e == cudaSuccess && s0 < nslots; s0 += chunk) {
            const int64_t m = std::min(chunk, nslots - s0);
            e = launch_rotate_f64(dvec, drows + s0, dsl + s0, dc, drot, m, d, R, nullptr);
            if (e == cudaSuccess) e = launch_sign_factors(R, s0, m, d, drows, dsl, dvec, dc, dsgn, dfac, nullptr);
        }
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        cudaFree(t1); cudaFree(t2); cudaFree(t3);
        if (e != cudaSuccess) return fail(BBC_ERR_CUDA, "sign encoding: %s", cudaGetErrorString(e));
    }
    D.sgn = dsgn; D.sfac = dfac; D.crot = dcrot;
    for (unsigned long long** tp : {&ix->prec_totals, &ix->sign_totals}) {
        void* t = nullptr;
        if (cudaMalloc(&t, 32) != cudaSuccess) return fail(BBC_ERR_OOM, "cudaMalloc(32)");
        *tp = static_cast<unsigned long long*>(t);
        CUDA_TRY(cudaMemset(t, 0, 32));
    }
    std::vector<int64_t> lens(list_len.begin(), list_len.end());
    std::sort(lens.begin(), lens.end(), std::greater<int64_t>());
    ix->cap_prefix.assign(L + 1, 0);
    for (int l = 0; l < L; ++l) ix->cap_prefix[l + 1] = ix->cap_prefix[l] + lens[l];
    bbc_index_info_t& I = ix->info;
    I.n = n; I.d = d; I.nlist = L; I.metric = BBC_METRIC_L2; I.pq_m = 0; I.pq_bits = 0;
    I.max_list_len = maxlen; I.vectors_u8_exact = 0; I.device = device; I.quantizer = BBC_QUANT_SIGN;
    *out = ix.release();
    return BBC_OK;
}

int bbc_index_load(const char* path, int device, bbc_index** out) {
    if (!path || !out) return fail(BBC_ERR_ARG, "null argument");
    FILE* f = fopen(path, "rb");
    if (!f) return fail(BBC_ERR_IO, "cannot open %s", path);
    std::unique_ptr<FILE, int (*)(FILE*)> fc(f, fclose);
    unsigned char hdr[64];
    if (fread(hdr, 1, 64, f) != 64) return fail(BBC_ERR_FORMAT, "short header");
    if (memcmp(hdr, "BBCIDX01", 8) != 0) return fail(BBC_ERR_FORMAT, "bad magic");
    uint32_t version, quant, metric, d, nlist, pq_m, pq_bits;
    uint64_t n;
    memcpy(&version, hdr + 8, 4); memcpy(&quant, hdr + 12, 4); memcpy(&metric, hdr + 16, 4);
    memcpy(&d, hdr + 20, 4); memcpy(&n, hdr + 24, 8); memcpy(&nlist, hdr + 32, 4);
    memcpy(&pq_m, hdr + 36, 4); memcpy(&pq_bits, hdr + 40, 4);
    if (version != 1) return fail(BBC_ERR_FORMAT, "unsupported version %u", version);
    if (quant != BBC_QUANT_PQ && quant != BBC_QUANT_SIGN && quant != BBC_QUANT_PQ_RESIDUAL)
        return fail(BBC_ERR_FORMAT, "unknown quantizer %u", quant);
    if (d == 0 || d > 65536 || nlist == 0 || nlist > (1u << 24) || n == 0 || n >= 0xFFFFFFFFull)
        return fail(BBC_ERR_FORMAT, "header fields out of range");
    if (quant != BBC_QUANT_SIGN && (pq_m == 0 || pq_m > d || (pq_bits != 4 && pq_bits != 8)))
        return fail(BBC_ERR_FORMAT, "PQ header fields out of range");
    auto rd = [&](void* dst, size_t bytes) -> bool {
        long pos = ftell(f);
        long pad = (64 - pos % 64) % 64;
        if (pad && fseek(f, pad, SEEK_CUR) != 0) return false;
        return fread(dst, 1, bytes, f) == bytes;
    };
    if (quant == BBC_QUANT_SIGN) {
        // centroids, list offsets, ids, rotation P [d][d], vectors
        std::vector<float> cent((size_t)nlist * d);
        std::vector<int64_t> offs(nlist + 1);
        std::vector<int64_t> ids(n);
        std::vector<float> rot((size_t)d * d);
        std::vector<float> vecs(n * d);
        if (!rd(cent.data(), cent.size() * 4) || !rd(offs.data(), offs.size() * 8) || !rd(ids.data(), ids.size() * 8) ||
            !rd(rot.data(), rot.size() * 4) || !rd(vecs.data(), vecs.size() * 4))
            return fail(BBC_ERR_FORMAT, "truncated index file");
        bbc_sign_host h{(int64_t)n, (int32_t)d, (int32_t)nlist, (int32_t)metric, cent.data(), offs.data(), ids.data(),
                        rot.data(), vecs.data()};
        return bbc_index_create_sign(&h, device, out);
    }
    const size_t cb = (size_t)pq_m * pq_bits / 8;
    std::vector<float> cent((size_t)nlist * d);
    std::vector<int64_t> offs(nlist + 1);
    std::vector<int64_t> ids(n);
    std::vector<uint8_t> codes(n * cb);
    std::vector<float> books((size_t)pq_m * (1u << pq_bits) * (d / pq_m));
    std::vector<float> vecs(n * d);
    if (!rd(cent.data(), cent.size() * 4) || !rd(offs.data(), offs.size() * 8) || !rd(ids.data(), ids.size() * 8) ||
        !rd(codes.data(), codes.size()) || !rd(books.data(), books.size() * 4) || !rd(vecs.data(), vecs.size() * 4))
        return fail(BBC_ERR_FORMAT, "truncated index file");
    bbc_index_host h{(int64_t)n, (int32_t)d, (int32_t)nlist, (int32_t)metric, (int32_t)pq_m, (int32_t)pq_bits,
                     cent.data(), offs.data(), ids.data(), codes.data(), books.data(), vecs.data(),
                     quant == BBC_QUANT_PQ_RESIDUAL ? 1 : 0};
    return bbc_index_create(&h, device, out);
}

int bbc_index_free(bbc_index* ix) {
    if (!ix) return fail(BBC_ERR_ARG, "null index");
    delete ix;
    return BBC_OK;
}

int bbc_index_info(const bbc_index* ix, bbc_index_info_t* out) {
    if (!ix || !out) return fail(BBC_ERR_ARG, "null argument");
    *out = ix->info;
    return BBC_OK;
}

int bbc_set_param(bbc_index* ix, const char* key, double v) {
    if (!ix || !key) return fail(BBC_ERR_ARG, "null argument");
    std::string k(key);
    if (k == "kc_ratio") {
        if (!(v >= 1.0 && v <= 1e6)) return fail(BBC_ERR_ARG, "kc_ratio must be >= 1");
        ix->kc_ratio = v;
    } else if (k == "buckets") {
        if (!(v >= 2 && v <= 256) || v != std::floor(v)) return fail(BBC_ERR_ARG, "buckets must be an integer in [2, 256]");
        ix->buckets = (int)v;
    } else if (k == "sample_lists") {
        if (!(v >= 1 && v <= 1e6) || v != std::floor(v)) return fail(BBC_ERR_ARG, "sample_lists must be a positive integer");
        ix->sample_lists = (int)v;
    } else if (k == "rerank") {
        if (v != 0 && v != 1) return fail(BBC_ERR_ARG, "rerank must be 0 (fp32) or 1 (u8)");
        if (v == 1 && !ix->dev.vec_u8) return fail(BBC_ERR_ARG, "no exact u8 copy for this index");
        ix->rerank_u8 = (int)v;
    } else if (k == "workspace_mb") {
        if (!(v >= 1)) return fail(BBC_ERR_ARG, "workspace_mb must be >= 1");
        ix->workspace_mb = v;
    } else if (k == "graphs") {
        if (v != 0 && v != 1) return fail(BBC_ERR_ARG, "graphs must be 0 or 1");
        ix->graphs = (int)v;
    } else if (k == "split") {
        if (!(v >= 0 && v <= 65536) || v != std::floor(v)) return fail(BBC_ERR_ARG, "split must be 0 (auto), 1 or a part count");
        ix->split = (int)v;
    } else if (k == "probe_gemm") {
        if (v != 0 && v != 1) return fail(BBC_ERR_ARG, "probe_gemm must be 0 (FP32 SIMT) or 1 (tensor cores)");
        ix->probe_gemm = (int)v;
    } else if (k == "bound_scale") {
        if (!(v > 0.0 && v <= 1.0)) return fail(BBC_ERR_ARG, "bound_scale must be in (0, 1]");
        ix->bound_scale = (float)v;
    } else if (k == "estimator") {
        if (v != 0 && v != 1) return fail(BBC_ERR_ARG, "estimator must be 0 (hard bounds) or 1 (RaBitQ)");
        ix->estimator = (int)v;
    } else if (k == "first_round") {
        if (!(v >= 1.0 && v <= 64.0)) return fail(BBC_ERR_ARG, "first_round must be in [1, 64]");
        ix->first_round = (float)v;
    } else if (k == "epsilon0") {
        if (!(v > 0.0 && v <= 100.0)) return fail(BBC_ERR_ARG, "epsilon0 must be in (0, 100]");
        ix->eps0 = (float)v;
    } else if (k == "precision") {
        if (v != 0 && v != 1 && v != 2)
            return fail(BBC_ERR_ARG, "precision must be 0 (FP32 re-rank), 1 (BF16 copy) or 2 (FP8-E4M3 copy)");
        return build_precision(ix, (int)v);
    } else if (k == "profile") {
        if (v != 0 && v != 1) return fail(BBC_ERR_ARG, "profile must be 0 or 1");
        ix->profile = (int)v;
    } else if (k == "early_rerank") {
        if (v != 0 && v != 1) return fail(BBC_ERR_ARG, "early_rerank must be 0 or 1");
        return set_early_rerank(ix, (int)v);
    } else if (k == "collector") {
        if (v != 0 && v != 1 && v != 2) return fail(BBC_ERR_ARG, "collector must be 0 (result buffer), 1 (lazy) or 2 (heap)");
        ix->collector = (int)v;
    } else if (k == "pair") {
        if (v != 0 && v != 1) return fail(BBC_ERR_ARG, "pair must be 0 (one query per CTA) or 1 (two)");
        ix->pair = (int)v;
    } else if (k == "lut_levels") {
        if (!(v >= 1 && v <= 65535) || v != std::floor(v)) return fail(BBC_ERR_ARG, "lut_levels must be an integer in [1, 65535]");
        if (ix->scan_tc && v > 2047) return fail(BBC_ERR_ARG, "lut_levels must be <= 2047 while scan_tc is 1");
        ix->lut_levels = (int)v;
    } else if (k == "scan_tc") {
        if (v != 0 && v != 1) return fail(BBC_ERR_ARG, "scan_tc must be 0 or 1");
        if (v == 1 && ix->dev.quant != 0) return fail(BBC_ERR_UNSUPPORTED, "scan_tc: PQ indexes only");
        if (v == 1 && !scan_tc_supported(ix->dev, 2))
            return fail(BBC_ERR_UNSUPPORTED, "scan_tc: needs plain 4-bit PQ codes with M = 32, 64 or 128");
        ix->scan_tc = (int)v;
        // the tensor cores take tables whose entries FP16 holds exactly
        if (v == 1 && ix->lut_levels > 2047) ix->lut_levels = 2047;
    } else if (k == "rerank_fused") {
        if (v != 0 && v != 1) return fail(BBC_ERR_ARG, "rerank_fused must be 0 or 1");
        ix->rerank_fused = (int)v;
    } else if (k == "region_cap") {
        if (!(v >= 0 && v <= 9.0e15) || v != std::floor(v)) return fail(BBC_ERR_ARG, "region_cap must be 0 (automatic) or a positive integer");
        ix->region_cap = (int64_t)v;
    } else {
        return fail(BBC_ERR_ARG, "unknown parameter '%s'", key);
    }
    return BBC_OK;
}

int bbc_get_param(const bbc_index* ix, const char* key, double* v) {
    if (!ix || !key || !v) return fail(BBC_ERR_ARG, "null argument");
    std::string k(key);
    if (k == "kc_ratio") *v = ix->kc_ratio;
    else if (k == "buckets") *v = ix->buckets;
    else if (k == "sample_lists") *v = ix->sample_lists;
    else if (k == "rerank") *v = (ix->rerank_u8 && ix->dev.vec_u8) ? 1 : 0;
    else if (k == "workspace_mb") *v = ix->workspace_mb;
    else if (k == "profile") *v = ix->profile;
    else if (k == "probe_gemm") *v = ix->probe_gemm;
    else if (k == "split") *v = ix->split;
    else if (k == "graphs") *v = ix->graphs;
    else if (k == "precision") *v = ix->dev.prec;
    else if (k == "bound_scale") *v = ix->bound_scale;
    else if (k == "estimator") *v = ix->estimator;
    else if (k == "epsilon0") *v = ix->eps0;
    else if (k == "first_round") *v = ix->first_round;
    else if (k == "region_cap") *v = (double)ix->region_cap;
    else if (k == "pair") *v = ix->pair;
    else if (k == "collector") *v = ix->collector;
    else if (k == "early_rerank") *v = ix->early_rerank;
    else if (k == "lut_levels") *v = ix->lut_levels;
    else if (k == "scan_tc") *v = ix->scan_tc;
    else if (k == "rerank_fused") *v = ix->rerank_fused;
    else return fail(BBC_ERR_ARG, "unknown parameter '%s'", key);
    return BBC_OK;
}

int bbc_search(bbc_index* ix, const float* queries, int64_t nq, int32_t k, int32_t nprobe, int64_t* out_ids,
               float* out_dists, void* stream) {
    int rc = check_search_args(ix, queries, nq, k, nprobe, out_ids, out_dists);
    if (rc) return rc;
    const int64_t kc = kc_for(ix, k);
    if (kc > (int64_t)0x7FFFFFFF) return fail(BBC_ERR_ARG, "K_c too large");
    if (nq == 0) return BBC_OK;
    DeviceGuard g(ix->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (ix->dev.quant == BBC_QUANT_SIGN) return search_sign(ix, queries, nq, k, nprobe, out_ids, out_dists, st, false);
    Plan p = make_plan(ix, nq, nprobe, kc, k, false);
    char* ws;
    if ((rc = get_workspace(ix, st, p.total, &ws))) return rc;
    auto run_all = [&]() -> int {
        for (int64_t q0 = 0; q0 < nq; q0 += p.chunk) {
            const int64_t nc = std::min(p.chunk, nq - q0);
            int r = run_chunk(ix, p, ws, queries + q0 * ix->dev.d, nc, out_ids + q0 * k, out_dists + q0 * k, st, 9);
            if (r) return r;
        }
        return BBC_OK;
    };
    if (!ix->graphs || st == nullptr) return run_all();
    // CUDA graph of the whole launch sequence for this call shape
    bbc_index::GraphKey key{queries, nq, k, nprobe, out_ids, out_dists, st, ix->kc_ratio, ix->buckets,
                            ix->sample_lists, ix->split, ix->probe_gemm, ix->rerank_u8, ix->dev.prec,
                            ix->region_cap, ix->pair, ix->collector, ix->early_rerank, ix->lut_levels,
                            ix->scan_tc, ix->rerank_fused};
    std::lock_guard<std::mutex> lk(ix->graph_mu);
    auto it = ix->graph_cache.find(key);
    if (it == ix->graph_cache.end()) {
        const int64_t before = ix->launches;
        CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
        ix->capturing = true;
        rc = run_all();
        ix->capturing = false;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(st, &graph);
        if (rc || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return rc ? rc : fail(BBC_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        }
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(BBC_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
        if (ix->graph_cache.size() >= 32) {
            cudaGraphExecDestroy(ix->graph_cache.begin()->second.exec);
            ix->graph_cache.erase(ix->graph_cache.begin());
        }
        {
            std::lock_guard<std::mutex> pl(ix->prof_mu);
            const int64_t n = ix->launches - before;
            ix->launches = before;
            it = ix->graph_cache.emplace(key, bbc_index::GraphEntry{exec, n}).first;
        }
    }
    CUDA_TRY(cudaGraphLaunch(it->second.exec, st));
    {
        std::lock_guard<std::mutex> pl(ix->prof_mu);
        ix->launches += it->second.launches;
    }
    return BBC_OK;
}

int bbc_search_ex(bbc_index* ix, const float* queries, int64_t nq, const int32_t* k, const int32_t* nprobe,
                  int64_t* out_ids, float* out_dists, void* stream) {
    if (!ix) return fail(BBC_ERR_ARG, "null index");

    if (nq < 0) return fail(BBC_ERR_ARG, "nq < 0");
    if (nq == 0) return BBC_OK;
    if (!queries || !k || !nprobe || !out_ids || !out_dists) return fail(BBC_ERR_ARG, "null buffer");
    for (int64_t q = 0; q < nq; ++q) {
        if (k[q] < 1) return fail(BBC_ERR_ARG, "k[%lld] = %d must be >= 1", (long long)q, k[q]);
        if (nprobe[q] < 1 || nprobe[q] > ix->dev.nlist)
            return fail(BBC_ERR_ARG, "nprobe[%lld] = %d outside [1, %d]", (long long)q, nprobe[q], ix->dev.nlist);
        if (nprobe[q] > 2048) return fail(BBC_ERR_UNSUPPORTED, "nprobe %d > 2048", nprobe[q]);
    }
    DeviceGuard g(ix->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (ix->dev.quant == BBC_QUANT_SIGN) return search_sign_ex(ix, queries, nq, k, nprobe, out_ids, out_dists, st);
    const size_t budget = (size_t)(ix->workspace_mb * 1024.0 * 1024.0);
    int64_t out_base = 0;
    for (int64_t q0 = 0; q0 < nq;) {
        // greedy chunk: add queries while the workspace fits
        ChunkShape sh;
        sh.mixed = true;
        Plan p{};
        int64_t q1 = q0;
        while (q1 < nq) {
            ChunkShape t = sh;
            const int64_t kc = kc_for(ix, k[q1]);
            t.nq += 1; t.sum_probe += nprobe[q1]; t.sum_cap += ix->cap_for(nprobe[q1]); t.sum_kc += kc;
            t.sum_k += k[q1]; t.max_probe = std::max(t.max_probe, nprobe[q1]); t.max_kc = std::max(t.max_kc, kc);
            Plan tp{};
            if (q1 > q0 && (layout(ix, t, tp) > budget || t.nq > kMaxChunkQueries)) break;
            sh = t;
            ++q1;
        }
        const int64_t nc = q1 - q0;
        layout(ix, sh, p);
        int maxk = 0;
        int64_t maxcap = 0;
        // per-query tables: nprobe i32, k i32, kc i64, then four i64 offset arrays of nc + 1
        const size_t n8 = (size_t)nc + 1;
        std::vector<int64_t> tab(n8 * 7, 0);
        int32_t* t_np = reinterpret_cast<int32_t*>(tab.data());
        int32_t* t_k = reinterpret_cast<int32_t*>(tab.data() + n8);
        int64_t* t_kc = tab.data() + 2 * n8;
        int64_t* t_po = tab.data() + 3 * n8;
        int64_t* t_ro = tab.data() + 4 * n8;
        int64_t* t_co = tab.data() + 5 * n8;
        int64_t* t_oo = tab.data() + 6 * n8;
        for (int64_t i = 0; i < nc; ++i) {
            const int64_t q = q0 + i;
            t_np[i] = nprobe[q];
            t_k[i] = k[q];
            t_kc[i] = kc_for(ix, k[q]);
            t_po[i + 1] = t_po[i] + nprobe[q];
            t_ro[i + 1] = t_ro[i] + ix->cap_for(nprobe[q]);
            t_co[i + 1] = t_co[i] + t_kc[i];
            t_oo[i + 1] = t_oo[i] + k[q];
            maxk = std::max(maxk, k[q]);
            maxcap = std::max(maxcap, ix->cap_for(nprobe[q]));
        }
        char* ws;
        int rc = get_workspace(ix, st, p.total, &ws);
        if (rc) return rc;
        int64_t* dtab = reinterpret_cast<int64_t*>(ws + p.off_params);
        CUDA_TRY(cudaMemcpyAsync(dtab, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice, st));
        QueryParams qp{};
        qp.nprobe = sh.max_probe; qp.kc = sh.max_kc; qp.k = maxk; qp.cap = maxcap;
        qp.nprobe_q = reinterpret_cast<const int32_t*>(dtab);
        qp.k_q = reinterpret_cast<const int32_t*>(dtab + n8);
        qp.kc_q = dtab + 2 * n8;
        qp.probe_off = dtab + 3 * n8;
        qp.region_off = dtab + 4 * n8;
        qp.cand_off = dtab + 5 * n8;
        qp.out_off = dtab + 6 * n8;
        p.nprobe = sh.max_probe;
        p.kc = sh.max_kc;
        p.chunk_slots = sh.sum_kc;
        p.chunk_probe = sh.sum_probe;
        p.k = maxk;
        p.cap = maxcap;
        rc = run_chunk(ix, p, ws, queries + q0 * ix->dev.d, nc, out_ids + out_base, out_dists + out_base, st, 9,
                       nullptr, nullptr, nullptr, nullptr, nullptr, &qp);
        if (rc) return rc;
        out_base += t_oo[nc];
        q0 = q1;
    }
    return BBC_OK;
}

int bbc_search_host(bbc_index* ix, const float* queries, int64_t nq, int32_t k, int32_t nprobe, int64_t* out_ids,
                    float* out_dists, void* stream) {
    int rc = check_search_args(ix, queries, nq, k, nprobe, out_ids, out_dists);
    if (rc) return rc;
    const int64_t kc = kc_for(ix, k);
    if (kc > (int64_t)0x7FFFFFFF) return fail(BBC_ERR_ARG, "K_c too large");
    if (nq == 0) return BBC_OK;
    DeviceGuard g(ix->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (ix->dev.quant == BBC_QUANT_SIGN) return search_sign(ix, queries, nq, k, nprobe, out_ids, out_dists, st, true);
    Plan p = make_plan(ix, nq, nprobe, kc, k, true);
    char* ws;
    if ((rc = get_workspace(ix, st, p.total, &ws))) return rc;
    const int d = ix->dev.d;
    // Sub-batches whose results go back on a second stream while the next
    // sub-batches compute: a sub-batch keeps >= 8 queries per SM (one CTA per
    // query fills the GPU), up to three result buffers rotate so that a slow
    // copy-out does not hold up the next sub-batch.  The list-grouped
    // tensor-core scan gains from more queries per list, so its sub-batches
    // are half the batch (the results of one copy out in less time than the
    // next half computes).
    int64_t sb = std::max<int64_t>(8ll * ix->dev.num_sms, tc_active(ix) ? (nq + 1) / 2 : (nq + 3) / 4);
    sb = std::min<int64_t>(sb, std::max<int64_t>(1, p.chunk / 2));
    int nbuf = 2 * sb <= p.chunk ? 2 : 1;
    if (nbuf == 2 && 3 * sb <= p.chunk) nbuf = 3;
    if (nbuf == 1) sb = p.chunk;
    {
        std::lock_guard<std::mutex> lk(ix->mu);
        if (!ix->copy_stream) CUDA_TRY(cudaStreamCreateWithFlags(&ix->copy_stream, cudaStreamNonBlocking));
    }
    cudaStream_t cs = ix->copy_stream;
    cudaEvent_t done[3] = {nullptr, nullptr, nullptr}, freed[3] = {nullptr, nullptr, nullptr};
    auto cleanup = [&]() {
        for (int b = 0; b < 3; ++b) {
            if (done[b]) cudaEventDestroy(done[b]);
            if (freed[b]) cudaEventDestroy(freed[b]);
        }
    };
    for (int b = 0; b < nbuf; ++b) {
        if (cudaEventCreateWithFlags(&done[b], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&freed[b], cudaEventDisableTiming) != cudaSuccess) {
            cleanup();
            return fail(BBC_ERR_CUDA, "event creation failed");
        }
    }
    // the copy-out of the last sub-batch is not hidden behind compute: the
    // remainder that fits one sub-batch is split in two halves
    int it = 0;
    int64_t nc = 0;
    bool halved = false;
    for (int64_t q0 = 0; q0 < nq; q0 += nc, ++it) {
        const int64_t rem = nq - q0;
        nc = std::min(sb, rem);
        if (nbuf >= 2 && !halved && it > 0 && rem <= sb && rem >= 4ll * ix->dev.num_sms) {
            nc = (rem + 1) / 2;
            halved = true;
        }
        const int b = it % nbuf;
        float* dq = reinterpret_cast<float*>(ws + p.off_q) + (size_t)b * sb * d;
        int64_t* di = reinterpret_cast<int64_t*>(ws + p.off_ids) + (size_t)b * sb * k;
        float* dd = reinterpret_cast<float*>(ws + p.off_dists) + (size_t)b * sb * k;
        cudaError_t e = cudaSuccess;
        if (it >= nbuf) e = cudaStreamWaitEvent(st, freed[b], 0);       // buffer b copied out
        if (e == cudaSuccess) e = cudaMemcpyAsync(dq, queries + q0 * d, (size_t)nc * d * 4, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) { cleanup(); return fail(BBC_ERR_CUDA, "copy-in: %s", cudaGetErrorString(e)); }
        rc = run_chunk(ix, p, ws, dq, nc, di, dd, st, 9);
        if (rc) { cleanup(); return rc; }
        e = cudaEventRecord(done[b], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, done[b], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out_ids + q0 * k, di, (size_t)nc * k * 8, cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out_dists + q0 * k, dd, (size_t)nc * k * 4, cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess) e = cudaEventRecord(freed[b], cs);
        if (e != cudaSuccess) { cleanup(); return fail(BBC_ERR_CUDA, "copy-out: %s", cudaGetErrorString(e)); }
    }
    cudaError_t e = cudaStreamSynchronize(cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return fail(BBC_ERR_CUDA, "synchronise: %s", cudaGetErrorString(e));
    return BBC_OK;
}

int bbc_probe(bbc_index* ix, const float* queries, int64_t nq, int32_t nprobe, int32_t* out_lists, void* stream) {
    int rc = check_search_args(ix, queries, nq, 1, nprobe, out_lists, out_lists);
    if (rc) return rc;
    if (nq == 0) return BBC_OK;
    DeviceGuard g(ix->device);
    cudaStream_t st = (cudaStream_t)stream;
    Plan p = make_plan(ix, nq, nprobe, 1, 1, false);
    char* ws;
    if ((rc = get_workspace(ix, st, p.total, &ws))) return rc;
    for (int64_t q0 = 0; q0 < nq; q0 += p.chunk) {
        const int64_t nc = std::min(p.chunk, nq - q0);
        rc = run_chunk(ix, p, ws, queries + q0 * ix->dev.d, nc, nullptr, nullptr, st, 2,
                       out_lists + q0 * nprobe);
        if (rc) return rc;
    }
    return BBC_OK;
}

int bbc_autotune(bbc_index* ix, const float* queries, int64_t nq, int32_t k, int32_t nprobe,
                 const char* cache_path, double* out_ms, void* stream) {
    if (int rc0 = pq_only(ix, "bbc_autotune")) return rc0;
    int rc = check_search_args(ix, queries, nq, k, nprobe, queries, queries);
    if (rc) return rc;
    if (nq < 1) return fail(BBC_ERR_ARG, "autotune needs at least one query");
    char key[512];
    snprintf(key, sizeof(key), "n=%lld,d=%d,nlist=%d,pq=%dx%d,metric=%d,nq=%lld,k=%d,nprobe=%d,kc_ratio=%.6g",
             (long long)ix->dev.n, ix->dev.d, ix->dev.nlist, ix->dev.M, ix->dev.bits, ix->dev.metric, (long long)nq, k,
             nprobe, ix->kc_ratio);
    if (out_ms) *out_ms = 0.0;
    if (cache_path) {
        if (FILE* f = fopen(cache_path, "r")) {
            char line[1024];
            int found_split = -1, found_m = -1, found_pair = 0;
            while (fgets(line, sizeof(line), f)) {
                char want[600];
                snprintf(want, sizeof(want), "\"key\": \"%s\"", key);
                if (!strstr(line, want)) continue;
                static const char ks[] = "\"split\": ";
                static const char kb[] = "\"buckets\": ";
                static const char kp[] = "\"pair\": ";
                const char* a = strstr(line, ks);
                const char* b = strstr(line, kb);
                const char* c = strstr(line, kp);
                if (a && b) {
                    found_split = atoi(a + strlen(ks));
                    found_m = atoi(b + strlen(kb));
                    found_pair = c ? (atoi(c + strlen(kp)) ? 1 : 0) : 0;
                }
            }
            fclose(f);
            if (found_split >= 0 && found_m >= 2 && found_m <= 256) {
                ix->split = found_split;
                ix->buckets = found_m;
                ix->pair = found_pair;
                return BBC_OK;
            }
        }
    }
    DeviceGuard g(ix->device);
    cudaStream_t st = (cudaStream_t)stream;
    int64_t* oi = nullptr;
    float* od = nullptr;
    CUDA_TRY(cudaMalloc(&oi, (size_t)nq * k * 8));
    if (cudaMalloc(&od, (size_t)nq * k * 4) != cudaSuccess) {
        cudaFree(oi);
        return fail(BBC_ERR_OOM, "autotune output buffers");
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int saved_split = ix->split, saved_m = ix->buckets, saved_graphs = ix->graphs, saved_pair = ix->pair;
    ix->graphs = 0;
    auto time_it = [&](double* ms) -> int {
        int r = bbc_search(ix, queries, nq, k, nprobe, oi, od, stream);       // warm-up (allocations)
        if (r) return r;
        double best = 1e300;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, st);
            r = bbc_search(ix, queries, nq, k, nprobe, oi, od, stream);
            if (r) return r;
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) return fail(BBC_ERR_CUDA, "autotune timing");
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            best = std::min(best, (double)t);
        }
        *ms = best;
        return BBC_OK;
    };
    // schedules: (split, pair) = one CTA per query, two queries per CTA (pair
    // form, where supported), G CTAs per query for batches too small to fill the GPU
    std::vector<std::pair<int, int>> scheds = {{1, 0}};
    if (nq >= 2 && scan_pair_supported(ix->dev, nprobe)) scheds.push_back({1, 1});
    const int64_t slots = 2ll * ix->dev.num_sms;
    for (int G : {2, 4, 8, 16, 32, 64, 128})
        if (G <= nprobe && nq * G <= 64 * slots && nq < 8 * slots) scheds.push_back({G, 0});
    double best_ms = 1e300;
    int best_split = 1, best_m = ix->buckets, best_pair = 0;
    for (const auto& sc : scheds) {
        ix->split = sc.first;
        ix->pair = sc.second;
        double t = 1e300;
        if ((rc = time_it(&t))) break;
        if (t < best_ms) { best_ms = t; best_split = sc.first; best_pair = sc.second; }
    }
    if (!rc) {
        ix->split = best_split;
        ix->pair = best_pair;
        for (int m : {32, 64, 128, 256}) {
            ix->buckets = m;
            double t = 1e300;
            if ((rc = time_it(&t))) break;
            if (t < best_ms * 0.98 || (m == best_m && t < best_ms)) { best_ms = t; best_m = m; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(oi);
    cudaFree(od);
    ix->graphs = saved_graphs;
    if (rc) {
        ix->split = saved_split;
        ix->buckets = saved_m;
        ix->pair = saved_pair;
        return rc;
    }
    ix->split = best_split;
    ix->buckets = best_m;
    ix->pair = best_pair;
    if (out_ms) *out_ms = best_ms;
    if (cache_path) {
        if (FILE* f = fopen(cache_path, "a")) {
            fprintf(f, "{\"key\": \"%s\", \"split\": %d, \"pair\": %d, \"buckets\": %d, \"ms\": %.4f}\n", key,
                    best_split, best_pair, best_m, best_ms);
            fclose(f);
        }
    }
    return BBC_OK;
}

int bbc_probe_scores(bbc_index* ix, const float* queries, int64_t nq, float* out_scores, void* stream) {
    if (!ix) return fail(BBC_ERR_ARG, "null index");
    if (nq < 0 || (nq > 0 && (!queries || !out_scores))) return fail(BBC_ERR_ARG, "bad buffers");
    if (nq == 0) return BBC_OK;
    DeviceGuard g(ix->device);
    cudaStream_t st = (cudaStream_t)stream;
    const DevIndex& d = ix->dev;
    if (!ix->probe_gemm) {
        CUDA_TRY(stage(ix, 0, st, [&] { return launch_probe_scores(d, queries, nq, out_scores, st); }));
        return BBC_OK;
    }
    const size_t budget = (size_t)(ix->workspace_mb * 1024.0 * 1024.0);
    int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(nq, (int64_t)(budget / (probe_tc_workspace(d, 1) + 256))));
    char* ws;
    int rc = get_workspace(ix, st, align_up(probe_tc_workspace(d, chunk)), &ws);
    if (rc) return rc;
    for (int64_t q0 = 0; q0 < nq; q0 += chunk) {
        const int64_t nc = std::min(chunk, nq - q0);
        CUDA_TRY(stage(ix, 0, st, [&] {
            return launch_probe_scores_tc(d, queries + q0 * d.d, nc, out_scores + q0 * d.nlist, ws, st);
        }));
    }
    return BBC_OK;
}

int bbc_lut(bbc_index* ix, const float* queries, int64_t nq, uint16_t* out_lut16, void* stream) {
    if (int rc0 = pq_only(ix, "bbc_lut")) return rc0;
    if (!ix) return fail(BBC_ERR_ARG, "null index");
    if (nq < 0 || (nq > 0 && (!queries || !out_lut16))) return fail(BBC_ERR_ARG, "bad buffers");
    if (nq == 0) return BBC_OK;
    DeviceGuard g(ix->device);
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(stage(ix, 2, st, [&] { return launch_lut16(ix->dev, queries, nq, out_lut16, st, nullptr, ix->lut_levels); }));
    return BBC_OK;
}

int bbc_collect(bbc_index* ix, const float* queries, int64_t nq, int32_t nprobe, const int32_t* probe_lists,
                int64_t kc, uint32_t* out_ids, int64_t* out_count, bbc_collector_state* out_state, void* stream) {
    if (int rc0 = pq_only(ix, "bbc_collect")) return rc0;
    int rc = check_search_args(ix, queries, nq, 1, nprobe, out_ids, out_count);
    if (rc) return rc;
    if (nq > 0 && !probe_lists) return fail(BBC_ERR_ARG, "null probe_lists");
    if (kc < 1) return fail(BBC_ERR_ARG, "kc must be >= 1");
    if (kc > (int64_t)0x7FFFFFFF) return fail(BBC_ERR_ARG, "kc too large");
    if (nq == 0) return BBC_OK;
    DeviceGuard g(ix->device);
    cudaStream_t st = (cudaStream_t)stream;
    Plan p = make_plan(ix, nq, nprobe, kc, 1, false);
    char* ws;
    if ((rc = get_workspace(ix, st, p.total, &ws))) return rc;
    for (int64_t q0 = 0; q0 < nq; q0 += p.chunk) {
        const int64_t nc = std::min(p.chunk, nq - q0);
        rc = run_chunk(ix, p, ws, queries + q0 * ix->dev.d, nc, nullptr, nullptr, st, 7, nullptr,
                       probe_lists + q0 * nprobe, out_ids + q0 * kc, out_count + q0,
                       out_state ? out_state + q0 : nullptr);
        if (rc) return rc;
    }
    return BBC_OK;
}

int bbc_rerank_topk(bbc_index* ix, const float* queries, int64_t nq, const uint32_t* cand_ids,
                    const int64_t* cand_count, int64_t kc, int32_t k, int64_t* out_ids, float* out_dists,
                    void* stream) {
    if (int rc0 = pq_only(ix, "bbc_rerank_topk")) return rc0;
    if (!ix) return fail(BBC_ERR_ARG, "null index");
    if (nq < 0 || k < 1 || kc < 1) return fail(BBC_ERR_ARG, "bad sizes");
    if (kc > (int64_t)0x7FFFFFFF) return fail(BBC_ERR_ARG, "kc too large");
    if (nq > 0 && (!queries || !cand_ids || !cand_count || !out_ids || !out_dists)) return fail(BBC_ERR_ARG, "null buffer");
    if (nq == 0) return BBC_OK;
    DeviceGuard g(ix->device);
    cudaStream_t st = (cudaStream_t)stream;
    const bool prec = prec_active(ix);
    const bool large = kc > kTopkSmemMax || (prec && k > kTopkSmemMax);
    // scratch per chunk: distances, keys of the large top-k, precision arrays
    auto bytes = [&](int64_t c) {
        size_t o = align_up((size_t)c * kc * 4);
        o += align_up(large ? (size_t)c * kc * 8 : 0);
        o += prec ? prec_bytes(c, c * kc) : 0;
        return o + 256;
    };
    const size_t budget = (size_t)(ix->workspace_mb * 1024.0 * 1024.0);
    int64_t chunk = std::min<int64_t>(nq, kMaxChunkQueries);
    while (chunk > 1 && bytes(chunk) > budget) chunk = (chunk + 1) / 2;
    char* ws;
    int rc = get_workspace(ix, st, bytes(chunk), &ws);
    if (rc) return rc;
    const int d = ix->dev.d;
    for (int64_t q0 = 0; q0 < nq; q0 += chunk) {
        const int64_t nc = std::min(chunk, nq - q0);
        size_t o = align_up((size_t)chunk * kc * 4);
        unsigned long long* keys = large ? reinterpret_cast<unsigned long long*>(ws + o) : nullptr;
        o += align_up(large ? (size_t)chunk * kc * 8 : 0);
        RerankArgs ra{queries + q0 * d, cand_ids + q0 * kc, cand_count + q0, kc,
                      ix->rerank_u8 && ix->dev.vec_u8 != nullptr, reinterpret_cast<float*>(ws), k,
                      out_ids + q0 * k, out_dists + q0 * k, keys, uniform_params(1, kc, k, 0)};
        if (prec) {
            const PrecArgs pa = prec_args_rerank(ix, ws + o, nc, nc * kc, reinterpret_cast<float*>(ws));
            rc = run_rerank(ix, nc, ra, &pa, k, st);
        } else {
            rc = run_rerank(ix, nc, ra, nullptr, k, st);
        }
        if (rc) return rc;
    }
    return BBC_OK;
}

int bbc_rerank_bounds(bbc_index* ix, const float* queries, int64_t nq, const uint32_t* cand_ids,
                      const int64_t* cand_count, int64_t kc, float* out_dist, float* out_rho, void* stream) {
    if (int rc0 = pq_only(ix, "bbc_rerank_bounds")) return rc0;
    if (!ix) return fail(BBC_ERR_ARG, "null index");
    if (nq < 0 || kc < 1 || kc > (int64_t)0x7FFFFFFF) return fail(BBC_ERR_ARG, "bad sizes");
    if (nq > 0 && (!queries || !cand_ids || !cand_count || !out_dist || !out_rho)) return fail(BBC_ERR_ARG, "null buffer");
    if (ix->dev.prec == 0 || !ix->dev.vec_lp) return fail(BBC_ERR_ARG, "no low-precision copy (set \"precision\" first)");
    if (nq == 0) return BBC_OK;
    DeviceGuard g(ix->device);
    cudaStream_t st = (cudaStream_t)stream;
    RerankArgs ra{queries, cand_ids, cand_count, kc, 0, out_dist, 1, nullptr, nullptr, nullptr,
                  uniform_params(1, kc, 1, 0)};
    PrecArgs pa{};
    pa.rho = out_rho;
    CUDA_TRY(stage(ix, 5, st, [&] { return launch_prec_score(ix->dev, nq, ra, pa, st); }));
    return BBC_OK;
}

int bbc_precision_copy(bbc_index* ix, void* out_rows, float* out_meta, void* stream) {
    if (!ix) return fail(BBC_ERR_ARG, "null index");
    if (ix->dev.prec == 0 || !ix->dev.vec_lp) return fail(BBC_ERR_ARG, "no low-precision copy (set \"precision\" first)");
    if (!out_rows || !out_meta) return fail(BBC_ERR_ARG, "null buffer");
    DeviceGuard g(ix->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t es = ix->dev.prec == 1 ? 2 : 1;
    CUDA_TRY(cudaMemcpyAsync(out_rows, ix->dev.vec_lp, (size_t)ix->dev.n * ix->dev.dpad * es, cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(out_meta, ix->dev.vec_meta, (size_t)ix->dev.n * sizeof(float4), cudaMemcpyDeviceToDevice, st));
    return BBC_OK;
}

int bbc_precision_stats(bbc_index* ix, int64_t* out4, int reset) {
    if (!ix || !out4) return fail(BBC_ERR_ARG, "null argument");
    for (int i = 0; i < 4; ++i) out4[i] = 0;
    if (!ix->prec_totals) return BBC_OK;
    DeviceGuard g(ix->device);
    CUDA_TRY(cudaDeviceSynchronize());
    unsigned long long t[4];
    CUDA_TRY(cudaMemcpy(t, ix->prec_totals, sizeof(t), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 4; ++i) out4[i] = (int64_t)t[i];
    if (reset) CUDA_TRY(cudaMemset(ix->prec_totals, 0, sizeof(t)));
    return BBC_OK;
}

int bbc_early_stats(bbc_index* ix, int64_t* out2, int reset) {
    if (!ix || !out2) return fail(BBC_ERR_ARG, "null argument");
    out2[0] = out2[1] = 0;
    if (!ix->early_totals) return BBC_OK;
    DeviceGuard g(ix->device);
    CUDA_TRY(cudaDeviceSynchronize());
    unsigned long long t[2];
    CUDA_TRY(cudaMemcpy(t, ix->early_totals, sizeof(t), cudaMemcpyDeviceToHost));
    out2[0] = (int64_t)t[0];
    out2[1] = (int64_t)t[1];
    if (reset) CUDA_TRY(cudaMemset(ix->early_totals, 0, sizeof(t)));
    return BBC_OK;
}

int bbc_sign_bounds(bbc_index* ix, const float* queries, int64_t nq, int32_t nprobe, const int32_t* probe_lists,
                    int64_t stride, float* out_lb, float* out_ub, int64_t* out_count, void* stream) {
    int rc = check_search_args(ix, queries, nq, 1, nprobe, out_lb, out_ub);
    if (rc) return rc;
    if (ix->dev.quant != BBC_QUANT_SIGN) return fail(BBC_ERR_UNSUPPORTED, "bbc_sign_bounds: not a sign-code index");
    if (nq > 0 && (!probe_lists || !out_count)) return fail(BBC_ERR_ARG, "null buffer");
    if (stride < 1) return fail(BBC_ERR_ARG, "stride must be >= 1");
    if (nq == 0) return BBC_OK;
    DeviceGuard g(ix->device);
    cudaStream_t st = (cudaStream_t)stream;
    const DevIndex& d = ix->dev;
    char* ws;
    const size_t qb = align_up((size_t)nq * d.d * 8);
    if ((rc = get_workspace(ix, st, qb + align_up(sign_prep_bytes(d, nq * (int64_t)nprobe)), &ws))) return rc;
    double* qrot = reinterpret_cast<double*>(ws);
    CUDA_TRY(stage(ix, 2, st, [&] { return launch_rotate_f64(queries, nullptr, nullptr, nullptr, d.rot, nq, d.d, qrot, st); }));
    SignArgs sa{};
    sa.qrot = qrot; sa.q = queries; sa.lists = probe_lists; sa.nprobe = nprobe; sa.k = 1; sa.m = ix->buckets;
    sa.sample_min = ix->sample_lists; sa.scale = ix->bound_scale; sa.est = ix->estimator; sa.eps0 = ix->eps0; sa.cap = stride; sa.scanned = out_count;
    sa.dbg_lb = out_lb; sa.dbg_ub = out_ub;
    sa.prep = reinterpret_cast<uint32_t*>(ws + qb);
    sa.qp = uniform_params(nprobe, stride, 1, stride);
    CUDA_TRY(stage(ix, 3, st, [&] { return launch_sign_scan(d, nq, sa, st); }));
    return BBC_OK;
}

int bbc_bounded_stats(bbc_index* ix, int64_t* out4, int reset) {
    if (!ix || !out4) return fail(BBC_ERR_ARG, "null argument");
    for (int i = 0; i < 4; ++i) out4[i] = 0;
    if (!ix->sign_totals) return BBC_OK;
    DeviceGuard g(ix->device);
    CUDA_TRY(cudaDeviceSynchronize());
    unsigned long long t[4];
    CUDA_TRY(cudaMemcpy(t, ix->sign_totals, sizeof(t), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 4; ++i) out4[i] = (int64_t)t[i];
    if (reset) CUDA_TRY(cudaMemset(ix->sign_totals, 0, sizeof(t)));
    return BBC_OK;
}

int bbc_profile_read(bbc_index* ix, double* stage_ms, int64_t* launches, int reset) {
    if (!ix) return fail(BBC_ERR_ARG, "null index");
    DeviceGuard g(ix->device);
    std::lock_guard<std::mutex> lk(ix->prof_mu);
    double acc[BBC_NUM_STAGES] = {0};
    for (auto& r : ix->recs) {
        CUDA_TRY(cudaEventSynchronize(r.b));
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, r.a, r.b));
        if (r.stage >= 0 && r.stage < BBC_NUM_STAGES) acc[r.stage] += ms;
    }
    if (stage_ms)
        for (int i = 0; i < BBC_NUM_STAGES; ++i) stage_ms[i] = acc[i];
    if (launches) *launches = ix->launches;
    if (reset) {
        for (auto& r : ix->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
        ix->recs.clear();
        ix->launches = 0;
    }
    return BBC_OK;
}

int bbc_stream_status(bbc_index* ix, void* stream) {
    if (!ix) return fail(BBC_ERR_ARG, "null index");
    DeviceGuard g(ix->device);
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    unsigned int s = 0;
    CUDA_TRY(cudaMemcpy(&s, ix->dev.status, 4, cudaMemcpyDeviceToHost));
    if (s) {
        unsigned int z = 0;
        CUDA_TRY(cudaMemcpy(ix->dev.status, &z, 4, cudaMemcpyHostToDevice));
        return fail(BBC_ERR_CAPACITY, "device status 0x%x (1 region, 2 select, 4 top-k overrun, 16 precision bound)", s);
    }
    return BBC_OK;
}

}  // extern "C"

// ===========================================================================
// Internal accessors for other translation units of the library.
// ===========================================================================
namespace bbc {
int api_error(int code, const char* msg) { return fail(code, "%s", msg); }
int api_check_search_args(const bbc_index* ix, const void* queries, int64_t nq, int k, int nprobe,
                          const void* out_ids, const void* out_dists) {
    return check_search_args(ix, queries, nq, k, nprobe, out_ids, out_dists);
}
const DevIndex& index_dev(const bbc_index* ix) { return ix->dev; }
int index_device(const bbc_index* ix) { return ix->device; }
int64_t index_cap(const bbc_index* ix, int nprobe) { return ix->cap_for(nprobe); }
int index_buckets(const bbc_index* ix) { return ix->buckets; }
int index_lut_levels(const bbc_index* ix) { return ix->lut_levels; }
int index_sample_lists(const bbc_index* ix) { return ix->sample_lists; }
int64_t index_kc(const bbc_index* ix, int k) { return kc_for(ix, k); }
}  // namespace bbc
