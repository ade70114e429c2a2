// S4-S6, list-grouped batched form on the tensor cores (4-bit PQ codes).
//
// The scan's estimated distance e(q, o) = sum_m T_q[m][code_m(o)] (Section 2,
// "Quantization", step (2)) is, for one list, a contraction
//     E[q][o] = sum_k T_q[k] * H_o[k],    k = 16 m + j,
// of the queries' tables T_q (K = 16 M entries) with one-hot code rows H_o
// (H_o[16 m + j] = 1 when code_m(o) = j).  A list is probed by thousands of
// queries of a batch, so one staged tile of its codes serves many queries: the
// work is a dense product with large reuse, which the tensor cores take
// (tcgen05.mma kind::f16, FP32 accumulation in tensor memory).  Tables with
// top level 2047 (k_lut.cu) are integers FP16 holds exactly, a product with a
// one-hot entry is exact, and every partial sum of M <= 128 such entries stays
// below 2^24, so the FP32 accumulator equals the integer table sum bit for bit
// in any summation order: the keys, and with them the result buffer's state
// and candidates, are those of the one-query scan on the same table.
//
// Work: first the one-query scan (k_scan.cu) scans each query's sampled lists
// (the first lists in probe order), appends all their objects and builds the
// query's codebook and threshold, then stops; it reads the same table, so its
// keys are the same.  The (query, probed list) pairs of the other lists are
// grouped by list (a device counting sort) into items of one list and up to
// 128 of its queries, and this kernel runs Push against each query's
// threshold (Algorithm 1) with Update after each item on the query's global
// bucket counts.  The final selection (k_select.cu) computes tau* from the
// counts of everything appended.  tau at any time is >= tau* and buckets are
// monotone in e, so every object of a bucket <= tau* is appended under this
// schedule too (the argument of the one-query scan).
//
// CTA (one per SM, persistent over items; 17 warps):
//   warps 0-7   epilogue: row r (tensor-memory lane r) belongs to warps
//               r / 32 and r / 32 + 4, one per half of the tile's columns;
//               reads a tile's accumulator columns, pushes (key, slot) pairs
//               whose key is at or below the query's current bound into its
//               region (one 64-bit cursor atomic per tile; each 32-column
//               group staged per row in shared memory and written as one
//               contiguous run per row), counts them per bucket in shared
//               memory, and after each item adds the counts to the query's
//               state and runs Update;
//   warp 8      MMA issuer (one elected thread) and tensor-memory owner;
//   warps 9-16  producers of every stage: thread t builds the one-hot row of
//               vector t of the current 256-vector tile from its code row
//               (rotated back to sub-space order), 128 bytes per stage (B), and
//               moves four 16-byte units of the item's 128 table rows (A,
//               coalesced, loaded one stage ahead into registers); both in the
//               128-byte-swizzled K-major layout.
// A 3-stage shared-memory ring (A 16 KB + B 32 KB per stage) feeds the MMA
// (M = 128 query rows, N = the tile's vectors rounded up to 16, K = 16 per
// instruction); two 256-column accumulators in tensor memory let the
// epilogue of one tile overlap the MMAs of the next.  Every mbarrier wait is
// bounded; on expiry the kernel latches the timeout status bit and every role
// stops at its next step, drains its own copies and MMAs (bounded) and frees
// the tensor memory.
#include <algorithm>

#include <cuda_fp16.h>

#include "bbc_internal.cuh"
#include "dev_util.cuh"
#include "tc_util.cuh"

namespace bbc {

constexpr int TQ_BM = 128;                      // query rows per item (tensor-memory lanes)
constexpr int TQ_BN = 256;                      // vectors per tile (accumulator columns)
constexpr int TQ_BK = 64;                       // table entries per stage (128-byte FP16 rows)
constexpr int TQ_STAGES = 3;                   // the MMA issuer selects among 3 stage descriptors
constexpr int TQ_A_BYTES = TQ_BM * TQ_BK * 2;
constexpr int TQ_B_BYTES = TQ_BN * TQ_BK * 2;
constexpr int TQ_STAGE_BYTES = TQ_A_BYTES + TQ_B_BYTES;
constexpr int TQ_E_WARPS = 8, TQ_MMA_WARP = 8, TQ_P_WARP0 = 9, TQ_P_WARPS = 8;
constexpr int TQ_THREADS = 32 * (TQ_P_WARP0 + TQ_P_WARPS);
constexpr uint32_t TQ_FULL_COUNT = 32u * TQ_P_WARPS;   // arrivals that fill one stage
constexpr int TQ_MAX_BUCKETS = 64;              // per-row bucket counts kept in shared memory

// kind::f16 instruction descriptor: FP32 accumulate, FP16 A and B, both
// K-major, M = 128; N >> 3 at bit 17.
__host__ __device__ constexpr uint32_t tq_idesc(int n) {
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TQ_BM >> 4) << 24);
}

constexpr int TQ_HW = TQ_MAX_BUCKETS / 2 + 1;    // words per row of packed 16-bit bucket counts
constexpr int TQ_STG_CAP = 512;                 // staged entries per epilogue warp
// dynamic shared memory: alignment pad; the ring; each row's bucket map (256
// bytes); its bucket counts as 16-bit halves of TQ_HW words; the admitted-
// column masks of a tile (8 per row); each warp's staged appends of one
// 32-column group (up to 32 x 32 packed entries); per-row region pointer,
// capacity, run position, staging offset, d_min and shift; barriers
constexpr size_t TQ_SMEM = 1024 + (size_t)TQ_STAGES * TQ_STAGE_BYTES + (size_t)TQ_BM * 256 +
                           (size_t)TQ_BM * TQ_HW * 4 + (size_t)TQ_BM * 8 * 4 + TQ_E_WARPS * TQ_STG_CAP * 4 +
                           (size_t)TQ_BM * (2 * 16 + 8 + 8 + 4) + 2 * (size_t)TQ_BM * 8 + 8 * (2 * TQ_STAGES + 5) + 16;

bool scan_tc_supported(const DevIndex& ix, int m) {
    return ix.quant == 0 && ix.bits == 4 && (ix.M == 32 || ix.M == 64 || ix.M == 128) && !ix.resid &&
           m >= 1 && m <= TQ_MAX_BUCKETS;
}

// The pairs of a query fall in three groups by probe rank: its sampled lists
// (pass 1), the nearest quarter of the others and the rest (pass 2, near
// items first: with persistent CTAs taking items in order, the near lists are
// scanned first, as in Algorithm 1's nearest-first order, so tau is tight
// before most objects are scanned).
// Plan arrays inside the scratch (int32 unless noted):
//   cnt [3][nlist]          pairs of each list per group
//   fill [3][nlist]         scatter cursors
//   seg [3 nlist + 1]       exclusive offsets into qlist ((group, list) order)
//   nitems [4]              items of pass 1, of the near group, of pass 2
//   qlist [sum of nprobe]   query index of each pair, grouped by (group, list)
//   items int4 [2][cap]     {list, first qlist index, rows, 0}: pass 1, then
//                           pass 2 (near group, then the rest)
struct TqPlan {
    int32_t* cnt;
    int32_t* fill;
    int32_t* seg;
    int32_t* nitems;
    int32_t* qlist;
    int4* items;
    int64_t item_cap;
};

static int64_t tq_item_cap(const DevIndex& ix, int64_t sum_probe) { return 2 * ix.nlist + (sum_probe + TQ_BM - 1) / TQ_BM; }

// Group of the pair at probe rank j of a query with P lists, nsl of them sampled.
__device__ __forceinline__ int tq_group(int j, int nsl, int P) {
    return j < nsl ? 0 : (j < nsl + (P - nsl + 3) / 4 ? 1 : 2);
}

size_t scan_tc_plan_bytes(const DevIndex& ix, int64_t sum_probe) {
    const size_t L = (size_t)ix.nlist;
    size_t o = 0;
    o += 4 * L * 3;                 // cnt
    o += 4 * L * 3;                 // fill
    o += 4 * (3 * L + 1);           // seg
    o += 16;                        // nitems
    o = (o + 15) / 16 * 16;
    o += 4 * (size_t)sum_probe;     // qlist
    o = (o + 15) / 16 * 16;
    o += 16 * 2 * (size_t)tq_item_cap(ix, sum_probe);
    return o;
}

static TqPlan tq_plan(const DevIndex& ix, void* scratch, int64_t sum_probe) {
    const size_t L = (size_t)ix.nlist;
    char* b = static_cast<char*>(scratch);
    TqPlan p{};
    size_t o = 0;
    p.cnt = reinterpret_cast<int32_t*>(b + o); o += 4 * L * 3;
    p.fill = reinterpret_cast<int32_t*>(b + o); o += 4 * L * 3;
    p.seg = reinterpret_cast<int32_t*>(b + o); o += 4 * (3 * L + 1);
    p.nitems = reinterpret_cast<int32_t*>(b + o); o += 16;
    o = (o + 15) / 16 * 16;
    p.qlist = reinterpret_cast<int32_t*>(b + o); o += 4 * (size_t)sum_probe;
    o = (o + 15) / 16 * 16;
    p.items = reinterpret_cast<int4*>(b + o);
    p.item_cap = tq_item_cap(ix, sum_probe);
    return p;
}

// Number of sampled lists of a query (warp-collective): at least
// min(sample_min, P) lists in probe order, extended until they hold
// min(K_c, S_q) vectors; *sq = S_q.
__device__ int tq_sample_lists(const DevIndex& ix, const int32_t* lists, int P, int64_t kc, int sample_min,
                               long long* sq) {
    const unsigned ln = lane_id();
    long long tot = 0;
    for (int base = 0; base < P; base += 32) {
        const int j = base + (int)ln;
        const unsigned long long inc = warp_incl_scan64(j < P ? (unsigned long long)ix.list_len[lists[j]] : 0ull);
        tot += (long long)__shfl_sync(0xFFFFFFFFu, inc, 31);
    }
    const long long want = kc < tot ? kc : tot;
    const int smin = sample_min < P ? sample_min : P;
    long long cum = 0;
    int nsl = P;
    for (int base = 0; base < P; base += 32) {
        const int j = base + (int)ln;
        const unsigned long long inc = warp_incl_scan64(j < P ? (unsigned long long)ix.list_len[lists[j]] : 0ull);
        const bool ok = j < P && (j + 1) >= smin && (long long)(cum + (long long)inc) >= want;
        const unsigned hit = __ballot_sync(0xFFFFFFFFu, ok);
        if (hit) { nsl = base + (int)(__ffs(hit) - 1) + 1; break; }
        cum += (long long)__shfl_sync(0xFFFFFFFFu, inc, 31);
    }
    *sq = tot;
    return nsl;
}

// One warp per query: its sample plan into the state, and the pair counts.
__global__ void tq_count_kernel(DevIndex ix, ScanArgs a, TqPlan p, int64_t nq) {
    const int64_t qi = (int64_t)blockIdx.x * (blockDim.x / 32) + warp_id();
    if (qi >= nq) return;
    const int P = a.qp.P(qi);
    const int32_t* lists = a.lists + a.qp.poff(qi);
    long long sq;
    const int nsl = tq_sample_lists(ix, lists, P, a.qp.KC(qi), a.sample_min, &sq);
    if (lane_id() == 0) {
        a.state[qi].sample_lists = nsl;
        a.state[qi].scanned = sq;
    }
    // the sampled lists were scanned by the one-query kernel
    for (int j = nsl + (int)lane_id(); j < P; j += 32) atomicAdd(&p.cnt[tq_group(j, nsl, P) * ix.nlist + lists[j]], 1);
}

// One CTA: exclusive offsets of the (pass, list) segments and the item lists.
__global__ void __launch_bounds__(1024) tq_offsets_kernel(DevIndex ix, TqPlan p) {
    __shared__ int32_t wsum[32];
    __shared__ int32_t carry_s;
    const int L3 = 3 * ix.nlist;
    const int tid = threadIdx.x, bs = blockDim.x;
    // segments over the 3 * nlist counts, then the items of each group
    for (int phase = 0; phase < 4; ++phase) {
        // phase 0: seg over all counts; phase 1 / 2 / 3: items of group 0 / 1 / 2
        const int n = phase == 0 ? L3 : ix.nlist;
        const int32_t* c = phase == 0 ? p.cnt : p.cnt + (phase - 1) * ix.nlist;
        // group 2's items follow group 1's in the second item array
        if (tid == 0) carry_s = phase == 3 ? p.nitems[1] : 0;
        __syncthreads();
        for (int base = 0; base < n; base += bs) {
            const int i = base + tid;
            int32_t v = 0;
            // (an empty list gets no items: every item has at least one tile)
            if (i < n) v = phase == 0 ? c[i] : (ix.list_len[i] > 0 ? (c[i] + TQ_BM - 1) / TQ_BM : 0);
            const int32_t inc = (int32_t)warp_incl_scan((uint32_t)v);
            if (lane_id() == 31) wsum[warp_id()] = inc;
            __syncthreads();
            if (warp_id() == 0) {
                const int nw = bs >> 5;
                const int32_t x = (int)lane_id() < nw ? wsum[lane_id()] : 0;
                const int32_t xi = (int32_t)warp_incl_scan((uint32_t)x);
                if ((int)lane_id() < nw) wsum[lane_id()] = xi - x;
            }
            __syncthreads();
            const int32_t excl = carry_s + wsum[warp_id()] + inc - v;
            if (i < n) {
                if (phase == 0) {
                    p.seg[i] = excl;
                } else {
                    // the items of this list
                    const int grp = phase - 1;
                    const int32_t cnt = c[i];
                    int4* it = p.items + (grp == 0 ? 0 : (size_t)p.item_cap);
                    for (int t = 0; t < v; ++t)
                        it[excl + t] = make_int4(i, p.seg[grp * ix.nlist + i] + t * TQ_BM, min(TQ_BM, cnt - t * TQ_BM), 0);
                }
            }
            __syncthreads();
            if (tid == bs - 1) carry_s = excl + v;
            __syncthreads();
        }
        if (tid == 0) {
            if (phase == 0) p.seg[L3] = carry_s;
            else p.nitems[phase == 3 ? 2 : phase - 1] = carry_s;    // nitems[2]: both groups of pass 2
        }
        __syncthreads();
    }
}

// One warp per query: each pair into its (pass, list) segment.
__global__ void tq_scatter_kernel(DevIndex ix, ScanArgs a, TqPlan p, int64_t nq) {
    const int64_t qi = (int64_t)blockIdx.x * (blockDim.x / 32) + warp_id();
    if (qi >= nq) return;
    const int P = a.qp.P(qi);
    const int32_t* lists = a.lists + a.qp.poff(qi);
    const int nsl = a.state[qi].sample_lists;
    for (int j = nsl + (int)lane_id(); j < P; j += 32) {
        const int key = tq_group(j, nsl, P) * ix.nlist + lists[j];
        const int32_t slot = atomicAdd(&p.fill[key], 1);
        p.qlist[p.seg[key] + slot] = (int32_t)qi;
    }
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint4 v) {
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

// The key bound of a query for threshold bucket tau: buckets are monotone in
// the equal-width bin, so bucket(e) <= tau exactly for the c bins whose map
// entry is <= tau, i.e. for e <= d_min + (c << sh) - 1 (all e when c = 256).
__device__ __forceinline__ uint32_t tq_etau(const bbc_collector_state* st, uint32_t tau) {
    if (tau >= 255u) return 0xFFFFFFFFu;
    const uint4* mp = reinterpret_cast<const uint4*>(st->map);
    const uint32_t tt = tau * 0x01010101u;
    uint32_t c = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const uint4 w = mp[i];
        c += (uint32_t)(__popc(__vcmpleu4(w.x, tt)) + __popc(__vcmpleu4(w.y, tt)) + __popc(__vcmpleu4(w.z, tt)) +
                        __popc(__vcmpleu4(w.w, tt)));
    }
    c >>= 3;
    if (c >= 256u) return 0xFFFFFFFFu;
    const unsigned long long v = (unsigned long long)st->d_min + ((unsigned long long)c << st->sh) - 1ull;
    return v > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)v;
}

struct TqArgs {
    const uint16_t* lut_f16;      // [nq][16 M] FP16 tables (entries <= 2047)
    const int4* items;            // this pass's items
    const int32_t* nitems;        // this pass's item count (device)
    const int32_t* qlist;
    bbc_collector_state* state;
    uint2* region;
    QueryParams qp;
    int m;                        // buckets
};

// M: sub-spaces (4-bit codes).  Push against each query's threshold, bucket
// counts and Update after every item (the sampled lists are scanned before,
// by the one-query scan).
template <int M>
__global__ void __launch_bounds__(TQ_THREADS, 1) scan_tc_kernel(DevIndex ix, TqArgs a) {
    constexpr int KT = 16 * M;                  // table entries per query
    constexpr int KCH = KT / TQ_BK;             // stages per tile
    constexpr int NW = M / 8;                   // 32-bit words of a code row
    constexpr int NCH = (M / 2 + 15) / 16;      // 16-byte chunks of a code row
    static_assert(KT % TQ_BK == 0, "table length must be a multiple of 64");
    extern __shared__ uint8_t tq_raw[];
    const uint32_t raw = smem_u32(tq_raw);
    const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
    uint8_t* sm = tq_raw + pad;
    const uint32_t sbase = raw + pad;
    constexpr uint32_t S = TQ_STAGES;
    // [128] per row and group: {region address of staging entry 0 of the row's
    // run (as an integer), entries the region still takes counted from staging
    // entry 0, (shift << 24) | d_min}
    uint4* s_rec = reinterpret_cast<uint4*>(sm + S * TQ_STAGE_BYTES);  // [2][128]: one per column half
    uint2** s_reg = reinterpret_cast<uint2**>(s_rec + 2 * TQ_BM);      // [128] region of each row's query
    unsigned long long* s_cap = reinterpret_cast<unsigned long long*>(s_reg + TQ_BM);   // [128] its capacity
    uint32_t* s_dmsh = reinterpret_cast<uint32_t*>(s_cap + TQ_BM);     // [128] (shift << 24) | d_min
    const uint4** s_asrc = reinterpret_cast<const uint4**>(s_dmsh + TQ_BM);   // [2][128] table rows of an item
    uint32_t* s_mk = reinterpret_cast<uint32_t*>(s_asrc + 2 * TQ_BM);  // [8][128] admitted columns per group
    uint32_t* stg = s_mk + 8 * TQ_BM;                                  // [8][TQ_STG_CAP] staged appends per warp
    uint32_t* hist = stg + TQ_E_WARPS * TQ_STG_CAP;                    // [128][TQ_HW] 16-bit bucket counts
    uint8_t* smap = reinterpret_cast<uint8_t*>(hist + TQ_BM * TQ_HW);  // [128][256] bucket maps
    uint64_t* bars = reinterpret_cast<uint64_t*>(smap + TQ_BM * 256);
    // bars: full[S], empty[S], accfull[2], accempty[2], done
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * TQ_STAGES + 5);
    volatile int* s_abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const uint32_t bar0 = smem_u32(bars);
    auto full = [&](uint32_t s) { return bar0 + 8u * s; };
    auto empty = [&](uint32_t s) { return bar0 + 8u * (TQ_STAGES + s); };
    auto accf = [&](uint32_t b) { return bar0 + 8u * (2 * TQ_STAGES + b); };
    auto acce = [&](uint32_t b) { return bar0 + 8u * (2 * TQ_STAGES + 2 + b); };
    const uint32_t done = bar0 + 8u * (2 * TQ_STAGES + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (uint32_t s = 0; s < S; ++s) {
            mbar_init(full(s), TQ_FULL_COUNT);
            mbar_init(empty(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf(b), 1);
            mbar_init(acce(b), 32u * TQ_E_WARPS);
        }
        mbar_init(done, 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    if (warp == TQ_MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (warp < 4)
        for (int w = 0; w < TQ_HW; ++w) hist[tid * TQ_HW + w] = 0u;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int n_items = *a.nitems;
    auto abort_now = [&]() {
        if (!*s_abort) {
            *s_abort = 1;
            atomicOr(ix.status, kStatusTimeout);
        }
    };

    if (warp == TQ_MMA_WARP) {
        // ---------------- MMA issuer ----------------
        // One thread; the per-stage path is kept short: descriptors of each
        // stage precomputed (the K step of 16 FP16 is 32 bytes, 2 in the
        // descriptor's 16-byte address units), a wait first tried without
        // reading the clock, and the stop flag read only after a wait failed
        // (the other roles stop by ceasing to arrive).
        if (lane == 0) {
            uint32_t g = 0, tcount = 0, s = 0, ph = 0;           // stage and its phase parity
            bool ok = true;
            uint64_t ad[TQ_STAGES], bd[TQ_STAGES];
#pragma unroll
            for (int q = 0; q < TQ_STAGES; ++q) {
                ad[q] = sw128_desc(sbase + q * TQ_STAGE_BYTES);
                bd[q] = sw128_desc(sbase + q * TQ_STAGE_BYTES + TQ_A_BYTES);
            }
            auto wait = [&](uint32_t bar, uint32_t par) -> bool {
                if (mbar_try_wait(bar, par)) return true;
                return mbar_wait(bar, par) && !*s_abort;
            };
            for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
                const int len = ix.list_len[a.items[it].x];
                for (int t = 0; t * TQ_BN < len && ok; ++t, ++tcount) {
                    const uint32_t b = tcount & 1u, v = tcount >> 1;
                    if (!wait(acce(b), (v & 1u) ^ 1u)) { ok = false; break; }
                    tc_fence_after();
                    const int nt = min(TQ_BN, len - t * TQ_BN);
                    const uint32_t idesc = tq_idesc((nt + 15) / 16 * 16);
                    const uint32_t dcol = tmem + b * (uint32_t)TQ_BN;
                    for (int i = 0; i < KCH; ++i, ++g) {
                        if (!wait(full(s), ph)) { ok = false; break; }
                        tc_fence_after();
                        const uint64_t a0 = ad[0], a1 = ad[1], a2 = ad[2], b0 = bd[0], b1 = bd[1], b2 = bd[2];
                        const uint64_t as = s == 0 ? a0 : (s == 1 ? a1 : a2), bs = s == 0 ? b0 : (s == 1 ? b1 : b2);
#pragma unroll
                        for (int k = 0; k < TQ_BK / 16; ++k)
                            tc_mma_f16(dcol, as + 2u * k, bs + 2u * k, idesc, (i | k) != 0 ? 1u : 0u);
                        tc_commit(empty(s));
                        if (++s == TQ_STAGES) { s = 0; ph ^= 1u; }
                    }
                    if (!ok) break;
                    tc_commit(accf(b));
                }
            }
            if (!ok) abort_now();
        }
        __syncwarp();
    } else if (warp >= TQ_P_WARP0) {
        // ---------------- producers: both operands of every stage ----------------
        // B: thread r builds the one-hot row of vector r of the tile.
        // A: the item's 128 table rows, 8 consecutive lanes per 128-byte row
        // segment (one 512-byte coalesced load per warp instruction covers 4
        // rows): thread r moves 16-byte unit r mod 8 of rows r / 8 + 32 k,
        // k < 4.  The A loads for the next stage are issued once this stage is
        // stored, so their latency overlaps the wait for the next free stage.
        // The item's row addresses are kept in shared memory (two sets, for
        // this item and the next).
        const int r = tid - 32 * TQ_P_WARP0;                  // 0..255
        const uint32_t rx = (uint32_t)(r & 7);
        const uint4* codes = reinterpret_cast<const uint4*>(ix.codes);
        const uint32_t uj = (uint32_t)(r & 7), rb = (uint32_t)(r >> 3);
        uint32_t g = 0;
        bool ok = true;
        // row addresses of item it into set h (threads 0..127, one row each)
        auto set_rows = [&](int it, int h) {
            if (r < TQ_BM) {
                const int4 item = a.items[it];
                s_asrc[h * TQ_BM + r] =
                    r < item.z ? reinterpret_cast<const uint4*>(a.lut_f16 + (int64_t)a.qlist[item.y + r] * KT) : nullptr;
            }
        };
        // table segments of two stages in flight: even and odd stages (KCH is even)
        uint4 cur[2][4];
        auto fetch = [&](uint4 (&c)[4], int h, int i) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint4* sp = s_asrc[h * TQ_BM + rb + 32 * k];
                c[k] = sp ? __ldg(sp + i * (TQ_BK / 8) + uj) : make_uint4(0u, 0u, 0u, 0u);
            }
        };
        // the 256 producer threads sync among themselves with named barrier 1;
        // each sync also agrees on whether to stop (a failed wait anywhere), so
        // all of them always leave the item loop together
        auto pbar = [&](bool bad) -> bool {
            uint32_t any;
            asm volatile(
                "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, 256, p;\n selp.u32 %0, 1, 0, q;\n}"
                : "=r"(any)
                : "r"((uint32_t)bad)
                : "memory");
            return any != 0u;
        };
        // raw code row of this thread's vector in the next tile (loaded one tile ahead)
        uint32_t rwn[NW];
        auto load_codes = [&](int blk0_, int len_, int t_) {
            const int vv = t_ * TQ_BN + r;
#pragma unroll
            for (int w = 0; w < NW; ++w) rwn[w] = 0u;
            if (vv < len_) {
                const uint4* cp = codes + ((size_t)(blk0_ + (vv >> 5)) * NCH) * 32 + (vv & 31);
#pragma unroll
                for (int c = 0; c < NCH; ++c) {
                    const uint4 x = __ldg(cp + c * 32);
                    if (4 * c + 0 < NW) rwn[4 * c + 0] = x.x;
                    if (4 * c + 1 < NW) rwn[4 * c + 1] = x.y;
                    if (4 * c + 2 < NW) rwn[4 * c + 2] = x.z;
                    if (4 * c + 3 < NW) rwn[4 * c + 3] = x.w;
                }
            }
        };
        // the code row in sub-space order: slot s of lane t holds sub-space
        // (s + t) mod M, so rotate left by 4 (t mod M) bits; the lane of this
        // thread's vector is r mod 32 in every tile
        const uint32_t rot = 4u * (uint32_t)((r & 31) % M);
        const uint32_t ws = rot >> 5, bsh = rot & 31u;
        int it = blockIdx.x, h = 0;
        if (it < n_items) set_rows(it, 0);
        if (pbar(false)) ok = false;
        if (it < n_items) {
            fetch(cur[0], 0, 0);
            fetch(cur[1], 0, 1);
            const int l0 = a.items[it].x;
            load_codes(ix.list_blk[l0], ix.list_len[l0], 0);
        }
        for (; it < n_items && ok; it += gridDim.x, h ^= 1) {
            const int4 item = a.items[it];
            const int len = ix.list_len[item.x];
            const int blk0 = ix.list_blk[item.x];
            const int T = (len + TQ_BN - 1) / TQ_BN;
            const int nit = it + (int)gridDim.x;
            int nblk0 = 0, nlen = 0;
            if (nit < n_items) {
                set_rows(nit, h ^ 1);
                const int nl = a.items[nit].x;
                nblk0 = ix.list_blk[nl];
                nlen = ix.list_len[nl];
            }
            if (pbar(*s_abort != 0)) { ok = false; break; }
            for (int t = 0; t < T && ok; ++t) {
                const int v = t * TQ_BN + r;                  // list position
                const int nt = min(TQ_BN, len - t * TQ_BN);
                const bool write = r < (nt + 15) / 16 * 16;   // rows the MMA reads
                uint32_t rw[NW];
#pragma unroll
                for (int w = 0; w < NW; ++w) rw[w] = rwn[w];
                // the next tile's code rows: this list's next tile or the next item's first
                if (t + 1 < T) load_codes(blk0, len, t + 1);
                else if (nit < n_items) load_codes(nblk0, nlen, 0);
                uint32_t cw[NW];
#pragma unroll
                for (int w = 0; w < NW; ++w) cw[w] = 0u;
                if (v < len) {
                    // word rotation by ws (0..3) in two conditional steps
                    uint32_t t1[NW];
#pragma unroll
                    for (int w = 0; w < NW; ++w) t1[w] = (ws & 1u) ? rw[(w + NW - 1) % NW] : rw[w];
#pragma unroll
                    for (int w = 0; w < NW; ++w) rw[w] = (ws & 2u) ? t1[(w + NW - 2) % NW] : t1[w];
#pragma unroll
                    for (int w = 0; w < NW; ++w) cw[w] = __funnelshift_l(rw[(w + NW - 1) % NW], rw[w], bsh);
                }
#pragma unroll
                for (int i = 0; i < KCH; ++i, ++g) {
                    const uint32_t s = g % S, u = g / S;
                    if (!mbar_wait(empty(s), (u & 1u) ^ 1u) || *s_abort) { abort_now(); ok = false; break; }
                    const uint32_t st0 = sbase + s * TQ_STAGE_BYTES;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint32_t ar = rb + 32u * (uint32_t)k;
                        st_shared_v4(st0 + ar * 128u + ((uj ^ (ar & 7u)) << 4), cur[i & 1][k]);
                    }
                    if (write) {
                        const uint32_t row = st0 + TQ_A_BYTES + (uint32_t)r * 128u;
                        const uint32_t h16 = (cw[i >> 1] >> ((i & 1) * 16)) & 0xFFFFu;   // sub-spaces 4i..4i+3
#pragma unroll
                        for (int q4 = 0; q4 < 4; ++q4) {
                            const uint32_t c = (h16 >> (4 * q4)) & 15u;
                            const uint32_t one = (v < len) ? (0x3C00u << ((c & 1u) << 4)) : 0u;   // FP16 1.0
                            const uint32_t w = (c >> 1) & 3u;
                            const uint4 x = make_uint4(w == 0 ? one : 0u, w == 1 ? one : 0u, w == 2 ? one : 0u,
                                                       w == 3 ? one : 0u);
                            const uint4 z = make_uint4(0u, 0u, 0u, 0u);
                            st_shared_v4(row + ((((uint32_t)(2 * q4)) ^ rx) << 4), (c & 8u) ? z : x);
                            st_shared_v4(row + ((((uint32_t)(2 * q4 + 1)) ^ rx) << 4), (c & 8u) ? x : z);
                        }
                    }
                    fence_async_smem();
                    mbar_arrive(full(s));
                    // the table segments two stages ahead: a later chunk of this tile, one
                    // of the next tile's first two, or of the next item's first two
                    if (i + 2 < KCH) fetch(cur[i & 1], h, i + 2);
                    else if (t + 1 < T) fetch(cur[i & 1], h, i + 2 - KCH);
                    else if (nit < n_items) fetch(cur[i & 1], h ^ 1, i + 2 - KCH);
                }
            }
            // every thread is done with this item's set before it is rewritten
            if (pbar(!ok || *s_abort != 0)) ok = false;
        }
        if (!ok) abort_now();
    } else {
        // ---------------- epilogue: warps 0-7 ----------------
        // Warp e reads tensor-memory lanes 32 (e mod 4) .. + 31 (rows = queries)
        // and the columns of groups 4 (e / 4) .. + 3 of each tile: two warps
        // share a row, one per half of the tile's 256 columns.  A row's appends
        // go to its own query's region.  Per 32-column group, the warp packs
        // the admitted entries of its 32 rows into one list ((key << 10) | (row
        // << 5) | column) in shared memory; the lanes then walk that list
        // together, so each writes one entry and counts it in its row's bucket
        // counts (16-bit halves, shared-memory atomics).  The two warps of a
        // lane quarter meet at a named barrier (2 + quarter) at each item's
        // start and end; each meeting also agrees on whether to stop.
        const int qd = warp & 3, hf = warp >> 2;
        const int r = qd * 32 + lane;                           // row (query) of this thread
        const uint32_t rl = (uint32_t)lane;                     // row within the warp
        const int wr0 = qd * 32;
        const uint32_t tl = tmem + ((uint32_t)(qd * 32) << 16);
        uint32_t* wstg = stg + warp * TQ_STG_CAP;
        uint4* srec = s_rec + hf * TQ_BM;
        uint32_t* hrow = hist + r * TQ_HW;
        uint32_t tcount = 0;
        bool ok = true;
        auto qbar = [&](bool bad) -> bool {
            uint32_t any;
            asm volatile(
                "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, 64, p;\n selp.u32 %0, 1, 0, q;\n}"
                : "=r"(any)
                : "r"((uint32_t)bad), "r"(2 + qd)
                : "memory");
            return any != 0u;
        };
        // the row's 16-bit counts into its query's bucket counts (read and cleared atomically:
        // the other warp of the row may be counting into them)
        auto flush_counts = [&](bbc_collector_state* st) {
            for (int w = 0; w < TQ_HW; ++w) {
                if (hrow[w]) {
                    const uint32_t c = atomicExch(&hrow[w], 0u);
                    if (c & 0xFFFFu) atomicAdd(&st->hist[2 * w], c & 0xFFFFu);
                    if (c >> 16) atomicAdd(&st->hist[2 * w + 1], c >> 16);
                }
            }
        };
        for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
            const int4 item = a.items[it];
            const int len = ix.list_len[item.x];
            const uint32_t slot0 = (uint32_t)ix.list_blk[item.x] * 32u;
            const int64_t qi = r < item.z ? (int64_t)a.qlist[item.y + r] : -1;
            bbc_collector_state* st = qi >= 0 ? a.state + qi : nullptr;
            uint32_t etau = 0xFFFFFFFFu;
            if (hf == 0) {
                s_reg[r] = st ? a.region + a.qp.roff(qi) : nullptr;
                s_cap[r] = st ? (unsigned long long)a.qp.rcap(qi) : 0ull;
                if (st) {
                    s_dmsh[r] = ((uint32_t)st->sh << 24) | st->d_min;   // d_min < 2^24 (keys are below 2^18)
                    const uint4* mp = reinterpret_cast<const uint4*>(st->map);
#pragma unroll
                    for (int i = 0; i < 16; ++i) reinterpret_cast<uint4*>(smap + r * 256)[i] = mp[i];
                }
            }
            if (st) etau = tq_etau(st, (uint32_t)*(volatile int*)&st->tau);
            if (qbar(*s_abort != 0)) { ok = false; break; }    // the row's descriptors are in place
            const float etf = etau >= (1u << 24) ? 3.0e38f : (float)etau;
            for (int t = 0; t * TQ_BN < len; ++t, ++tcount) {
                const uint32_t b = tcount & 1u, v = tcount >> 1;
                const bool got = __all_sync(0xFFFFFFFFu, mbar_wait(accf(b), v & 1u)) && !*s_abort;
                if (!got) { abort_now(); ok = false; break; }
                tc_fence_after();
                if (hf == 0 && st && t > 0 && t % 255 == 0) flush_counts(st);   // 16-bit counts stay below 2^16
                const int nt = min(TQ_BN, len - t * TQ_BN);
                const int g0 = hf * 4, g1 = min((nt + 31) / 32, g0 + 4);     // this warp's groups
                const uint32_t tb = tl + b * (uint32_t)TQ_BN;
                // pass 1: which columns Push admits (key <= the query's bound)
                uint32_t tot = 0;
#pragma unroll 1
                for (int gi = g0; gi < g1; ++gi) {
                    uint32_t acc[32];
                    tmem_ld32(tb + (uint32_t)(gi * 32), acc);
                    const int nv = min(32, nt - gi * 32);
                    uint32_t mk = 0u;
#pragma unroll
                    for (int j = 0; j < 32; ++j) mk |= (j < nv && __uint_as_float(acc[j]) <= etf) ? (1u << j) : 0u;
                    if (!st) mk = 0u;
                    s_mk[gi * TQ_BM + r] = mk;
                    tot += (uint32_t)__popc(mk);
                }
                // one cursor atomic per tile, row and column half
                unsigned long long pos = 0;
                if (tot) pos = atomicAdd(reinterpret_cast<unsigned long long*>(&st->pushed), (unsigned long long)tot);
                // pass 2, per group: pack the admitted entries, then write and count them;
                // in two rounds of 16 rows when more than the staging holds
#pragma unroll 1
                for (int gi = g0; gi < g1; ++gi) {
                    const uint32_t mk = s_mk[gi * TQ_BM + r];
                    const uint32_t n = (uint32_t)__popc(mk);
                    const uint32_t Tall = __reduce_add_sync(0xFFFFFFFFu, n);
                    if (Tall == 0u) continue;
                    uint32_t acc[32];
                    tmem_ld32(tb + (uint32_t)(gi * 32), acc);
                    const int rounds = Tall > (uint32_t)TQ_STG_CAP ? 2 : 1;
                    const uint32_t c0 = slot0 + (uint32_t)(t * TQ_BN + gi * 32);
#pragma unroll 1
                    for (int rd = 0; rd < rounds; ++rd) {
                        const bool mine = rounds == 1 || (int)(rl >> 4) == rd;
                        const uint32_t nn = mine ? n : 0u;
                        const uint32_t inc = warp_incl_scan(nn);
                        const uint32_t T = __shfl_sync(0xFFFFFFFFu, inc, 31);
                        uint32_t k = inc - nn;
                        if (mine) {
                            // region address of staging entry 0 of this run, and how many
                            // entries (counted from staging entry 0) the region still takes
                            const long long lim = (long long)s_cap[r] - (long long)pos + (long long)k;
                            const unsigned long long ra = reinterpret_cast<unsigned long long>(s_reg[r]) +
                                                          8ull * (pos - (unsigned long long)k);
                            srec[r] = make_uint4((uint32_t)ra, (uint32_t)(ra >> 32),
                                                 (uint32_t)(lim < 0 ? 0 : (lim > 0x7FFFFFFF ? 0x7FFFFFFF : lim)),
                                                 s_dmsh[r]);
                            pos += n;
#pragma unroll
                            for (int j = 0; j < 32; ++j) {
                                if ((mk >> j) & 1u) {
                                    wstg[k] = (__float2uint_rn(__uint_as_float(acc[j])) << 10) | (rl << 5) | (uint32_t)j;
                                    ++k;
                                }
                            }
                        }
                        __syncwarp();
                        for (uint32_t e0 = 0; e0 < T; e0 += 128) {
                            // four entries per lane, their loads issued together
                            uint32_t e[4];
                            uint4 rc[4];
#pragma unroll
                            for (int q = 0; q < 4; ++q) e[q] = e0 + 32 * q + rl < T ? wstg[e0 + 32 * q + rl] : 0xFFFFFFFFu;
#pragma unroll
                            for (int q = 0; q < 4; ++q) rc[q] = srec[wr0 + (int)((e[q] >> 5) & 31u)];
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const uint32_t ei = e0 + 32 * q + rl;
                                if (ei < T) {
                                    const uint32_t key = e[q] >> 10;
                                    if (ei < rc[q].z) {
                                        uint2* dst = reinterpret_cast<uint2*>(((unsigned long long)rc[q].y << 32) | rc[q].x) + ei;
                                        *dst = make_uint2(key, c0 + (e[q] & 31u));
                                    } else {
                                        atomicOr(ix.status, kStatusRegionOverrun);
                                    }
                                    const uint32_t dm = rc[q].w & 0xFFFFFFu, sh = rc[q].w >> 24;
                                    uint32_t bn = 0u;
                                    if (key > dm) {
                                        bn = (key - dm) >> sh;
                                        bn = bn > 255u ? 255u : bn;
                                    }
                                    const int rr = wr0 + (int)((e[q] >> 5) & 31u);
                                    const uint32_t bk = smap[rr * 256 + bn];
                                    atomicAdd(&hist[rr * TQ_HW + (bk >> 1)], 1u << ((bk & 1u) << 4));
                                }
                            }
                        }
                        __syncwarp();
                    }
                }
                tc_fence_before();
                mbar_arrive(acce(b));
            }
            // both warps of the row are done with this item
            if (qbar(!ok || *s_abort != 0)) ok = false;
            if (!ok) break;
            if (hf == 0 && st) {
                // this item's counts into the query's state, then Update on them
                flush_counts(st);
                // Update: the first bucket whose running count reaches K_c, read 32
                // counts at a time with independent loads
                const unsigned long long kc = (unsigned long long)a.qp.KC(qi);
                unsigned long long run = 0;
                int tnew = a.m;
                for (int b0 = 0; b0 < a.m && tnew == a.m; b0 += 32) {
                    uint32_t h[32];
#pragma unroll
                    for (int v4 = 0; v4 < 8; ++v4) {
                        uint4 w;
                        asm volatile("ld.volatile.global.v4.u32 {%0, %1, %2, %3}, [%4];"
                                     : "=r"(w.x), "=r"(w.y), "=r"(w.z), "=r"(w.w)
                                     : "l"(st->hist + b0 + 4 * v4));
                        h[4 * v4] = w.x; h[4 * v4 + 1] = w.y; h[4 * v4 + 2] = w.z; h[4 * v4 + 3] = w.w;
                    }
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        run += (b0 + j < a.m) ? h[j] : 0u;
                        if (tnew == a.m && b0 + j < a.m && run >= kc) tnew = b0 + j;
                    }
                }
                if (tnew < *(volatile int*)&st->tau) atomicMin(&st->tau, tnew);
            }
        }
        if (!ok) abort_now();
    }
    // every role is done; the MMA thread's last commit arrives when all the
    // MMAs it issued have completed (bounded wait), then the tensor memory
    // is freed
    tc_fence_before();
    __syncthreads();
    if (warp == TQ_MMA_WARP) {
        if (lane == 0) {
            tc_commit(done);
            if (!mbar_wait(done, 0u)) atomicOr(ix.status, kStatusTimeout);
        }
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u));
    }
}


template <int M>
static cudaError_t launch_tc_t(const DevIndex& ix, int64_t nq, const ScanArgs& sa, const uint16_t* lut_f16,
                               void* scratch, int64_t sum_probe, cudaStream_t st) {
    const TqPlan p = tq_plan(ix, scratch, sum_probe);
    const size_t smem = TQ_SMEM;
    cudaError_t e;
    if ((e = smem_attr_once((const void*)scan_tc_kernel<M>, (int)smem)) != cudaSuccess) return e;
    // the sample and the codebooks: the one-query scan stopped after its phase C
    // (the same keys: it reads the same table), then the plan over the other lists
    ScanArgs ss = sa;
    ss.sample_only = 1;
    ss.fuse_select = 0;
    if ((e = launch_scan(ix, nq, ss, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(p.cnt, 0, sizeof(int32_t) * 6 * (size_t)ix.nlist, st)) != cudaSuccess) return e;   // cnt + fill
    const unsigned wblocks = (unsigned)((nq + 7) / 8);
    tq_count_kernel<<<wblocks, 256, 0, st>>>(ix, sa, p, nq);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    tq_offsets_kernel<<<1, 1024, 0, st>>>(ix, p);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    tq_scatter_kernel<<<wblocks, 256, 0, st>>>(ix, sa, p, nq);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    TqArgs ta{lut_f16, p.items, p.nitems, p.qlist, sa.state, sa.region, sa.qp, sa.m};
    const unsigned grid = (unsigned)ix.num_sms;
    ta.items = p.items + p.item_cap;
    ta.nitems = p.nitems + 2;
    scan_tc_kernel<M><<<grid, TQ_THREADS, smem, st>>>(ix, ta);
    return cudaGetLastError();
}

cudaError_t launch_scan_tc(const DevIndex& ix, int64_t nq, const ScanArgs& sa, const uint16_t* lut_f16,
                           void* scratch, int64_t sum_probe, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    if (!scan_tc_supported(ix, sa.m)) return cudaErrorInvalidValue;
    switch (ix.M) {
        case 32: return launch_tc_t<32>(ix, nq, sa, lut_f16, scratch, sum_probe, st);
        case 64: return launch_tc_t<64>(ix, nq, sa, lut_f16, scratch, sum_probe, st);
        case 128: return launch_tc_t<128>(ix, nq, sa, lut_f16, scratch, sum_probe, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace bbc
