// S8: exact distances of the collected candidates (the re-rank of Section 2:
// methods without an error bound collect n_cand candidates by estimated
// distance and compute their exact distances); S9: the k smallest
// (distance, id), ascending (the result Algorithm 4 returns).
//
// Re-rank: a group of G lanes gathers one candidate row with 16-byte loads
// (G = row bytes / 16, at most 32) and reduces with shuffles.  Rows come from
// the FP32 vectors, or from the exact u8 copy when every component is an
// integer in [0, 255] (then the FP32 distance is exact: all partial sums are
// integers below 2^24).  Accumulation is FP32.
//
// Top-k: one CTA per query orders 64-bit keys (order-preserving distance bits
// << 32 | id) with a counting sort into fine distance bins followed by exact
// ranking inside each bin, and writes the first k.
#include <algorithm>
#include <cfloat>

#include "bbc_internal.cuh"
#include "dev_util.cuh"

namespace bbc {

constexpr int RR_THREADS = 256;
constexpr int RR_CAND_PER_CTA = 1024;

// Float accumulation of one 16-byte chunk of a row against the query chunk.
__device__ __forceinline__ void add_chunk_f32(const uint4 raw, const float4 q, int metric, float& acc) {
    const float v[4] = {__uint_as_float(raw.x), __uint_as_float(raw.y), __uint_as_float(raw.z),
                        __uint_as_float(raw.w)};
    const float qq[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (metric == BBC_METRIC_L2) {
            const float t = qq[i] - v[i];
            acc = fmaf(t, t, acc);
        } else {
            acc = fmaf(qq[i], v[i], acc);
        }
    }
}

__device__ __forceinline__ void add_chunk_u8f(const uint4 raw, const float4* q4, int metric, float& acc) {
    const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float4 q = q4[j];
        const float qq[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float v = (float)((w[j] >> (8 * i)) & 0xFFu);
            if (metric == BBC_METRIC_L2) {
                const float t = qq[i] - v;
                acc = fmaf(t, t, acc);
            } else {
                acc = fmaf(qq[i], v, acc);
            }
        }
    }
}

// ||q - v||^2 = ||q||^2 + ||v||^2 - 2 <q, v> for integer rows, rounded once to
// FP32.  The value is below d * 255^2, so for d * 255^2 < 2^32 it is formed
// in 32-bit modular arithmetic and converted from 32 bits (the 64-bit
// integer conversion runs on the slow double-precision pipe of this GPU).
__device__ __forceinline__ float u8_dist(int qn2, unsigned vv, unsigned qv, int d) {
    if (d <= 66051) return __uint2float_rn((unsigned)qn2 + vv - 2u * qv);
    return (float)((long long)qn2 + (long long)vv - 2ll * (long long)qv);
}

// Rows of a fixed shape (G * CPL 16-byte chunks): G lanes per candidate, each
// lane CPL consecutive chunks, the query's chunks held in registers, the
// lane reduction unrolled; four candidates per lane group in flight.
// early (may be null): per candidate, an exact distance the scan already
// computed (Algorithm 4's early re-rank; < 0: none); such rows are not read.
template <typename T, int G, int CPL, bool INT, bool EARLY = false>
__device__ __forceinline__ void rerank_rows(const DevIndex& ix, const T* __restrict__ vec, int d,
                                            const uint32_t* sid, int64_t c0, int64_t c1, float* out,
                                            const float4* q4, const uint4* qb, int qn2,
                                            const float* early = nullptr, unsigned long long* etot = nullptr) {
    constexpr int PW = 32 / G;
    constexpr int U = 4;
    const int ln = (int)lane_id(), grp = ln / G, gl = ln % G;
    const int nwarp = blockDim.x / 32;
    uint4 qq[CPL];
    float4 qf[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
        if (INT) qq[c] = qb[gl * CPL + c];
        else qf[c] = q4[gl * CPL + c];
    }
    for (int64_t cb = c0 + (int64_t)warp_id() * PW * U; cb < c1; cb += (int64_t)nwarp * PW * U) {
        uint32_t id[U];
        bool live[U];
        float ev[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t c = cb + (int64_t)u * PW + grp;
            live[u] = c < c1;
            id[u] = live[u] ? sid[c - c0] : 0u;
            if (live[u] && (int64_t)id[u] >= ix.n) {
                atomicOr(ix.status, kStatusSelectOverrun);   // never expected
                live[u] = false;
            }
            ev[u] = (EARLY && live[u]) ? early[c] : -1.f;
            if (EARLY && ev[u] >= 0.f) live[u] = false;     // scored in the scan: no row to read
        }
        uint4 v[U][CPL];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint4* row = reinterpret_cast<const uint4*>(vec + (size_t)id[u] * d) + gl * CPL;
#pragma unroll
            for (int c = 0; c < CPL; ++c) v[u][c] = live[u] ? __ldg(row + c) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            float dist;
            if (INT) {
                unsigned qv = 0, vv = 0;
#pragma unroll
                for (int c = 0; c < CPL; ++c) {
                    qv = __dp4a(v[u][c].x, qq[c].x, qv); qv = __dp4a(v[u][c].y, qq[c].y, qv);
                    qv = __dp4a(v[u][c].z, qq[c].z, qv); qv = __dp4a(v[u][c].w, qq[c].w, qv);
                    vv = __dp4a(v[u][c].x, v[u][c].x, vv); vv = __dp4a(v[u][c].y, v[u][c].y, vv);
                    vv = __dp4a(v[u][c].z, v[u][c].z, vv); vv = __dp4a(v[u][c].w, v[u][c].w, vv);
                }
#pragma unroll
                for (int o = G >> 1; o; o >>= 1) {
                    qv += __shfl_xor_sync(0xFFFFFFFFu, qv, o);
                    vv += __shfl_xor_sync(0xFFFFFFFFu, vv, o);
                }
                dist = ix.metric == BBC_METRIC_L2 ? u8_dist(qn2, vv, qv, d) : -(float)qv;
            } else {
                float acc = 0.f;
#pragma unroll
                for (int c = 0; c < CPL; ++c) add_chunk_f32(v[u][c], qf[c], ix.metric, acc);
#pragma unroll
                for (int o = G >> 1; o; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
                dist = ix.metric == BBC_METRIC_L2 ? acc : -acc;
            }
            const int64_t c = cb + (int64_t)u * PW + grp;
            if (c < c1 && gl == 0) out[c] = (EARLY && ev[u] >= 0.f) ? ev[u] : dist;
        }
        if (EARLY && etot) {
            unsigned used = 0;
#pragma unroll
            for (int u = 0; u < U; ++u) used += (gl == 0 && ev[u] >= 0.f) ? 1u : 0u;
            used = __reduce_add_sync(0xFFFFFFFFu, used);
            if (lane_id() == 0 && used) atomicAdd(etot, (unsigned long long)used);
        }
    }
}

// Stages one query row for the re-rank: rq = its FP32 components; for u8 rows
// also q8 = the components as bytes, with *s_int cleared unless every
// component is an integer in [0, 255] and *s_qn2 accumulating ||q||^2.  The
// caller sets *s_int = 1 and *s_qn2 = 0 and synchronises before and after.
template <typename T>
__device__ __forceinline__ void rr_stage_query(const float* __restrict__ qrow, int d, float* rq, uint8_t* q8,
                                               int* s_int, int* s_qn2) {
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
        const float v = qrow[i];
        rq[i] = v;
        if (sizeof(T) == 1) {
            const bool ok = v >= 0.f && v <= 255.f && v == floorf(v);
            if (!ok) *s_int = 0;
            q8[i] = ok ? (uint8_t)v : 0;
            if (ok) atomicAdd(s_qn2, (int)v * (int)v);
        }
    }
}

// Exact distances of candidates [c0, c1) of query qi, every thread of the block
// taking part: candidate c has id sid[c - c0] and its distance goes to out[c].
// One group of G lanes per candidate row; rows gathered with 16-byte loads.
// Exact-u8 rows with a query whose components are integers in [0, 255] take
// the integer path: <q, v> and <v, v> with dp4a, ||q - v||^2 = ||q||^2 +
// ||v||^2 - 2 <q, v> in exact integer arithmetic.
// FAST: rows of the two common shapes (128-byte integer rows with an integer
// query, 512-byte FP32 rows) take the fixed-shape path.  Other shapes use the
// FAST = false instantiation, whose general loop then keeps its own register
// allocation and schedule.
template <typename T, bool FAST, bool EARLY>
__device__ __forceinline__ void rr_span(const DevIndex& ix, const RerankArgs& a, int64_t qi, const T* __restrict__ vec,
                                        const uint32_t* sid, int64_t c0, int64_t c1, float* out, const float* rq,
                                        const uint8_t* q8, bool intpath, int qn2) {
    const int d = ix.d;
    const int nchunk = d * (int)sizeof(T) / 16;        // d * sizeof(T) is a multiple of 16
    // the common row shapes: 128-byte integer rows, 512-byte FP32 rows
    if (FAST && sizeof(T) == 1 && intpath && nchunk == 8) {
        if (EARLY)
            rerank_rows<T, 4, 2, true, true>(ix, vec, d, sid, c0, c1, out, reinterpret_cast<const float4*>(rq),
                                             reinterpret_cast<const uint4*>(q8), qn2, a.early + a.qp.coff(qi),
                                             a.early_totals ? a.early_totals + 1 : nullptr);
        else
            rerank_rows<T, 4, 2, true>(ix, vec, d, sid, c0, c1, out, reinterpret_cast<const float4*>(rq),
                                       reinterpret_cast<const uint4*>(q8), qn2);
        return;
    }
    if (FAST && sizeof(T) == 4 && nchunk == 32) {
        rerank_rows<T, 16, 2, false>(ix, vec, d, sid, c0, c1, out, reinterpret_cast<const float4*>(rq),
                                     reinterpret_cast<const uint4*>(q8), qn2);
        return;
    }
    int G = 1;                                         // lanes per candidate: a power of two <= 32
    while (G * 2 <= nchunk && G < 32) G *= 2;
    const int per_warp = 32 / G;
    const int ln = (int)lane_id();
    const int grp = ln / G, gl = ln % G;
    const float4* q4 = reinterpret_cast<const float4*>(rq);
    const uint4* qb = reinterpret_cast<const uint4*>(q8);
    // RR_U candidates per group per step, their row loads issued together
    constexpr int RR_U = 4;
    const int64_t stride = (int64_t)(blockDim.x / 32) * per_warp * RR_U;
    for (int64_t cb = c0 + (int64_t)warp_id() * per_warp * RR_U; cb < c1; cb += stride) {
        uint32_t id[RR_U];
        bool ok[RR_U];
#pragma unroll
        for (int u = 0; u < RR_U; ++u) {
            const int64_t c = cb + (int64_t)u * per_warp + grp;
            const bool live = c < c1;
            id[u] = live ? sid[c - c0] : 0u;
            ok[u] = live && (int64_t)id[u] < ix.n;
            if (live && !ok[u]) atomicOr(ix.status, kStatusSelectOverrun);   // never expected
        }
        float dist[RR_U];
        if (nchunk == G) {
            // one 16-byte chunk per lane and candidate: all loads first
            uint4 v[RR_U];
#pragma unroll
            for (int u = 0; u < RR_U; ++u)
                v[u] = ok[u] ? __ldg(reinterpret_cast<const uint4*>(vec + (size_t)id[u] * d) + gl)
                             : make_uint4(0, 0, 0, 0);
            if (intpath) {
                const uint4 qq = qb[gl];
#pragma unroll
                for (int u = 0; u < RR_U; ++u) {
                    unsigned qv = 0, vv = 0;
                    qv = __dp4a(v[u].x, qq.x, qv); qv = __dp4a(v[u].y, qq.y, qv);
                    qv = __dp4a(v[u].z, qq.z, qv); qv = __dp4a(v[u].w, qq.w, qv);
                    vv = __dp4a(v[u].x, v[u].x, vv); vv = __dp4a(v[u].y, v[u].y, vv);
                    vv = __dp4a(v[u].z, v[u].z, vv); vv = __dp4a(v[u].w, v[u].w, vv);
                    for (int o = G >> 1; o; o >>= 1) {
                        qv += __shfl_xor_sync(0xFFFFFFFFu, qv, o);
                        vv += __shfl_xor_sync(0xFFFFFFFFu, vv, o);
                    }
                    dist[u] = ix.metric == BBC_METRIC_L2
                                  ? u8_dist(qn2, vv, qv, d)
                                  : -(float)qv;
                }
            } else {
#pragma unroll
                for (int u = 0; u < RR_U; ++u) {
                    float acc = 0.f;
                    if (sizeof(T) == 4) add_chunk_f32(v[u], q4[gl], ix.metric, acc);
                    else add_chunk_u8f(v[u], q4 + 4 * gl, ix.metric, acc);
                    for (int o = G >> 1; o; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
                    dist[u] = ix.metric == BBC_METRIC_L2 ? acc : -acc;
                }
            }
        } else {
            // several chunks per lane: loop over the row
#pragma unroll
            for (int u = 0; u < RR_U; ++u) {
                const uint4* row = reinterpret_cast<const uint4*>(vec + (size_t)(ok[u] ? id[u] : 0u) * d);
                if (intpath) {
                    unsigned qv = 0, vv = 0;
                    if (ok[u]) {
                        for (int ch = gl; ch < nchunk; ch += G) {
                            const uint4 v = __ldg(row + ch);
                            const uint4 qq = qb[ch];
                            qv = __dp4a(v.x, qq.x, qv); qv = __dp4a(v.y, qq.y, qv);
                            qv = __dp4a(v.z, qq.z, qv); qv = __dp4a(v.w, qq.w, qv);
                            vv = __dp4a(v.x, v.x, vv); vv = __dp4a(v.y, v.y, vv);
                            vv = __dp4a(v.z, v.z, vv); vv = __dp4a(v.w, v.w, vv);
                        }
                    }
                    for (int o = G >> 1; o; o >>= 1) {
                        qv += __shfl_xor_sync(0xFFFFFFFFu, qv, o);
                        vv += __shfl_xor_sync(0xFFFFFFFFu, vv, o);
                    }
                    dist[u] = ix.metric == BBC_METRIC_L2
                                  ? u8_dist(qn2, vv, qv, d)
                                  : -(float)qv;
                } else {
                    float acc = 0.f;
                    if (ok[u]) {
                        for (int ch = gl; ch < nchunk; ch += G) {
                            const uint4 v = __ldg(row + ch);
                            if (sizeof(T) == 4) add_chunk_f32(v, q4[ch], ix.metric, acc);
                            else add_chunk_u8f(v, q4 + 4 * ch, ix.metric, acc);
                        }
                    }
                    for (int o = G >> 1; o; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
                    dist[u] = ix.metric == BBC_METRIC_L2 ? acc : -acc;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < RR_U; ++u) {
            const int64_t c = cb + (int64_t)u * per_warp + grp;
            if (c < c1 && gl == 0) out[c] = dist[u];
        }
    }
}

// S8 alone: a CTA per (query, RR_CAND_PER_CTA candidates); distances to RerankArgs::cdist.
template <typename T, bool FAST, bool EARLY = false>
__global__ void __launch_bounds__(RR_THREADS) rerank_kernel(DevIndex ix, RerankArgs a, const T* __restrict__ vec) {
    extern __shared__ uint4 rsm[];
    const int d = ix.d;
    float* rq = reinterpret_cast<float*>(rsm);                 // d floats
    uint8_t* q8 = reinterpret_cast<uint8_t*>(rsm + d / 4);     // d bytes (u8 rows only)
    __shared__ int s_int, s_qn2;
    __shared__ uint32_t sid[RR_CAND_PER_CTA];                  // this CTA's candidate ids
    const int64_t qi = blockIdx.y;
    const int64_t cnt = min(a.cand_count[qi], a.qp.KC(qi));
    const int64_t c0 = (int64_t)blockIdx.x * RR_CAND_PER_CTA;
    const int64_t c1 = min(c0 + RR_CAND_PER_CTA, cnt);
    if (threadIdx.x == 0) { s_int = 1; s_qn2 = 0; }
    {
        // ids staged with coalesced loads, so row gathers wait on one latency
        const uint32_t* cp = a.cand + a.qp.coff(qi);
        for (int i = threadIdx.x; i < RR_CAND_PER_CTA; i += blockDim.x)
            sid[i] = c0 + i < cnt ? cp[c0 + i] : 0u;
    }
    __syncthreads();
    rr_stage_query<T>(a.q + qi * d, d, rq, q8, &s_int, &s_qn2);
    __syncthreads();
    rr_span<T, FAST, EARLY>(ix, a, qi, vec, sid, c0, c1, a.cdist + a.qp.coff(qi), rq, q8, sizeof(T) == 1 && s_int,
                            s_qn2);
}

// The early re-rank's slot-ordered copy: one warp per slot copies the u8 row
// of the slot's vector (zero for padding slots) and sums its squares.
__global__ void early_copy_kernel(const uint8_t* __restrict__ vec, const uint32_t* __restrict__ ids, int64_t nslots,
                                  int d, uint8_t* __restrict__ rows, uint32_t* __restrict__ norms) {
    const int64_t slot = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id();
    if (slot >= nslots) return;
    const uint32_t id = ids[slot];
    uint32_t s2 = 0;
    for (int i = (int)lane_id(); i < d; i += 32) {
        const uint8_t v = id == kPadId ? (uint8_t)0 : vec[(int64_t)id * d + i];
        rows[slot * d + i] = v;
        s2 += (uint32_t)v * v;
    }
    s2 = __reduce_add_sync(0xFFFFFFFFu, s2);
    if (lane_id() == 0) norms[slot] = s2;
}

cudaError_t launch_early_copy(const DevIndex& ix, int64_t nslots, uint8_t* rows, uint32_t* norms, cudaStream_t st) {
    if (nslots <= 0) return cudaSuccess;
    if (!ix.vec_u8) return cudaErrorInvalidValue;
    early_copy_kernel<<<(unsigned)((nslots + 7) / 8), 256, 0, st>>>(ix.vec_u8, ix.ids, nslots, ix.d, rows, norms);
    return cudaGetLastError();
}

cudaError_t launch_rerank(const DevIndex& ix, int64_t nq, const RerankArgs& a, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    dim3 grid((unsigned)((a.kc + RR_CAND_PER_CTA - 1) / RR_CAND_PER_CTA), (unsigned)nq);
    const size_t smem = sizeof(float) * ix.d + ix.d + 16;
    // the early re-rank's candidates carry exact distances from the scan: its own instantiation,
    // so the plain kernel keeps its code
    if (a.use_u8 && ix.vec_u8 && a.early)
        rerank_kernel<uint8_t, true, true><<<grid, RR_THREADS, smem, st>>>(ix, a, ix.vec_u8);
    else if (a.use_u8 && ix.vec_u8)
        rerank_kernel<uint8_t, true><<<grid, RR_THREADS, smem, st>>>(ix, a, ix.vec_u8);
    else if (ix.d * 4 == 32 * 16)
        rerank_kernel<float, true><<<grid, RR_THREADS, smem, st>>>(ix, a, ix.vectors);
    else
        rerank_kernel<float, false><<<grid, RR_THREADS, smem, st>>>(ix, a, ix.vectors);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// S9 top-k.  Keys: order-preserving distance bits << 32 | id (unique).  Both
// forms count keys into fine bins in value space, bin = floor((dist - min) *
// bins / (max - min)) evaluated in FP32 -- a monotone function of the
// distance (rounding is monotone) -- scatter them by bin and give each key
// its bin's start plus the number of smaller keys in its bin; bins with many
// keys (many equal distances) are sorted instead.  The constants below belong
// to the form for large k (global scratch); the shared-memory form has its own
// (TKS_*).
constexpr int TK_THREADS = 1024;
constexpr int TK_BINS = 4096;
constexpr int TK_BIG = 2048;
constexpr int TK_HEAVY = 8192;   // a heavy bin of the large top-k sorted in shared memory

__device__ __forceinline__ float tk_scale(float vmin, float vmax) {
    const float range = __fsub_rn(vmax, vmin);
    return range > 0.f ? fminf((float)TK_BINS / range, 3.0e38f) : 0.f;
}
__device__ __forceinline__ uint32_t tk_vbin(float v, float vmin, float scale) {
    const float t = fminf(__fmul_rn(__fsub_rn(v, vmin), scale), (float)(TK_BINS - 1));
    return t > 0.f ? (uint32_t)t : 0u;
}

// Exclusive scan of bins[NB] in place (blockDim.x == THREADS threads, NB =
// PER * THREADS); returns, per thread, the counts of its PER consecutive
// bins in loc.
template <int PER, int THREADS = TK_THREADS>
__device__ __forceinline__ void tk_scan(uint32_t* bins, uint32_t* wsum, uint32_t (&loc)[PER]) {
    const int tid = threadIdx.x;
    uint32_t tot = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) { loc[j] = bins[tid * PER + j]; tot += loc[j]; }
    const uint32_t winc = warp_incl_scan(tot);
    if (lane_id() == 31) wsum[warp_id()] = winc;
    __syncthreads();
    if (warp_id() == 0) {
        const uint32_t v = lane_id() < THREADS / 32 ? wsum[lane_id()] : 0u;
        const uint32_t x = warp_incl_scan(v) - v;
        if (lane_id() < THREADS / 32) wsum[lane_id()] = x;
    }
    __syncthreads();
    uint32_t run = wsum[warp_id()] + winc - tot;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        bins[tid * PER + j] = run;
        run += loc[j];
    }
}

// In-place ascending sort of n 64-bit keys (any n) with a bitonic network
// whose merges all run ascending: the first step of a merge of blocks of size
// kb pairs i with i ^ (kb - 1), the later steps pair i with i ^ j.  Places
// past n then act as +infinity, so their compare-exchanges are skipped.
__device__ void cta_sort_any_u64(unsigned long long* a, int n) {
    const int np2 = next_pow2(n);
    for (int kb = 2; kb <= np2; kb <<= 1) {
        for (int j = kb >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < np2; i += blockDim.x) {
                const int p = j == (kb >> 1) ? (i ^ (kb - 1)) : (i ^ j);
                if (p > i && p < n) {
                    const unsigned long long x = a[i], y = a[p];
                    if (x > y) { a[i] = y; a[p] = x; }
                }
            }
            __syncthreads();
        }
    }
}

// Top-k of any number of candidates when k + TKS_BIG keys fit in shared memory
// (TK_SMEM_KEYS), one CTA per query (two per SM while the keys take half of it).
// 1. min / max of the distances; histogram over BINS bins in value space
//    (bin = floor((dist - min) * BINS / (max - min)) in FP32, a monotone
//    function of the distance); exclusive scan -> bin starts;
// 2. the bin b_k holding rank kk - 1 (kk = min(k, candidates)); when it has
//    more than TKS_BIG keys, the (kk - start)-th smallest key of that bin T
//    (radix select on (distance key << 32 | id));
// 3. keys of the bins below b_k, and of b_k up to T, are scattered into shared
//    memory by bin (at most k - 1 + TKS_BIG keys);
// 4. a key of a bin with at most TKS_BIG keys takes position bin start + the
//    number of smaller keys in its bin; larger bins are sorted in place.
// Positions below k go to the output.
constexpr int TKS_THREADS = 512;
constexpr int TKS_BINS = 2048;
// Bins of the standalone kernel while two CTAs per SM still fit: a key is ranked
// against the other keys of its bin, so finer bins cut that work
constexpr int TKS_BINS_FINE = 4096;
constexpr int TKS_BIG = 1024;
constexpr int TKS_MAXHEAVY = 64;
constexpr int TKS_U = 8;
constexpr int TK_SMEM_KEYS = 24576;   // keys of the shared-memory form: k - 1 + TKS_BIG at most

// The body for query qi, its n candidates' distances cd[] and ids cand[] (in
// global or shared memory), keys[kcap] in shared memory; blockDim.x == THREADS.
template <int THREADS, int U, int BINS>
__device__ __forceinline__ void topk_query(const DevIndex& ix, const RerankArgs& a, int64_t qi, int n,
                                           const float* cd, const uint32_t* cand, unsigned long long* keys,
                                           int kcap) {
    __shared__ uint32_t bins[BINS];
    __shared__ uint32_t wsum[THREADS / 32];
    __shared__ uint32_t hist[256], sc[2];
    __shared__ uint32_t heavy[TKS_MAXHEAVY];
    __shared__ uint32_t s_min, s_max, s_bk, s_nheavy;
    const int tid = threadIdx.x;
    const int kq = a.qp.K(qi);
    int64_t* oid = a.out_ids + a.qp.ooff(qi);
    float* od = a.out_dists + a.qp.ooff(qi);
    for (int i = n + tid; i < kq; i += blockDim.x) { oid[i] = -1; od[i] = INFINITY; }
    if (n == 0 || kq <= 0) return;
    const uint32_t kk = (uint32_t)(kq < n ? kq : n);
    if (tid == 0) { s_min = 0xFFFFFFFFu; s_max = 0u; s_nheavy = 0u; }
    for (int i = tid; i < BINS; i += blockDim.x) bins[i] = 0;
    __syncthreads();
    // passes over the candidates load U values per thread before using them
    const int step = U * THREADS;
    uint32_t mn = 0xFFFFFFFFu, mx = 0u;
    for (int i0 = tid; i0 < n; i0 += step) {
        float v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = i0 + u * THREADS < n ? cd[i0 + u * THREADS] : 0.f;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (i0 + u * THREADS < n) {
                const uint32_t kv = f32_key(v[u]);
                mn = min(mn, kv);
                mx = max(mx, kv);
            }
        }
    }
    mn = __reduce_min_sync(0xFFFFFFFFu, mn);
    mx = __reduce_max_sync(0xFFFFFFFFu, mx);
    if (lane_id() == 0) { atomicMin(&s_min, mn); atomicMax(&s_max, mx); }
    __syncthreads();
    const float vmin = key_f32(s_min);
    const float range = __fsub_rn(key_f32(s_max), vmin);
    const float scale = range > 0.f ? fminf((float)BINS / range, 3.0e38f) : 0.f;
    auto vbin = [&](float v) -> uint32_t {
        const float t = fminf(__fmul_rn(__fsub_rn(v, vmin), scale), (float)(BINS - 1));
        return t > 0.f ? (uint32_t)t : 0u;
    };
    for (int i0 = tid; i0 < n; i0 += step) {
        float v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = i0 + u * THREADS < n ? cd[i0 + u * THREADS] : 0.f;
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i0 + u * THREADS < n) atomicAdd(&bins[vbin(v[u])], 1u);
    }
    __syncthreads();
    constexpr int PER = BINS / THREADS;
    uint32_t loc[PER];
    tk_scan<PER, THREADS>(bins, wsum, loc);
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const uint32_t b = (uint32_t)tid * PER + j;
        const uint32_t st = bins[b];
        if (loc[j] && st <= kk - 1 && kk - 1 < st + loc[j]) s_bk = b;
    }
    __syncthreads();
    const uint32_t bk = s_bk;
    const uint32_t stk = bins[bk];
    const uint32_t nbk = (bk + 1 < (uint32_t)BINS ? bins[bk + 1] : (uint32_t)n) - stk;
    unsigned long long T = ~0ull;
    if (nbk > (uint32_t)TKS_BIG) {
        T = cta_select_u64(n, kk - 1 - stk, [&](int64_t i) {
            const float v = cd[i];
            return vbin(v) == bk ? (((unsigned long long)f32_key(v) << 32) | cand[i]) : ~0ull;
        }, hist, sc, 56);
    }
    for (int i0 = tid; i0 < n; i0 += step) {
        float v[U];
        uint32_t c[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool in = i0 + u * THREADS < n;
            v[u] = in ? cd[i0 + u * THREADS] : 0.f;
            c[u] = in ? cand[i0 + u * THREADS] : 0u;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (i0 + u * THREADS >= n) continue;
            const uint32_t b = vbin(v[u]);
            const unsigned long long key = ((unsigned long long)f32_key(v[u]) << 32) | c[u];
            if (b < bk || (b == bk && key <= T)) {
                const uint32_t p = atomicAdd(&bins[b], 1u);
                if (p < (uint32_t)kcap) keys[p] = key;
                else atomicOr(ix.status, kStatusTopkOverrun);
            }
        }
    }
    __syncthreads();
    // bins[b] now ends bin b (b <= bk); bin b starts at bins[b - 1]
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const uint32_t b = (uint32_t)tid * PER + j;
        if (b <= bk) {
            const uint32_t st = b ? bins[b - 1] : 0u;
            if (bins[b] - st > (uint32_t)TKS_BIG) {
                const uint32_t h = atomicAdd(&s_nheavy, 1u);
                if (h < (uint32_t)TKS_MAXHEAVY) heavy[h] = b;
            }
        }
    }
    const uint32_t nkeep = min(bins[bk], (uint32_t)kcap);
    for (uint32_t p = tid; p < nkeep; p += blockDim.x) {
        const unsigned long long me = keys[p];
        const uint32_t b = vbin(key_f32((uint32_t)(me >> 32)));
        const uint32_t st = b ? bins[b - 1] : 0u;
        const uint32_t en = bins[b];
        if (en - st > (uint32_t)TKS_BIG) continue;                // sorted below
        uint32_t rank = 0;
        for (uint32_t j = st; j < en; ++j) rank += keys[j] < me ? 1u : 0u;
        const uint32_t pos = st + rank;
        if ((int)pos < kq) {
            oid[pos] = (int64_t)(me & 0xFFFFFFFFull);
            od[pos] = key_f32((uint32_t)(me >> 32));
        }
    }
    __syncthreads();
    const uint32_t nh = min(s_nheavy, (uint32_t)TKS_MAXHEAVY);
    if (s_nheavy > (uint32_t)TKS_MAXHEAVY && tid == 0) atomicOr(ix.status, kStatusTopkOverrun);
    for (uint32_t h = 0; h < nh; ++h) {
        const uint32_t b = heavy[h];
        const uint32_t st = b ? bins[b - 1] : 0u;
        const uint32_t en = min(bins[b], (uint32_t)kcap);
        cta_sort_any_u64(keys + st, (int)(en - st));
        for (uint32_t i = st + tid; i < en && (int)i < kq; i += blockDim.x) {
            oid[i] = (int64_t)(keys[i] & 0xFFFFFFFFull);
            od[i] = key_f32((uint32_t)(keys[i] >> 32));
        }
    }
}

template <int BINS>
__global__ void __launch_bounds__(TKS_THREADS, 2) topk_kernel(DevIndex ix, RerankArgs a, int kcap) {
    extern __shared__ unsigned long long keys[];   // [kcap]
    const int64_t qi = blockIdx.x;
    const int n = (int)min(a.cand_count[qi], a.qp.KC(qi));
    topk_query<TKS_THREADS, TKS_U, BINS>(ix, a, qi, n, a.cdist + a.qp.coff(qi), a.cand + a.qp.coff(qi), keys, kcap);
}

// S8 + S9 in one kernel: a CTA per query computes the exact distances of its
// candidates into shared memory (rr_span) and takes their top-k there
// (topk_query), so the distances never travel to global memory and the
// top-k's passes over the candidates read shared memory.  Applies when the
// batch's largest K_c distances and ids and the k - 1 + TKS_BIG kept keys fit
// in one CTA's shared memory (K_c = 15,000 with k = 10,000: 204 KB).  Same
// arithmetic, so the same results, as rerank_kernel followed by topk_kernel.
constexpr int RT_THREADS = 1024;
constexpr int RT_U = 4;
constexpr int RT_SMEM_MAX = 215 * 1024;     // dynamic part; the static part (top-k bins) is under 12 KB

__host__ __device__ inline size_t rt_smem_bytes(long long kcap, long long ncap, int d) {
    return (size_t)((kcap + 1) & ~1ll) * 8 + (size_t)((ncap + 3) & ~3ll) * 8 + (size_t)d * 5;
}

template <typename T, bool FAST, bool EARLY>
__global__ void __launch_bounds__(RT_THREADS, 1)
    rerank_topk_kernel(DevIndex ix, RerankArgs a, const T* __restrict__ vec, int kcap, int ncap) {
    extern __shared__ uint4 fsm[];
    const int d = ix.d;
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(fsm);    // [kcap]
    float* dist = reinterpret_cast<float*>(keys + ((kcap + 1) & ~1));         // [ncap]
    uint32_t* sid = reinterpret_cast<uint32_t*>(dist + ((ncap + 3) & ~3));    // [ncap]
    float* rq = reinterpret_cast<float*>(sid + ((ncap + 3) & ~3));           // d floats (16-byte aligned)
    uint8_t* q8 = reinterpret_cast<uint8_t*>(rq + d);                         // d bytes (u8 rows only)
    __shared__ int s_int, s_qn2;
    const int64_t qi = blockIdx.x;
    int n = (int)min(a.cand_count[qi], a.qp.KC(qi));
    if (n > ncap) {                                                            // never expected
        if (threadIdx.x == 0) atomicOr(ix.status, kStatusTopkOverrun);
        n = ncap;
    }
    if (threadIdx.x == 0) { s_int = 1; s_qn2 = 0; }
    const uint32_t* cp = a.cand + a.qp.coff(qi);
    for (int i = threadIdx.x; i < n; i += blockDim.x) sid[i] = cp[i];
    __syncthreads();
    rr_stage_query<T>(a.q + qi * d, d, rq, q8, &s_int, &s_qn2);
    __syncthreads();
    rr_span<T, FAST, EARLY>(ix, a, qi, vec, sid, 0, n, dist, rq, q8, sizeof(T) == 1 && s_int, s_qn2);
    __syncthreads();
    topk_query<RT_THREADS, RT_U, TKS_BINS>(ix, a, qi, n, dist, sid, keys, kcap);
}

// Same output when k - 1 + TKS_BIG keys do not fit in shared memory.  The
// distance of rank k is found first
// (radix select); only keys at or below it are binned (value space between
// the minimum and that distance) and scattered into a global scratch area
// (RerankArgs::keys, per QueryParams::coff).  Bins of at most TK_BIG keys are
// ranked in place; heavier bins (many equal distances) are sorted one at a
// time in shared memory when they fit TK_HEAVY keys, else ranked in place.
__global__ void __launch_bounds__(TK_THREADS) topk_large_kernel(DevIndex ix, RerankArgs a) {
    extern __shared__ unsigned long long hsm[];       // [TK_HEAVY]
    __shared__ uint32_t bins[TK_BINS];
    __shared__ uint32_t wsum[TK_THREADS / 32];
    __shared__ uint32_t hist[256], sc[2];
    __shared__ uint32_t s_min;
    const int64_t qi = blockIdx.x;
    const int64_t n = min(a.cand_count[qi], a.qp.KC(qi));
    const int tid = threadIdx.x;
    const int kq = a.qp.K(qi);
    const uint32_t* cand = a.cand + a.qp.coff(qi);
    const float* cd = a.cdist + a.qp.coff(qi);
    unsigned long long* keys = a.keys + a.qp.coff(qi);
    int64_t* oid = a.out_ids + a.qp.ooff(qi);
    float* od = a.out_dists + a.qp.ooff(qi);
    for (int64_t i = n + tid; i < kq; i += blockDim.x) { oid[i] = -1; od[i] = INFINITY; }
    if (n == 0) return;
    const int64_t kk = (int64_t)kq < n ? (int64_t)kq : n;
    // distance key of rank kk - 1
    const uint32_t dk = cta_select_u32(n, (uint32_t)(kk - 1), [&](int64_t i) { return f32_key(cd[i]); }, hist, sc, 24);
    if (tid == 0) s_min = 0xFFFFFFFFu;
    for (int i = tid; i < TK_BINS; i += blockDim.x) bins[i] = 0;
    __syncthreads();
    uint32_t mn = 0xFFFFFFFFu;
    for (int64_t i = tid; i < n; i += blockDim.x) mn = min(mn, f32_key(cd[i]));
    mn = __reduce_min_sync(0xFFFFFFFFu, mn);
    if (lane_id() == 0) atomicMin(&s_min, mn);
    __syncthreads();
    const float vmin = key_f32(s_min);
    const float scale = tk_scale(vmin, key_f32(dk));
    for (int64_t i = tid; i < n; i += blockDim.x) {
        const float v = cd[i];
        if (f32_key(v) <= dk) atomicAdd(&bins[tk_vbin(v, vmin, scale)], 1u);
    }
    __syncthreads();
    constexpr int PER = TK_BINS / TK_THREADS;
    uint32_t loc[PER];
    tk_scan<PER>(bins, wsum, loc);
    __syncthreads();
    for (int64_t i = tid; i < n; i += blockDim.x) {
        const float v = cd[i];
        const uint32_t kv = f32_key(v);
        if (kv <= dk) {
            const uint32_t p = atomicAdd(&bins[tk_vbin(v, vmin, scale)], 1u);
            keys[p] = ((unsigned long long)kv << 32) | cand[i];
        }
    }
    __syncthreads();
    const uint32_t upto = bins[TK_BINS - 1];                 // keys at or below the rank-k distance
    for (uint32_t p = tid; p < upto; p += blockDim.x) {
        const unsigned long long me = keys[p];
        const uint32_t b = tk_vbin(key_f32((uint32_t)(me >> 32)), vmin, scale);
        const uint32_t st = b ? bins[b - 1] : 0u;
        const uint32_t en = bins[b];
        if (en - st > (uint32_t)TK_BIG && en - st <= (uint32_t)TK_HEAVY) continue;   // sorted below
        uint32_t rank = 0;
        for (uint32_t j = st; j < en; ++j) rank += keys[j] < me ? 1u : 0u;
        const uint32_t pos = st + rank;
        if ((int64_t)pos < kq) {
            oid[pos] = (int64_t)(me & 0xFFFFFFFFull);
            od[pos] = key_f32((uint32_t)(me >> 32));
        }
    }
    for (int b = 0; b < TK_BINS; ++b) {                     // heavy bins, one at a time
        const uint32_t st = b ? bins[b - 1] : 0u, en = bins[b];
        const uint32_t cntb = en - st;
        if (cntb <= (uint32_t)TK_BIG || cntb > (uint32_t)TK_HEAVY || (int64_t)st >= kq) continue;
        const int np2 = next_pow2((int)cntb);
        __syncthreads();
        for (int i = tid; i < np2; i += blockDim.x) hsm[i] = (uint32_t)i < cntb ? keys[st + i] : ~0ull;
        __syncthreads();
        cta_bitonic_u64(hsm, np2);
        for (uint32_t i = tid; i < cntb && (int64_t)(st + i) < kq; i += blockDim.x) {
            oid[st + i] = (int64_t)(hsm[i] & 0xFFFFFFFFull);
            od[st + i] = key_f32((uint32_t)(hsm[i] >> 32));
        }
    }
}

cudaError_t launch_topk(const DevIndex& ix, int64_t nq, const RerankArgs& a, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    if ((long long)a.k + TKS_BIG > TK_SMEM_KEYS) {
        // the k kept keys do not fit in shared memory: global scratch
        if (!a.keys) return cudaErrorInvalidValue;
        cudaError_t e = smem_attr_once((const void*)topk_large_kernel, TK_HEAVY * 8);
        if (e != cudaSuccess) return e;
        topk_large_kernel<<<(unsigned)nq, TK_THREADS, (size_t)TK_HEAVY * 8, st>>>(ix, a);
        return cudaGetLastError();
    }
    // keys held per query: all candidates, or at most k - 1 + TKS_BIG of them
    const long long kcap = std::min<long long>(a.kc, (long long)a.k + TKS_BIG);
    const size_t smem = (size_t)std::max<long long>(kcap, 1) * 8;
    // the finer bins while two CTAs (keys, bins, 2 KB of the rest and the
    // 1 KB the SM reserves per CTA) fit in 228 KB
    if (2 * (smem + TKS_BINS_FINE * 4 + 3 * 1024) <= 228 * 1024) {
        cudaError_t e = smem_attr_once((const void*)topk_kernel<TKS_BINS_FINE>, TK_SMEM_KEYS * 8);
        if (e != cudaSuccess) return e;
        topk_kernel<TKS_BINS_FINE><<<(unsigned)nq, TKS_THREADS, smem, st>>>(ix, a, (int)std::max<long long>(kcap, 1));
        return cudaGetLastError();
    }
    cudaError_t e = smem_attr_once((const void*)topk_kernel<TKS_BINS>, TK_SMEM_KEYS * 8);
    if (e != cudaSuccess) return e;
    topk_kernel<TKS_BINS><<<(unsigned)nq, TKS_THREADS, smem, st>>>(ix, a, (int)std::max<long long>(kcap, 1));
    return cudaGetLastError();
}

bool rerank_topk_fits(const DevIndex& ix, const RerankArgs& a) {
    if ((long long)a.k + TKS_BIG > TK_SMEM_KEYS) return false;
    const long long kcap = std::max<long long>(std::min<long long>(a.kc, (long long)a.k + TKS_BIG), 1);
    return rt_smem_bytes(kcap, std::max<long long>(a.kc, 1), ix.d) <= (size_t)RT_SMEM_MAX;
}

template <typename T, bool FAST, bool EARLY>
static cudaError_t rt_launch(const DevIndex& ix, int64_t nq, const RerankArgs& a, const T* vec, cudaStream_t st) {
    const long long kcap = std::max<long long>(std::min<long long>(a.kc, (long long)a.k + TKS_BIG), 1);
    const long long ncap = std::max<long long>(a.kc, 1);
    cudaError_t e = smem_attr_once((const void*)rerank_topk_kernel<T, FAST, EARLY>, RT_SMEM_MAX);
    if (e != cudaSuccess) return e;
    rerank_topk_kernel<T, FAST, EARLY><<<(unsigned)nq, RT_THREADS, rt_smem_bytes(kcap, ncap, ix.d), st>>>(
        ix, a, vec, (int)kcap, (int)ncap);
    return cudaGetLastError();
}

cudaError_t launch_rerank_topk(const DevIndex& ix, int64_t nq, const RerankArgs& a, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    if (!rerank_topk_fits(ix, a)) return cudaErrorInvalidValue;
    if (a.use_u8 && ix.vec_u8 && a.early) return rt_launch<uint8_t, true, true>(ix, nq, a, ix.vec_u8, st);
    if (a.use_u8 && ix.vec_u8) return rt_launch<uint8_t, true, false>(ix, nq, a, ix.vec_u8, st);
    if (ix.d * 4 == 32 * 16) return rt_launch<float, true, false>(ix, nq, a, ix.vectors, st);
    return rt_launch<float, false, false>(ix, nq, a, ix.vectors, st);
}

}  // namespace bbc
