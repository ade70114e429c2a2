// S8: exact distances of the collected candidates (the re-rank of Section 2,
// "unbounded methods ... gather n_cand candidates ... which are then
// re-ranked"); S9: the k smallest (distance, id), ascending (Algorithm 4,
// last line).
//
// Re-rank: a group of G lanes gathers one candidate row with 16-byte loads
// (G = row bytes / 16, at most 32) and reduces with shuffles.  Rows come from
// the FP32 vectors, or from the exact u8 copy when every component is an
// integer in [0, 255] (then the FP32 distance is exact: all partial sums are
// integers below 2^24).  Accumulation is FP32.
//
// Top-k: one CTA per query sorts 64-bit keys (order-preserving distance bits
// << 32 | id) in shared memory and writes the first k.
#include <cfloat>

#include "bbc_internal.cuh"
#include "dev_util.cuh"

namespace bbc {

constexpr int RR_THREADS = 256;
constexpr int RR_CAND_PER_CTA = 256;

template <typename T>
__device__ __forceinline__ void add_chunk(const uint4 raw, const float* qv, int metric, float& acc);

template <>
__device__ __forceinline__ void add_chunk<float>(const uint4 raw, const float* qv, int metric, float& acc) {
    const float v[4] = {__uint_as_float(raw.x), __uint_as_float(raw.y), __uint_as_float(raw.z),
                        __uint_as_float(raw.w)};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (metric == BBC_METRIC_L2) {
            const float t = qv[i] - v[i];
            acc = fmaf(t, t, acc);
        } else {
            acc = fmaf(qv[i], v[i], acc);
        }
    }
}

template <>
__device__ __forceinline__ void add_chunk<uint8_t>(const uint4 raw, const float* qv, int metric, float& acc) {
    const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const float v = (float)((w[i >> 2] >> (8 * (i & 3))) & 0xFFu);
        if (metric == BBC_METRIC_L2) {
            const float t = qv[i] - v;
            acc = fmaf(t, t, acc);
        } else {
            acc = fmaf(qv[i], v, acc);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(RR_THREADS) rerank_kernel(DevIndex ix, RerankArgs a, const T* __restrict__ vec) {
    extern __shared__ float rq[];    // query, d floats
    const int d = ix.d;
    const int64_t qi = blockIdx.y;
    for (int i = threadIdx.x; i < d; i += blockDim.x) rq[i] = a.q[qi * d + i];
    __syncthreads();
    const int64_t cnt = a.cand_count[qi];
    const int row_bytes = d * (int)sizeof(T);
    const int nchunk = row_bytes / 16;                 // d * sizeof(T) is a multiple of 16
    int G = 1;                                         // lanes per candidate: a power of two <= 32
    while (G * 2 <= nchunk && G < 32) G *= 2;
    const int per_warp = 32 / G;
    const int ln = (int)lane_id();
    const int grp = ln / G, gl = ln % G;
    const int elems = 16 / (int)sizeof(T);
    const int64_t c0 = (int64_t)blockIdx.x * RR_CAND_PER_CTA;
    const int64_t c1 = min(c0 + RR_CAND_PER_CTA, cnt);
    const uint32_t* cand = a.cand + qi * a.kc;
    float* out = a.cdist + qi * a.kc;
    for (int64_t c = c0 + (int64_t)warp_id() * per_warp + grp; c - grp < c1; c += (int64_t)(blockDim.x / 32) * per_warp) {
        float acc = 0.f;
        const bool live = c < c1;
        const uint32_t id = live ? cand[c] : 0u;
        if (live && (int64_t)id >= ix.n) atomicOr(ix.status, kStatusSelectOverrun);   // never expected
        if (live && (int64_t)id < ix.n) {
            const uint4* row = reinterpret_cast<const uint4*>(vec + (size_t)id * d);
            for (int ch = gl; ch < nchunk; ch += G) add_chunk<T>(__ldg(row + ch), rq + ch * elems, ix.metric, acc);
        }
        for (int o = G >> 1; o; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        if (live && gl == 0) out[c] = ix.metric == BBC_METRIC_L2 ? acc : -acc;
    }
}

cudaError_t launch_rerank(const DevIndex& ix, int64_t nq, const RerankArgs& a, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    dim3 grid((unsigned)((a.kc + RR_CAND_PER_CTA - 1) / RR_CAND_PER_CTA), (unsigned)nq);
    const size_t smem = sizeof(float) * ix.d;
    if (a.use_u8 && ix.vec_u8)
        rerank_kernel<uint8_t><<<grid, RR_THREADS, smem, st>>>(ix, a, ix.vec_u8);
    else
        rerank_kernel<float><<<grid, RR_THREADS, smem, st>>>(ix, a, ix.vectors);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
constexpr int TK_THREADS = 1024;
constexpr int TK_MAX = 16384;    // candidates sorted in shared memory per query

__global__ void __launch_bounds__(TK_THREADS) topk_kernel(DevIndex ix, RerankArgs a) {
    extern __shared__ unsigned long long keys[];   // [np2]
    const int64_t qi = blockIdx.x;
    const int64_t cnt = a.cand_count[qi];
    const int n = (int)(cnt < TK_MAX ? cnt : TK_MAX);
    if (cnt > TK_MAX && threadIdx.x == 0) atomicOr(ix.status, kStatusTopkOverrun);
    const int np2 = next_pow2(n > 1 ? n : 1);
    const uint32_t* cand = a.cand + qi * a.kc;
    const float* cd = a.cdist + qi * a.kc;
    for (int i = threadIdx.x; i < np2; i += blockDim.x)
        keys[i] = i < n ? (((unsigned long long)f32_key(cd[i]) << 32) | cand[i]) : ~0ull;
    __syncthreads();
    cta_bitonic_u64(keys, np2);
    for (int i = threadIdx.x; i < a.k; i += blockDim.x) {
        int64_t id = -1;
        float dv = INFINITY;
        if (i < n) {
            const unsigned long long kk = keys[i];
            id = (int64_t)(kk & 0xFFFFFFFFull);
            dv = key_f32((uint32_t)(kk >> 32));
        }
        a.out_ids[qi * a.k + i] = id;
        a.out_dists[qi * a.k + i] = dv;
    }
}

cudaError_t launch_topk(const DevIndex& ix, int64_t nq, const RerankArgs& a, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    if (a.kc > TK_MAX) return cudaErrorInvalidValue;
    const int np2 = next_pow2((int)(a.kc > 1 ? a.kc : 1));
    const size_t smem = (size_t)np2 * 8;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(topk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             TK_MAX * 8);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    topk_kernel<<<(unsigned)nq, TK_THREADS, smem, st>>>(ix, a);
    return cudaGetLastError();
}

}  // namespace bbc
