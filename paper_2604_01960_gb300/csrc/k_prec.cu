// S8, precision form of the re-rank.
//
// The candidates are first scored from a low-precision copy v~ of the vectors
// (BF16, or FP8-E4M3 with one scale s per vector) in FP32 arithmetic, and each
// score d^ carries a bound rho with |d^ - d64| <= rho, where d64 is the FP64
// distance of the FP32-stored vector (the exact re-rank distance):
//   IP:  rho = ||q|| (e_v + g (||v|| + e_v))
//   L2:  rho = g D + e_v (2 sqrt(D) + e_v),   D = d^ (1 + g)
// with e_v = ||v - v~||_2 and ||v||_2 stored per vector (rounded up), and
// g = 2 n u (u = 2^-24) for a score whose terms go through at most n FP32
// roundings (the sequential chain of a lane, the shuffle tree, the squared
// difference and the final scale).  The factor 2 also covers the second-order
// terms and the rounding of d64 itself.
//
// Classification per query with k results among c > k candidates, using
// lb = d^ - rho and ub = d^ + rho (rounded outwards):
//   certainly in:   ub_v <  L_(k+1), the (k+1)-th smallest lb.  At most k
//                   candidates (v among them) have lb <= ub_v, so fewer than k
//                   can precede v.
//   certainly out:  lb_v >  U_k, the k-th smallest ub.  k candidates are
//                   strictly nearer than v.
//   uncertain:      the rest.  The k - |in| missing members are the nearest
//                   uncertain candidates in exact order.
// The uncertain candidates are re-scored from the FP32 rows with an FP32 bound
// of the same form (rho32 = g32 d32 (1 + g32) for L2, g32 ||q|| ||v|| for IP),
// classified the same way against the k - |in| places, and the rest is decided
// by (d64, id) with d64 computed in FP64 in ascending dimension order.  The
// final set therefore equals the k smallest (d64, id) of the candidates.
// Reported distances: d^ for the certainly-in members (within rho of d64), d32
// for the members placed by the FP32 bound, d64 rounded to FP32 for the rest.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "bbc_internal.cuh"
#include "dev_util.cuh"

namespace bbc {

namespace {

constexpr float kU = 5.9604644775390625e-8f;       // 2^-24
constexpr float kEvalSlack = 1.0f + 3.814697265625e-6f;   // 1 + 2^-18: rounding of the bound itself
constexpr float kTiny = 1.401298464324817e-45f;    // 2^-149: underflow of one product
constexpr int PS_THREADS = 256;
constexpr int PS_CAND_PER_CTA = 1024;
constexpr int PC_THREADS = 512;
constexpr int PR_THREADS = 256;

// Lanes per candidate row: the largest power of two <= 32 dividing nchunk.
__host__ __device__ inline int lanes_for(int nchunk) {
    int G = 1;
    while (G < 32 && nchunk % (2 * G) == 0) G *= 2;
    return G;
}
__host__ __device__ inline int ilog2(int x) {
    int r = 0;
    while ((1 << r) < x) ++r;
    return r;
}

// One E4M3 byte pair -> two floats (exact).
__device__ __forceinline__ float2 e4m3x2_to_f32(uint32_t pair) {
    const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(pair & 0xFFFFu), __NV_E4M3);
    return __half22float2(__half2(h));
}

// ---------------------------------------------------------------------------
// The copy and its per-vector metadata.  One warp per vector.
// ---------------------------------------------------------------------------
__global__ void prec_copy_kernel(const float* __restrict__ v, int64_t n, int d, int dpad, int prec, void* rows,
                                 float4* __restrict__ meta) {
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    const float* row = v + i * d;
    const unsigned ln = lane_id();
    float amax = 0.f;
    for (int j = ln; j < d; j += 32) amax = fmaxf(amax, fabsf(row[j]));
    for (int o = 16; o; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xFFFFFFFFu, amax, o));
    float s = 1.f;
    if (prec == 2) {
        s = __fdiv_rn(amax, 448.f);                 // E4M3's largest finite magnitude
        if (!(s > 0.f) || !isfinite(s)) s = 1.f;
    }
    double e2 = 0.0, n2 = 0.0;
    for (int j = ln; j < dpad; j += 32) {
        const float x = j < d ? row[j] : 0.f;
        double vt;
        if (prec == 2) {
            const __nv_fp8_storage_t c = __nv_cvt_float_to_fp8(__fdiv_rn(x, s), __NV_SATFINITE, __NV_E4M3);
            static_cast<uint8_t*>(rows)[i * dpad + j] = (uint8_t)c;
            const __half_raw hr = __nv_cvt_fp8_to_halfraw(c, __NV_E4M3);
            vt = (double)__half2float(__half(hr)) * (double)s;     // exact: 4 x 24 significant bits
        } else {
            const __nv_bfloat16 b = __float2bfloat16_rn(x);
            static_cast<uint16_t*>(rows)[i * dpad + j] = __bfloat16_as_ushort(b);
            vt = (double)__bfloat162float(b);
        }
        const double df = (double)x - vt;
        e2 += df * df;
        n2 += (double)x * (double)x;
    }
    for (int o = 16; o; o >>= 1) {
        e2 += __shfl_xor_sync(0xFFFFFFFFu, e2, o);
        n2 += __shfl_xor_sync(0xFFFFFFFFu, n2, o);
    }
    if (ln == 0) {
        const float e = e2 > 0.0 ? __double2float_ru(sqrt(e2) * (1.0 + 1e-12)) : 0.f;
        const float nv = __double2float_ru(sqrt(n2) * (1.0 + 1e-12));
        meta[i] = make_float4(s, e, nv, 0.f);
    }
}

// ||q||_2 of the CTA's query in FP64, rounded up to FP32.  All threads call it.
__device__ float cta_qnorm(const float* q, int d, double* red) {
    double t = 0.0;
    for (int j = threadIdx.x; j < d; j += blockDim.x) t += (double)q[j] * (double)q[j];
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
    if (lane_id() == 0) red[warp_id()] = t;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    __syncthreads();
    return __double2float_ru(sqrt(s) * (1.0 + 1e-12));
}

// ---------------------------------------------------------------------------
// Pass 1: low-precision scores and bounds.  G lanes per candidate, 16-byte
// loads, PS_U candidates per group in flight.
// ---------------------------------------------------------------------------
template <int PREC>
__global__ void __launch_bounds__(PS_THREADS) prec_score_kernel(DevIndex ix, RerankArgs a, PrecArgs p) {
    extern __shared__ float4 psm[];
    float* sq = reinterpret_cast<float*>(psm);             // dpad floats, zero beyond d
    __shared__ double red[PS_THREADS / 32];
    const int d = ix.d, dpad = ix.dpad;
    const int64_t qi = blockIdx.y;
    const float* q = a.q + qi * d;
    for (int j = threadIdx.x; j < dpad; j += blockDim.x) sq[j] = j < d ? q[j] : 0.f;
    const float qn = cta_qnorm(q, d, red);                  // contains __syncthreads
    if (p.qnorm && blockIdx.x == 0 && threadIdx.x == 0) p.qnorm[qi] = qn;
    constexpr int ES = PREC == 1 ? 2 : 1;                   // bytes per element
    constexpr int E = 16 / ES;                              // elements per 16-byte chunk
    const int nchunk = dpad * ES / 16;
    const int G = lanes_for(nchunk);
    const int per_lane = nchunk / G;
    const float g = 2.f * (float)(per_lane * E + ilog2(G) + 3) * kU;
    const bool l2 = ix.metric == BBC_METRIC_L2;
    const int64_t cnt = min(a.cand_count[qi], a.qp.KC(qi));
    const int ln = (int)lane_id(), grp = ln / G, gl = ln % G, per_warp = 32 / G;
    const int64_t c0 = (p.sc_from ? p.sc_from[qi] : 0) + (int64_t)blockIdx.x * PS_CAND_PER_CTA;
    const int64_t c1 = min(c0 + PS_CAND_PER_CTA, cnt);
    const uint32_t* cand = a.cand + a.qp.coff(qi);
    float* out = a.cdist + a.qp.coff(qi);
    float* rho = p.rho + a.qp.coff(qi);
    const uint4* rows = static_cast<const uint4*>(ix.vec_lp);
    const int rstride = nchunk;                             // uint4 per row
    constexpr int PS_U = 4;
    const int64_t stride = (int64_t)(blockDim.x >> 5) * per_warp * PS_U;
    for (int64_t cb = c0 + (int64_t)warp_id() * per_warp * PS_U; cb < c1; cb += stride) {
        uint32_t id[PS_U];
        bool ok[PS_U];
#pragma unroll
        for (int u = 0; u < PS_U; ++u) {
            const int64_t c = cb + (int64_t)u * per_warp + grp;
            const bool live = c < c1;
            id[u] = live ? cand[c] : 0u;
            ok[u] = live && (int64_t)id[u] < ix.n;
            if (live && !ok[u]) atomicOr(ix.status, kStatusSelectOverrun);   // never expected
        }
        float4 mt[PS_U];
#pragma unroll
        for (int u = 0; u < PS_U; ++u) mt[u] = ok[u] ? __ldg(ix.vec_meta + id[u]) : make_float4(1.f, 0.f, 0.f, 0.f);
        float acc[PS_U];
#pragma unroll
        for (int u = 0; u < PS_U; ++u) acc[u] = 0.f;
        for (int ch0 = 0; ch0 < per_lane; ++ch0) {
            const int ch = ch0 * G + gl;
            uint4 raw[PS_U];
#pragma unroll
            for (int u = 0; u < PS_U; ++u)
                raw[u] = ok[u] ? __ldg(rows + (size_t)id[u] * rstride + ch) : make_uint4(0, 0, 0, 0);
            const float* qc = sq + ch * E;
#pragma unroll
            for (int u = 0; u < PS_U; ++u) {
                const uint32_t w[4] = {raw[u].x, raw[u].y, raw[u].z, raw[u].w};
                if (PREC == 1) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float v0 = __uint_as_float(w[k] << 16);
                        const float v1 = __uint_as_float(w[k] & 0xFFFF0000u);
                        if (l2) {
                            const float t0 = qc[2 * k] - v0, t1 = qc[2 * k + 1] - v1;
                            acc[u] = fmaf(t0, t0, acc[u]);
                            acc[u] = fmaf(t1, t1, acc[u]);
                        } else {
                            acc[u] = fmaf(qc[2 * k], v0, acc[u]);
                            acc[u] = fmaf(qc[2 * k + 1], v1, acc[u]);
                        }
                    }
                } else {
                    const float ns = -mt[u].x;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float2 a01 = e4m3x2_to_f32(w[k]);
                        const float2 a23 = e4m3x2_to_f32(w[k] >> 16);
                        const float vv[4] = {a01.x, a01.y, a23.x, a23.y};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            if (l2) {
                                const float t = fmaf(ns, vv[e], qc[4 * k + e]);    // q - s h, one rounding
                                acc[u] = fmaf(t, t, acc[u]);
                            } else {
                                acc[u] = fmaf(qc[4 * k + e], vv[e], acc[u]);
                            }
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < PS_U; ++u) {
            for (int o = G >> 1; o; o >>= 1) acc[u] += __shfl_xor_sync(0xFFFFFFFFu, acc[u], o);
            const int64_t c = cb + (int64_t)u * per_warp + grp;
            if (c < c1 && gl == 0) {
                const float s = PREC == 2 ? mt[u].x : 1.f;
                const float e = mt[u].y, nv = mt[u].z;
                float dist, r;
                if (l2) {
                    dist = acc[u];
                    const float D = acc[u] * (1.f + g);
                    r = g * D + e * (2.f * sqrtf(D) + e);
                } else {
                    const float ip = PREC == 2 ? acc[u] * s : acc[u];
                    dist = -ip;
                    r = qn * (e + g * (nv + e));
                }
                r = r * kEvalSlack + (float)(d + 2) * kTiny * fmaxf(s, 1.f) * (1.f + qn);
                out[c] = dist;
                rho[c] = r;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Two CTA-wide selections in one sweep: the r1-th smallest of the .x keys and
// the r2-th smallest of the .y keys that get(i) returns for the same n items
// (u32 keys, 8-bit digits).  hist: 512 u32 in shared memory; sc: 4 u32.
// ---------------------------------------------------------------------------
template <typename Get>
__device__ void cta_select2_u32(int64_t n, uint32_t r1, uint32_t r2, Get get, uint32_t* hist, uint32_t* sc,
                                uint32_t& out1, uint32_t& out2) {
    uint32_t p1 = 0, p2 = 0, mask = 0;
    for (int sh = 24; sh >= 0; sh -= 8) {
        for (int i = threadIdx.x; i < 512; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        const int64_t bs = blockDim.x;
        for (int64_t i = threadIdx.x; i < n; i += 4 * bs) {
            uint2 k[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) k[u] = i + u * bs < n ? get(i + u * bs) : make_uint2(0u, 0u);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (i + u * bs < n) {
                    if ((k[u].x & mask) == p1) atomicAdd(&hist[(k[u].x >> sh) & 255u], 1u);
                    if ((k[u].y & mask) == p2) atomicAdd(&hist[256 + ((k[u].y >> sh) & 255u)], 1u);
                }
            }
        }
        __syncthreads();
        if (warp_id() == 0) warp_find_digit(hist, r1, &sc[0], &sc[1]);
        if (warp_id() == 1) warp_find_digit(hist + 256, r2, &sc[2], &sc[3]);
        __syncthreads();
        p1 |= sc[0] << sh;
        p2 |= sc[2] << sh;
        mask |= 255u << sh;
        r1 = sc[1];
        r2 = sc[3];
        __syncthreads();
    }
    out1 = p1;
    out2 = p2;
}

// Keys of the bounds: x = ub (rounded up), y = lb (rounded down).
__device__ __forceinline__ uint2 bound_keys(float dist, float r) {
    return make_uint2(f32_key(__fadd_ru(dist, r)), f32_key(__fsub_rd(dist, r)));
}

// Warp-aggregated append to a shared counter; returns this lane's slot.  All
// lanes of the warp call it.
__device__ __forceinline__ uint32_t warp_append(bool take, uint32_t* counter) {
    const unsigned m = __ballot_sync(0xFFFFFFFFu, take);
    const unsigned ln = lane_id();
    const int leader = m ? __ffs(m) - 1 : 0;
    uint32_t base = 0;
    if (m && (int)ln == leader) base = atomicAdd(counter, (uint32_t)__popc(m));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    return base + __popc(m & ((1u << ln) - 1u));
}

// ---------------------------------------------------------------------------
// Pass 2: classification of the low-precision scores (one CTA per query).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(PC_THREADS) prec_classify_kernel(DevIndex ix, RerankArgs a, PrecArgs p) {
    __shared__ uint32_t hist[512];
    __shared__ uint32_t sc[4];
    __shared__ uint32_t s_in, s_unc;
    const int64_t qi = blockIdx.x;
    const int64_t cnt = min(a.cand_count[qi], a.qp.KC(qi));
    const int64_t kq = a.qp.K(qi);
    const int64_t off = a.qp.coff(qi);
    const uint32_t* cand = a.cand + off;
    const float* dh = a.cdist + off;
    const float* rho = p.rho + off;
    if (threadIdx.x == 0) { s_in = 0; s_unc = 0; }
    __syncthreads();
    uint32_t Uk = 0xFFFFFFFFu, Lk1 = 0u;
    const bool all_in = cnt <= kq;
    if (!all_in) {
        auto get = [&](int64_t i) { return bound_keys(dh[i], rho[i]); };
        cta_select2_u32(cnt, (uint32_t)(kq - 1), (uint32_t)kq, get, hist, sc, Uk, Lk1);
    }
    const int64_t n_pad = (cnt + 31) / 32 * 32;           // whole warps through the ballots
    for (int64_t i = threadIdx.x; i < n_pad; i += blockDim.x) {
        bool in = false, unc = false;
        uint32_t id = 0;
        float dist = 0.f;
        if (i < cnt) {
            id = cand[i];
            dist = dh[i];
            if (all_in) {
                in = true;
            } else {
                const uint2 k = bound_keys(dist, rho[i]);
                in = k.x < Lk1;
                unc = !in && !(k.y > Uk);
            }
            if ((int64_t)id >= ix.n) { in = false; unc = false; }   // invalid id (latched by pass 1)
        }
        const uint32_t si = warp_append(in, &s_in);
        if (in) { p.fin_id[off + si] = id; p.fin_d[off + si] = dist; }
        const uint32_t su = warp_append(unc, &s_unc);
        if (unc) {
            p.unc[off + su] = id;
            if (p.copy_unc) { p.unc_d[off + su] = dist; p.unc_r[off + su] = rho[i]; }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        p.n_fin[qi] = s_in;
        p.n_unc[qi] = s_unc;
        atomicAdd(&p.totals[0], (unsigned long long)cnt);
        atomicAdd(&p.totals[1], (unsigned long long)s_unc);
    }
}

// Recheck work items: item_off[q + 1] - item_off[q] = ceil((rc_count[q] - rc_from[q]) / kPrecItem).
__global__ void __launch_bounds__(1024) prec_plan_kernel(int64_t nq, PrecArgs p) {
    __shared__ unsigned long long wsum[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) { carry = 0; p.item_off[0] = 0; }
    __syncthreads();
    for (int64_t base = 0; base < nq; base += blockDim.x) {
        const int64_t q = base + threadIdx.x;
        const int64_t span = q < nq ? p.rc_count[q] - (p.rc_from ? p.rc_from[q] : 0) : 0;
        const unsigned long long v = span > 0 ? (unsigned long long)((span + kPrecItem - 1) / kPrecItem) : 0ull;
        const unsigned long long inc = warp_incl_scan64(v);
        if (lane_id() == 31) wsum[warp_id()] = inc;
        __syncthreads();
        if (warp_id() == 0) {
            const unsigned long long w = wsum[lane_id()];
            wsum[lane_id()] = warp_incl_scan64(w) - w;
        }
        __syncthreads();
        const unsigned long long tot = carry + wsum[warp_id()] + inc;
        if (q < nq) p.item_off[q + 1] = (int64_t)tot;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = tot;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Pass 3: FP32 recheck.  Persistent CTAs over the (query, item) work list of
// positions [rc_from, rc_count) of rc_ids; d32 and rho32 go to rc_d / rc_r at
// the same positions.  (Precision path: the uncertain list, written over the
// dead pass-1 scores; bounded re-rank: the candidate list of each round.)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(PR_THREADS) prec_recheck_kernel(DevIndex ix, int64_t nq, RerankArgs a,
                                                                  PrecArgs p) {
    extern __shared__ float4 rsm4[];
    float* sq = reinterpret_cast<float*>(rsm4);
    __shared__ int64_t s_q;
    const int d = ix.d;
    const int nchunk = d / 4;
    const int G = lanes_for(nchunk);
    const int per_lane = nchunk / G;
    const float g = 2.f * (float)(per_lane * 4 + ilog2(G) + 3) * kU;
    const bool l2 = ix.metric == BBC_METRIC_L2;
    const int ln = (int)lane_id(), grp = ln / G, gl = ln % G, per_warp = 32 / G;
    const int64_t total = p.item_off[nq];
    const uint4* rows = reinterpret_cast<const uint4*>(ix.vectors);
    for (int64_t it = blockIdx.x; it < total; it += gridDim.x) {
        if (threadIdx.x == 0) {
            int64_t lo = 0, hi = nq - 1;                    // last q with item_off[q] <= it
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (p.item_off[mid] <= it) lo = mid; else hi = mid - 1;
            }
            s_q = lo;
        }
        __syncthreads();
        const int64_t qi = s_q;
        for (int j = threadIdx.x; j < d; j += blockDim.x) sq[j] = a.q[qi * d + j];
        __syncthreads();
        const float qn = p.qnorm[qi];
        const int64_t off = a.qp.coff(qi);
        const int64_t from = p.rc_from ? p.rc_from[qi] : 0;
        const int64_t c0 = from + (it - p.item_off[qi]) * kPrecItem;
        const int64_t c1 = min(c0 + kPrecItem, p.rc_count[qi]);
        const float4* q4 = reinterpret_cast<const float4*>(sq);
        constexpr int PU = 4;
        const int64_t stride = (int64_t)(blockDim.x >> 5) * per_warp * PU;
        for (int64_t cb = c0 + (int64_t)warp_id() * per_warp * PU; cb < c1; cb += stride) {
            uint32_t id[PU];
            bool ok[PU];
#pragma unroll
            for (int u = 0; u < PU; ++u) {
                const int64_t c = cb + (int64_t)u * per_warp + grp;
                ok[u] = c < c1;
                id[u] = ok[u] ? p.rc_ids[off + c] : 0u;
                if (ok[u] && (int64_t)id[u] >= ix.n) { ok[u] = false; atomicOr(ix.status, kStatusSelectOverrun); }
            }
            float acc[PU];
#pragma unroll
            for (int u = 0; u < PU; ++u) acc[u] = 0.f;
            for (int ch0 = 0; ch0 < per_lane; ++ch0) {
                const int ch = ch0 * G + gl;
                uint4 raw[PU];
#pragma unroll
                for (int u = 0; u < PU; ++u)
                    raw[u] = ok[u] ? __ldg(rows + (size_t)id[u] * nchunk + ch) : make_uint4(0, 0, 0, 0);
                const float4 qq = q4[ch];
#pragma unroll
                for (int u = 0; u < PU; ++u) {
                    const float v[4] = {__uint_as_float(raw[u].x), __uint_as_float(raw[u].y),
                                        __uint_as_float(raw[u].z), __uint_as_float(raw[u].w)};
                    const float qv[4] = {qq.x, qq.y, qq.z, qq.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (l2) {
                            const float t = qv[e] - v[e];
                            acc[u] = fmaf(t, t, acc[u]);
                        } else {
                            acc[u] = fmaf(qv[e], v[e], acc[u]);
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < PU; ++u) {
                for (int o = G >> 1; o; o >>= 1) acc[u] += __shfl_xor_sync(0xFFFFFFFFu, acc[u], o);
                const int64_t c = cb + (int64_t)u * per_warp + grp;
                if (ok[u] && gl == 0) {
                    float dist, r;
                    if (l2) {
                        dist = acc[u];
                        r = g * acc[u] * (1.f + g);
                    } else {
                        dist = -acc[u];
                        r = g * qn * __ldg(&ix.vec_meta[id[u]].z);
                    }
                    p.rc_d[off + c] = dist;
                    p.rc_r[off + c] = r * kEvalSlack + (float)(d + 2) * kTiny * (1.f + qn);
                }
            }
        }
        __syncthreads();
    }
}

// FP64 distance in ascending dimension order, without contraction.
__device__ double exact64(const float* q, const float* v, int d, bool l2) {
    double s = 0.0;
    if (l2) {
        for (int i = 0; i < d; ++i) {
            const double t = __dsub_rn((double)q[i], (double)__ldg(v + i));
            s = __dadd_rn(s, __dmul_rn(t, t));
        }
        return s;
    }
    for (int i = 0; i < d; ++i) s = __dadd_rn(s, __dmul_rn((double)q[i], (double)__ldg(v + i)));
    return -s;
}

// ---------------------------------------------------------------------------
// Pass 4: FP32 classification of the uncertain candidates against the
// remaining places, FP64 decision of the rest (one CTA per query).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(PC_THREADS) prec_finalize_kernel(DevIndex ix, RerankArgs a, PrecArgs p) {
    __shared__ uint32_t hist[512];
    __shared__ uint32_t sc[4];
    __shared__ uint32_t s_fin, s_band, s_lt, s_eq;
    const int64_t qi = blockIdx.x;
    const int d = ix.d;
    const bool l2 = ix.metric == BBC_METRIC_L2;
    const int64_t cnt = min(a.cand_count[qi], a.qp.KC(qi));
    const int64_t kq = a.qp.K(qi);
    const int64_t kk = cnt < kq ? cnt : kq;
    const int64_t off = a.qp.coff(qi);
    const int64_t nin = p.n_fin[qi];
    const int64_t nu = p.n_unc[qi];
    const int64_t need = kk - nin;
    const uint32_t* unc = p.unc + off;
    const float* d32 = p.unc_d + off;
    const float* r32 = p.unc_r + off;
    uint32_t* fid = p.fin_id + off;
    float* fdist = p.fin_d + off;
    if (threadIdx.x == 0) { s_fin = (uint32_t)nin; s_band = 0; s_lt = 0; s_eq = 0; }
    __syncthreads();
    if (need <= 0) {
        if (threadIdx.x == 0) atomicAdd(&p.totals[3], (unsigned long long)nin);
        return;
    }
    if (nu < need) {                                        // a bound was wrong: cannot happen
        if (threadIdx.x == 0) atomicOr(ix.status, kStatusPrecBound);
        return;
    }
    const float* q = a.q + qi * d;
    uint32_t* bid = p.band_id + off;
    double* bd = p.band_d + off;
    uint32_t Up = 0xFFFFFFFFu, Lp = 0u;
    const bool all_in = nu == need;
    if (!all_in) {
        auto get = [&](int64_t i) { return bound_keys(d32[i], r32[i]); };
        cta_select2_u32(nu, (uint32_t)(need - 1), (uint32_t)need, get, hist, sc, Up, Lp);
    }
    const int64_t n_pad = (nu + 31) / 32 * 32;
    for (int64_t i = threadIdx.x; i < n_pad; i += blockDim.x) {
        bool in = false, band = false;
        uint32_t id = 0;
        float dist = 0.f;
        if (i < nu) {
            id = unc[i];
            dist = d32[i];
            if (all_in) {
                in = true;
            } else {
                const uint2 k = bound_keys(dist, r32[i]);
                in = k.x < Lp;
                band = !in && !(k.y > Up);
            }
        }
        const uint32_t si = warp_append(in, &s_fin);
        if (in) { fid[si] = id; fdist[si] = dist; }
        const uint32_t sb = warp_append(band, &s_band);
        if (band) bid[sb] = id;
    }
    __syncthreads();
    const int64_t nb = s_band;
    const int64_t take = nin + need - (int64_t)s_fin;       // band members still to place
    if (take > nb) {                                        // a bound was wrong: cannot happen
        if (threadIdx.x == 0) atomicOr(ix.status, kStatusPrecBound);
        return;
    }
    for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) bd[b] = exact64(q, ix.vectors + (size_t)bid[b] * d, d, l2);
    __syncthreads();
    if (take > 0) {
        // the take smallest (d64, id): cut key, then ids among the members equal to it
        unsigned long long kcut = ~0ull;
        uint32_t idcut = 0xFFFFFFFFu;
        if (take < nb) {
            kcut = cta_select_u64(nb, (uint32_t)(take - 1), [&](int64_t i) { return f64_key(bd[i]); }, hist, sc, 56);
            for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) {
                const unsigned long long kb = f64_key(bd[b]);
                if (kb < kcut) atomicAdd(&s_lt, 1u);
                else if (kb == kcut) atomicAdd(&s_eq, 1u);
            }
            __syncthreads();
            const uint32_t want = (uint32_t)(take - s_lt);  // members equal to the cut that are taken
            if (want < s_eq)
                idcut = cta_select_u32(nb, want - 1,
                                       [&](int64_t i) { return f64_key(bd[i]) == kcut ? bid[i] : 0xFFFFFFFFu; },
                                       hist, sc, 24);
        }
        const int64_t nb_pad = (nb + 31) / 32 * 32;
        for (int64_t b = threadIdx.x; b < nb_pad; b += blockDim.x) {
            bool t = false;
            if (b < nb) {
                const unsigned long long kb = f64_key(bd[b]);
                t = kb < kcut || (kb == kcut && bid[b] <= idcut);
            }
            const uint32_t si = warp_append(t, &s_fin);
            if (t) { fid[si] = bid[b]; fdist[si] = (float)bd[b]; }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if ((int64_t)s_fin != kk) atomicOr(ix.status, kStatusPrecBound);
        p.n_fin[qi] = s_fin;
        atomicAdd(&p.totals[2], (unsigned long long)nb);
        atomicAdd(&p.totals[3], (unsigned long long)s_fin);
    }
}

}  // namespace

cudaError_t launch_prec_copy(const DevIndex& ix, int prec, void* rows, float4* meta, cudaStream_t st) {
    if (prec != 1 && prec != 2) return cudaErrorInvalidValue;
    const int wpb = 8;
    const unsigned grid = (unsigned)((ix.n + wpb - 1) / wpb);
    prec_copy_kernel<<<grid, 32 * wpb, 0, st>>>(ix.vectors, ix.n, ix.d, ix.dpad, prec, rows, meta);
    return cudaGetLastError();
}

cudaError_t launch_prec_score(const DevIndex& ix, int64_t nq, const RerankArgs& a, const PrecArgs& p,
                              cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    if (!ix.vec_lp || !ix.vec_meta) return cudaErrorInvalidValue;
    dim3 grid((unsigned)std::max<int64_t>(1, (a.kc + PS_CAND_PER_CTA - 1) / PS_CAND_PER_CTA), (unsigned)nq);
    const size_t smem = (size_t)ix.dpad * sizeof(float);
    if (ix.prec == 1) prec_score_kernel<1><<<grid, PS_THREADS, smem, st>>>(ix, a, p);
    else if (ix.prec == 2) prec_score_kernel<2><<<grid, PS_THREADS, smem, st>>>(ix, a, p);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_prec_classify(const DevIndex& ix, int64_t nq, const RerankArgs& a, const PrecArgs& p,
                                 cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    prec_classify_kernel<<<(unsigned)nq, PC_THREADS, 0, st>>>(ix, a, p);
    return cudaGetLastError();
}

cudaError_t launch_prec_plan(int64_t nq, const PrecArgs& p, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    prec_plan_kernel<<<1, 1024, 0, st>>>(nq, p);
    return cudaGetLastError();
}

cudaError_t launch_prec_recheck(const DevIndex& ix, int64_t nq, const RerankArgs& a, const PrecArgs& p,
                                cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)(4 * std::max(1, ix.num_sms));
    prec_recheck_kernel<<<grid, PR_THREADS, (size_t)ix.d * sizeof(float), st>>>(ix, nq, a, p);
    return cudaGetLastError();
}

cudaError_t launch_prec_finalize(const DevIndex& ix, int64_t nq, const RerankArgs& a, const PrecArgs& p,
                                 cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    prec_finalize_kernel<<<(unsigned)nq, PC_THREADS, 0, st>>>(ix, a, p);
    return cudaGetLastError();
}

}  // namespace bbc
