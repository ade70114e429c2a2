// Coarse probe (Section 2, "Quantization": IVF routes each query to the
// n_probe nearest clusters; Algorithm 4 scans them nearest first).
//
// S1  approximate scores  a[q][l] = ||c_l||^2 - 2<q, c_l>   (L2)
//                                   -<q, c_l>                (IP)
//     (||q||^2 is constant per query and dropped.)
// S2  exact selection: the nprobe smallest (FP64 score, list id), nearest
//     first, where the FP64 score is evaluated in ascending dimension order
//     with no fused multiply-add.  Approximate scores only prune and order;
//     FP64 decides wherever the approximations cannot (see the kernel).
#include <cfloat>
#include <algorithm>
#include <cmath>

#include "bbc_internal.cuh"
#include "dev_util.cuh"

namespace bbc {

// ---------------------------------------------------------------------------
// S1: FP32 SIMT scores, 64x64 output tile per CTA, 4x4 per thread.
// ---------------------------------------------------------------------------
constexpr int PT = 64, PK = 32;

__global__ void __launch_bounds__(256) probe_scores_f32_kernel(const float* __restrict__ q, int64_t nq,
                                                                const float* __restrict__ c,
                                                                const float* __restrict__ cnorm,
                                                                int L, int d, int metric,
                                                                float* __restrict__ out) {
    __shared__ float qs[PK][PT + 4];
    __shared__ float cs[PK][PT + 4];
    const int tid = threadIdx.x;
    const int tr = tid >> 4, tc = tid & 15;
    const int64_t q0 = (int64_t)blockIdx.y * PT;
    const int l0 = blockIdx.x * PT;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < d; k0 += PK) {
        for (int i = tid; i < PT * PK; i += 256) {
            int r = i / PK, kk = i % PK;
            int64_t gq = q0 + r;
            int gl = l0 + r, gk = k0 + kk;
            qs[kk][r] = (gq < nq && gk < d) ? q[gq * d + gk] : 0.f;
            cs[kk][r] = (gl < L && gk < d) ? c[(int64_t)gl * d + gk] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < PK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = qs[kk][tr + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = cs[kk][tc + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t gq = q0 + tr + 16 * i;
        if (gq >= nq) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gl = l0 + tc + 16 * j;
            if (gl >= L) continue;
            float s = metric == BBC_METRIC_L2 ? cnorm[gl] - 2.f * acc[i][j] : -acc[i][j];
            out[gq * L + gl] = s;
        }
    }
}

cudaError_t launch_probe_scores(const DevIndex& ix, const float* q, int64_t nq, float* scores,
                                cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    dim3 grid((ix.nlist + PT - 1) / PT, (unsigned)((nq + PT - 1) / PT));
    probe_scores_f32_kernel<<<grid, 256, 0, st>>>(q, nq, ix.centroids, ix.cnorm, ix.nlist, ix.d,
                                                  ix.metric, scores);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// S2: exact selection.
// ---------------------------------------------------------------------------
constexpr int SEL_THREADS = 256;
constexpr int SEL_MAXC = 4096;   // lists re-scored exactly per query

// FP64 score, one rounding per operation, ascending dimension order; the same
// definition the CPU reference evaluates.
__device__ double exact_score(const float* __restrict__ q, const float* __restrict__ c, int d,
                              int metric) {
    double s = 0.0;
    if (metric == BBC_METRIC_L2) {
        for (int i = 0; i < d; ++i) {
            double t = __dsub_rn((double)q[i], (double)c[i]);
            s = __dadd_rn(s, __dmul_rn(t, t));
        }
    } else {
        for (int i = 0; i < d; ++i) s = __dadd_rn(s, __dmul_rn((double)q[i], (double)c[i]));
        s = -s;
    }
    return s;
}

// Double-FP32 ("float-float") helpers: a value is hi + lo with |lo| <= ulp(hi)/2.
// TwoSum and the FMA-based TwoProd are error-free, so sums of exact products
// keep about 44 bits; intrinsics keep the compiler from contracting them.
struct ff { float hi, lo; };
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, err};
}
__device__ __forceinline__ ff ff_add(ff x, ff y) {
    ff s = two_sum(x.hi, y.hi);
    const float lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return two_sum(s.hi, lo);
}
// exact square of a difference of two floats, as a float-float plus residue
__device__ __forceinline__ ff ff_sqdiff(float a, float b) {
    const ff t = two_sum(a, -b);                        // a - b = t.hi + t.lo exactly
    const float p = __fmul_rn(t.hi, t.hi);
    const float pe = __fmaf_rn(t.hi, t.hi, -p);         // t.hi^2 = p + pe exactly
    const float cross = __fmul_rn(__fmul_rn(2.f, t.hi), t.lo);
    return two_sum(p, __fadd_rn(pe, cross));            // drops t.lo^2 (< 2^-48 (a-b)^2)
}
__device__ __forceinline__ ff ff_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// Selection in steps of rising precision: (1) the approximate GEMM scores
// prune to every list that can still reach the nprobe-th; (2) those lists
// are re-scored in FP32 with a rigorous error bound and sorted; lists closer
// than that bound to a neighbour are re-scored in float-float arithmetic
// (about 2^-38 relative) and re-sorted; (3) any run of neighbours whose
// float-float scores are too close to order is re-scored in FP64 and
// re-sorted by (FP64 score, list id).  FP64 is slow on this GPU, so it is
// kept to genuine near-ties.  Every pair outside a run is provably in exact
// order, so the result equals sorting every list by its FP64 score.
__global__ void __launch_bounds__(SEL_THREADS) probe_select_kernel(DevIndex ix, const float* __restrict__ q,
                                                                    QueryParams qp,
                                                                    const float* __restrict__ scores,
                                                                    int32_t* __restrict__ lists, int tc) {
    extern __shared__ unsigned long long psm[];
    const int L = ix.nlist, d = ix.d;
    unsigned long long* ckey = psm;                                  // [SEL_MAXC]
    uint32_t* cval = (uint32_t*)(ckey + SEL_MAXC);                   // [SEL_MAXC]
    uint32_t* keys = cval + SEL_MAXC;                                // [L]
    __shared__ uint32_t hist[256];
    __shared__ uint32_t sc[2];
    __shared__ float red[SEL_THREADS / 32];
    __shared__ uint32_t ncand;
    __shared__ float s_fmax, s_smax;
    __shared__ int s_any;
    __shared__ uint32_t s_thr;
    __shared__ double s_qn, s_eps;   // per-query scalars, computed once (FP64 is slow here)

    const int64_t qi = blockIdx.x;
    const int nprobe = qp.P(qi);
    const float* qv = q + qi * d;
    const float* sv = scores + qi * L;
    for (int l = threadIdx.x; l < L; l += blockDim.x) keys[l] = f32_key(sv[l]);
    // ||q||_2
    float acc = 0.f;
    for (int i = threadIdx.x; i < d; i += blockDim.x) acc = fmaf(qv[i], qv[i], acc);
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if (lane_id() == 0) red[warp_id()] = acc;
    if (threadIdx.x == 0) { ncand = 0; s_fmax = 0.f; s_smax = 0.f; s_any = 0; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float qn2 = 0.f;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) qn2 += red[w];
        s_qn = sqrt((double)qn2);
    }

    // step 1: prune with the approximate scores
    const uint32_t kth = cta_select_u32(L, (uint32_t)(nprobe - 1), [&](int64_t i) { return keys[i]; },
                                        hist, sc, 24);
    // |a - (exact - ||q||^2)| <= eps for the approximate score.
    //  FP32 SIMT GEMM: dot product of length d plus ||c||^2 and the final
    //    subtraction, (d + 4) 2^-24 (||q|| + max||c||)^2, safety factor 4.
    //  Tensor-core GEMM with the 3-term BF16 split: dropped terms
    //    3.1 2^-16 ||q|| ||c||, FP32 accumulation of 3d products
    //    3.06 d 2^-23 ||q|| ||c||, doubled for the factor 2 of the L2 score,
    //    plus ||c||^2 and subtraction rounding; safety factor 2.
    const double cm = (double)ix.cmax;
    if (threadIdx.x == 0) {
        const double qn = s_qn;
        double eps;
        if (!tc) {
            eps = (double)(d + 4) * ldexp(1.0, -22) * (qn + cm) * (qn + cm);
        } else {
            const double rel = 3.1 * ldexp(1.0, -16) + 3.06 * (double)d * ldexp(1.0, -23);
            eps = ix.metric == BBC_METRIC_L2
                      ? 2.0 * (2.0 * rel * qn * cm + ldexp(1.0, -23) * (cm * cm + 2.0 * qn * cm))
                      : 2.0 * (rel * qn * cm + ldexp(1.0, -24) * qn * cm);
        }
        // a float x satisfies x <= thr exactly when x <= thr rounded down to float
        s_thr = f32_key(__double2float_rd((double)key_f32(kth) + 2.0 * eps));
    }
    __syncthreads();
    const double qn = s_qn;
    const uint32_t thr = s_thr;
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
        if (keys[l] <= thr) {
            uint32_t p = atomicAdd(&ncand, 1u);
            if (p < SEL_MAXC) cval[p] = (uint32_t)l;
        }
    }
    __syncthreads();
    int nc = (int)ncand;
    if (nc > SEL_MAXC) {
        if (threadIdx.x == 0) atomicOr(ix.status, kStatusSelectOverrun);
        nc = SEL_MAXC;
    }
    // step 2: FP32 re-score (one warp per list, lanes over dimensions, so
    // centroid rows are read coalesced), then sort by (score, list id).  A
    // term passes through at most nr = ceil(d / 32) + 5 roundings once formed
    // (the fused multiply-add chain of its lane, then the five shuffle-tree
    // additions); forming (q - c)^2 adds 2u + u^2 (u = 2^-24).  So
    //   L2: |fl - s| <= (nr + 3) u s,   IP: |fl - s| <= nr u ||q|| max ||c||,
    // taken with a 2 % margin.
    const int np2 = next_pow2(nc);
    const int nw = blockDim.x / 32;
    for (int i = nc + threadIdx.x; i < np2; i += blockDim.x) {
        ckey[i] = ~0ull;
        cval[i] = 0xFFFFFFFFu;
    }
    for (int i = warp_id(); i < nc; i += nw) {
        const float* cr = ix.centroids + (int64_t)cval[i] * d;
        float acc = 0.f;
        if (ix.metric == BBC_METRIC_L2) {
            for (int j = lane_id(); j < d; j += 32) {
                const float t = __fsub_rn(qv[j], cr[j]);
                acc = __fmaf_rn(t, t, acc);
            }
        } else {
            for (int j = lane_id(); j < d; j += 32) acc = __fmaf_rn(qv[j], cr[j], acc);
        }
        for (int o = 16; o; o >>= 1) acc = __fadd_rn(acc, __shfl_xor_sync(0xFFFFFFFFu, acc, o));
        if (lane_id() == 0) {
            ckey[i] = f64_key_f32(ix.metric == BBC_METRIC_L2 ? acc : -acc);
            if (ix.metric == BBC_METRIC_L2) atomicMax((int*)&s_smax, __float_as_int(acc));   // acc >= 0
        }
    }
    __syncthreads();
    cta_bitonic_kv(ckey, cval, np2);
    if (threadIdx.x == 0) {
        const double u24 = ldexp(1.0, -24);
        const double nr = (double)((d + 31) / 32 + 5);
        s_eps = ix.metric == BBC_METRIC_L2 ? 1.02 * (nr + 3.0) * u24 * (double)s_smax * (1.0 + 16.0 * u24)
                                           : 1.02 * nr * u24 * qn * cm;
    }
    __syncthreads();
    const double eps1 = s_eps;
    // Lists within 2 eps1 of a neighbour are re-scored in float-float
    // arithmetic (about 2^-38 relative), then everything is re-sorted.  The
    // others keep their FP32 score: their order against every other list is
    // already certain, and a float-float score stays within eps1 + its own
    // bound of the FP32 one, so no such pair comes closer than the link bound
    // of step 3.
    uint8_t* link = reinterpret_cast<uint8_t*>(keys);
    for (int i = threadIdx.x; i < nc; i += blockDim.x)
        link[i] = (i + 1 < nc && key_f64(ckey[i + 1]) - key_f64(ckey[i]) <= 2.0 * eps1) ? 1 : 0;
    __syncthreads();
    for (int i = warp_id(); i < nc; i += nw) {
        if (!link[i] && !(i > 0 && link[i - 1])) continue;
        const float* cr = ix.centroids + (int64_t)cval[i] * d;
        ff part = {0.f, 0.f};
        for (int j = lane_id(); j < d; j += 32)
            part = ff_add(part, ix.metric == BBC_METRIC_L2 ? ff_sqdiff(qv[j], cr[j]) : ff_prod(qv[j], cr[j]));
        for (int o = 16; o; o >>= 1) {
            const ff other = {__shfl_xor_sync(0xFFFFFFFFu, part.hi, o), __shfl_xor_sync(0xFFFFFFFFu, part.lo, o)};
            part = ff_add(part, other);
        }
        const double f = ix.metric == BBC_METRIC_L2 ? (double)part.hi + (double)part.lo
                                                    : -((double)part.hi + (double)part.lo);
        if (lane_id() == 0) {
            ckey[i] = f64_key(f);
            atomicMax((int*)&s_fmax, __float_as_int(fabsf(part.hi)));   // non-negative floats order as ints
            s_any = 1;
        }
    }
    __syncthreads();
    if (s_any) cta_bitonic_kv(ckey, cval, np2);
    // step 3: bound on |float-float score - FP64 score|, uniform over the
    // re-scored lists.  Float-float accumulation of d exact (or
    // 2^-47-accurate) terms loses at most about (d + 8) 2^-45 of sum |terms|;
    // the FP64 sequential sum itself is within d 2^-53 of the real value.
    // Safety factor 4.
    //   L2: sum |terms| = the score (max over re-scored lists, +1 ulp for hi);
    //   IP: sum |terms| <= ||q|| max ||c||.
    __syncthreads();
    if (threadIdx.x == 0) {
        const double base = ix.metric == BBC_METRIC_L2 ? (double)s_fmax * (1.0 + ldexp(1.0, -20)) : qn * cm;
        s_eps = 4.0 * ((double)(d + 8) * ldexp(1.0, -45) + (double)d * ldexp(1.0, -53)) * base + 1e-300;
    }
    __syncthreads();
    const double e32 = s_eps;
    // link[i]: lists i and i+1 (in re-score order) are too close to order
    // without FP64.  Flags are computed before any run is rewritten.
    for (int i = threadIdx.x; i < nc; i += blockDim.x)
        link[i] = (i + 1 < nc && key_f64(ckey[i + 1]) - key_f64(ckey[i]) <= 2.0 * e32) ? 1 : 0;
    __syncthreads();
    for (int i = threadIdx.x; i < nc; i += blockDim.x) {
        if ((i == 0 || !link[i - 1]) && link[i]) {
            // run [i, j]: exact FP64 scores, insertion sort by (score, list id)
            int j = i + 1;
            while (j < nc - 1 && link[j]) ++j;
            for (int t = i; t <= j; ++t)
                ckey[t] = f64_key(exact_score(qv, ix.centroids + (int64_t)cval[t] * d, d, ix.metric));
            for (int t = i + 1; t <= j; ++t) {
                const unsigned long long kk = ckey[t];
                const uint32_t vv = cval[t];
                int u = t - 1;
                while (u >= i && (ckey[u] > kk || (ckey[u] == kk && cval[u] > vv))) {
                    ckey[u + 1] = ckey[u];
                    cval[u + 1] = cval[u];
                    --u;
                }
                ckey[u + 1] = kk;
                cval[u + 1] = vv;
            }
        }
    }
    __syncthreads();
    int32_t* lo = lists + qp.poff(qi);
    for (int j = threadIdx.x; j < nprobe; j += blockDim.x) lo[j] = (int32_t)cval[j];
}

cudaError_t launch_probe_select(const DevIndex& ix, const float* q, int64_t nq, const QueryParams& qp,
                                int max_nprobe, const float* scores, int32_t* lists, int tc, cudaStream_t st) {
    (void)max_nprobe;
    if (nq <= 0) return cudaSuccess;
    size_t smem = (size_t)SEL_MAXC * (8 + 4) + (size_t)ix.nlist * 4;
    cudaError_t e = smem_attr_once((const void*)probe_select_kernel, 200 * 1024);
    if (e != cudaSuccess) return e;
    probe_select_kernel<<<(unsigned)nq, SEL_THREADS, smem, st>>>(ix, q, qp, scores, lists, tc);
    return cudaGetLastError();
}

}  // namespace bbc
