// Coarse probe (Section 2, "Quantization": IVF routes each query to the
// n_probe nearest clusters; Algorithm 4 scans them nearest first).
//
// S1  approximate scores  a[q][l] = ||c_l||^2 - 2<q, c_l>   (L2)
//                                   -<q, c_l>                (IP)
//     (||q||^2 is constant per query and dropped.)
// S2  exact selection: every list whose approximate score can still reach
//     the nprobe-th is re-scored exactly in FP64 (ascending dimension order,
//     no fused multiply-add), and the nprobe smallest (FP64 score, list id)
//     are written nearest first.  The approximate scores only prune.
#include <cfloat>
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

__global__ void __launch_bounds__(SEL_THREADS) probe_select_kernel(DevIndex ix, const float* __restrict__ q,
                                                                    int nprobe,
                                                                    const float* __restrict__ scores,
                                                                    int32_t* __restrict__ lists) {
    extern __shared__ unsigned long long psm[];
    const int L = ix.nlist, d = ix.d;
    unsigned long long* ckey = psm;                                  // [SEL_MAXC]
    uint32_t* cval = (uint32_t*)(ckey + SEL_MAXC);                   // [SEL_MAXC]
    uint32_t* keys = cval + SEL_MAXC;                                // [L]
    __shared__ uint32_t hist[256];
    __shared__ uint32_t sc[2];
    __shared__ float red[SEL_THREADS / 32];
    __shared__ uint32_t ncand;

    const int64_t qi = blockIdx.x;
    const float* qv = q + qi * d;
    const float* sv = scores + qi * L;
    for (int l = threadIdx.x; l < L; l += blockDim.x) keys[l] = f32_key(sv[l]);
    // ||q||_2
    float acc = 0.f;
    for (int i = threadIdx.x; i < d; i += blockDim.x) acc = fmaf(qv[i], qv[i], acc);
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if (lane_id() == 0) red[warp_id()] = acc;
    if (threadIdx.x == 0) ncand = 0;
    __syncthreads();
    float qn2 = 0.f;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) qn2 += red[w];
    const double qn = sqrt((double)qn2);

    const uint32_t kth = cta_select_u32(L, (uint32_t)(nprobe - 1), [&](int64_t i) { return keys[i]; },
                                        hist, sc, 24);
    // |a - (exact - ||q||^2)| <= eps for the FP32 score (dot product of length d
    // plus ||c||^2 and the final subtraction), with a safety factor of 4.
    const double cm = (double)ix.cmax;
    const double eps = (double)(d + 4) * ldexp(1.0, -22) * (qn + cm) * (qn + cm);
    const double thr = (double)key_f32(kth) + 2.0 * eps;
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
        if ((double)key_f32(keys[l]) <= thr) {
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
    for (int i = threadIdx.x; i < nc; i += blockDim.x) {
        uint32_t l = cval[i];
        ckey[i] = f64_key(exact_score(qv, ix.centroids + (int64_t)l * d, d, ix.metric));
    }
    const int np2 = next_pow2(nc);
    for (int i = nc + threadIdx.x; i < np2; i += blockDim.x) {
        ckey[i] = ~0ull;
        cval[i] = 0xFFFFFFFFu;
    }
    __syncthreads();
    cta_bitonic_kv(ckey, cval, np2);
    for (int j = threadIdx.x; j < nprobe; j += blockDim.x) lists[qi * nprobe + j] = (int32_t)cval[j];
}

cudaError_t launch_probe_select(const DevIndex& ix, const float* q, int64_t nq, int nprobe,
                                const float* scores, int32_t* lists, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    size_t smem = (size_t)SEL_MAXC * (8 + 4) + (size_t)ix.nlist * 4;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(probe_select_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    probe_select_kernel<<<(unsigned)nq, SEL_THREADS, smem, st>>>(ix, q, nprobe, scores, lists);
    return cudaGetLastError();
}

}  // namespace bbc
