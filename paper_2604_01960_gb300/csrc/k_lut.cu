// S3: per-query PQ lookup table (Section 2, "Quantization", step (1): the
// query's distances to every codebook vector), quantised to uint16 so that
// the scan accumulates exact integers.
//
// FP32 entry    L[m][j] = sum_i (q_i - y_{m,j,i})^2        (L2, ascending i)
//                         -(sum_i q_i * y_{m,j,i})           (IP)
//               with one rounding per operation (no fused multiply-add);
// offsets       lo_m = min_j L[m][j];
// scale         span = max_m (max_j L[m][j] - lo_m), inv = 65535 / span
//               (0 when span is 0 or the quotient overflows);
// uint16 entry  min(65535, floor((L[m][j] - lo_m) * inv + 0.5)).
// The per-query constant sum_m lo_m does not change any order and is dropped.
#include <cfloat>

#include "bbc_internal.cuh"
#include "dev_util.cuh"

namespace bbc {

constexpr int LUT_THREADS = 256;

__global__ void __launch_bounds__(LUT_THREADS) lut16_kernel(DevIndex ix, const float* __restrict__ q,
                                                             uint16_t* __restrict__ out) {
    extern __shared__ float lsm[];
    const int M = ix.M, K = ix.K, ds = ix.dsub, d = ix.d;
    float* lut = lsm;                 // [M*K]
    float* qs = lut + M * K;          // [d]
    float* lo = qs + d;               // [M]
    float* wid = lo + M;              // [M]
    const int64_t qi = blockIdx.x;
    for (int i = threadIdx.x; i < d; i += blockDim.x) qs[i] = q[qi * d + i];
    __syncthreads();
    const int MK = M * K;
    for (int e = threadIdx.x; e < MK; e += blockDim.x) {
        const int m = e / K;
        const float* y = ix.books + (int64_t)e * ds;
        const float* qm = qs + m * ds;
        float acc = 0.f;
        if (ix.metric == BBC_METRIC_L2) {
            for (int i = 0; i < ds; ++i) {
                float t = __fsub_rn(qm[i], y[i]);
                acc = __fadd_rn(acc, __fmul_rn(t, t));
            }
        } else {
            for (int i = 0; i < ds; ++i) acc = __fadd_rn(acc, __fmul_rn(qm[i], y[i]));
            acc = -acc;
        }
        lut[e] = acc;
    }
    __syncthreads();
    for (int m = warp_id(); m < M; m += blockDim.x / 32) {
        float mn = FLT_MAX, mx = -FLT_MAX;
        for (int j = lane_id(); j < K; j += 32) {
            float v = lut[m * K + j];
            mn = v < mn ? v : mn;
            mx = v > mx ? v : mx;
        }
        for (int o = 16; o; o >>= 1) {
            float a = __shfl_xor_sync(0xFFFFFFFFu, mn, o);
            float b = __shfl_xor_sync(0xFFFFFFFFu, mx, o);
            mn = a < mn ? a : mn;
            mx = b > mx ? b : mx;
        }
        if (lane_id() == 0) {
            lo[m] = mn;
            wid[m] = __fsub_rn(mx, mn);
        }
    }
    __syncthreads();
    float span = 0.f;
    for (int m = 0; m < M; ++m) span = wid[m] > span ? wid[m] : span;
    float inv = span > 0.f ? __fdiv_rn(65535.0f, span) : 0.f;
    if (!(inv <= FLT_MAX)) inv = 0.f;
    uint16_t* o = out + qi * MK;
    for (int e = threadIdx.x; e < MK; e += blockDim.x) {
        const int m = e / K;
        float t = __fsub_rn(lut[e], lo[m]);
        float u = __fmul_rn(t, inv);
        float v = floorf(__fadd_rn(u, 0.5f));
        v = v > 65535.f ? 65535.f : v;
        o[e] = (uint16_t)v;
    }
}

cudaError_t launch_lut16(const DevIndex& ix, const float* q, int64_t nq, uint16_t* lut16,
                         cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    size_t smem = sizeof(float) * ((size_t)ix.M * ix.K + ix.d + 2 * ix.M);
    cudaError_t e = smem_attr_once((const void*)lut16_kernel, 200 * 1024);
    if (e != cudaSuccess) return e;
    lut16_kernel<<<(unsigned)nq, LUT_THREADS, smem, st>>>(ix, q, lut16);
    return cudaGetLastError();
}

}  // namespace bbc
