// S3: per-query PQ lookup table (Section 2, "Quantization", step (1): the
// query's distances to every codebook vector), quantised to uint16 so that
// the scan accumulates exact integers.
//
// FP32 entry    L[m][j] = sum_i (q_i - y_{m,j,i})^2        (L2, ascending i)
//                         -(sum_i q_i * y_{m,j,i})           (IP)
//               with one rounding per operation (no fused multiply-add);
// offsets       lo_m = min_j L[m][j];
// scale         span = max_m (max_j L[m][j] - lo_m), inv = T / span
//               (0 when span is 0 or the quotient overflows);
// uint16 entry  min(T, floor((L[m][j] - lo_m) * inv + 0.5)),
// with top level T = 65535, or a smaller T chosen by the caller: at T = 2047
// every entry is an integer FP16 holds exactly, which the tensor-core scan
// (k_scan_tc.cu) uses; the kernel then also writes the entries as FP16.
// The per-query constant sum_m lo_m does not change any order and is dropped.
//
// Residual IVF-PQ (the codes quantise o - c_l, y their reconstruction): the
// estimated distance is the same table's sum plus a per-(query, list) and a
// per-object term,
//   L2  ||q - c_l - y||^2 = sum_m L[m][code_m] + (||c_l||^2 - 2 <q, c_l>) + 2 <c_l, y>,
//   IP  -<q, c_l + y>     = sum_m L[m][code_m] - <q, c_l>,
// which the scan adds in the table's integer units: base_ql = 2^30 +
// rint(clamp(A_ql * inv, +-2^29)) per probed list (resid_base_kernel) and
// w_o = rint(clamp(V_o * inv, +-2^28)) per object, V_o = 2 <c_l, y> stored
// per code slot at index build (resid_v_kernel).  A_ql and V_o are FP32 dot
// products as chains of fused multiply-adds over ascending dimension; the
// 2^30 keeps every key positive and the clamps keep it below 2^31.
#include <cfloat>

#include <cuda_fp16.h>

#include "bbc_internal.cuh"
#include "dev_util.cuh"

namespace bbc {

constexpr int LUT_THREADS = 256;

__global__ void __launch_bounds__(LUT_THREADS) lut16_kernel(DevIndex ix, const float* __restrict__ q,
                                                             uint16_t* __restrict__ out, float* __restrict__ inv_out,
                                                             float top, uint16_t* __restrict__ out_f16) {
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
    float inv = span > 0.f ? __fdiv_rn(top, span) : 0.f;
    if (!(inv <= FLT_MAX)) inv = 0.f;
    if (inv_out && threadIdx.x == 0) inv_out[qi] = inv;
    uint16_t* o = out + qi * MK;
    uint16_t* oh = out_f16 ? out_f16 + qi * MK : nullptr;
    for (int e = threadIdx.x; e < MK; e += blockDim.x) {
        const int m = e / K;
        float t = __fsub_rn(lut[e], lo[m]);
        float u = __fmul_rn(t, inv);
        float v = floorf(__fadd_rn(u, 0.5f));
        v = v > top ? top : v;
        o[e] = (uint16_t)v;
        if (oh) oh[e] = __half_as_ushort(__float2half_rn(v));    // exact for v <= 2048
    }
}

cudaError_t launch_lut16(const DevIndex& ix, const float* q, int64_t nq, uint16_t* lut16,
                         cudaStream_t st, float* inv, int levels, uint16_t* lut_f16) {
    if (nq <= 0) return cudaSuccess;
    if (levels < 1 || levels > 65535 || (lut_f16 && levels > 2048)) return cudaErrorInvalidValue;
    size_t smem = sizeof(float) * ((size_t)ix.M * ix.K + ix.d + 2 * ix.M);
    cudaError_t e = smem_attr_once((const void*)lut16_kernel, 200 * 1024);
    if (e != cudaSuccess) return e;
    lut16_kernel<<<(unsigned)nq, LUT_THREADS, smem, st>>>(ix, q, lut16, inv, (float)levels, lut_f16);
    return cudaGetLastError();
}

// x * inv rounded to the nearest integer (ties to even) after clamping to +-lim.
__device__ __forceinline__ int32_t resid_units(float x, float inv, float lim) {
    float u = __fmul_rn(x, inv);
    u = fminf(fmaxf(u, -lim), lim);
    return __float2int_rn(u);
}

constexpr int RB_THREADS = 128;

// One thread per (query, probed list): A_ql from the query (staged in shared
// memory) and the list's centroid row, ||c_l||^2 from the index (the same
// FP32 chain, computed once per list at build).
__global__ void __launch_bounds__(RB_THREADS) resid_base_kernel(DevIndex ix, const float* __restrict__ q,
                                                                QueryParams qp, const int32_t* __restrict__ lists,
                                                                const float* __restrict__ inv,
                                                                int32_t* __restrict__ base) {
    extern __shared__ float qs[];
    const int64_t qi = blockIdx.y;
    const int d = ix.d;
    for (int i = threadIdx.x; i < d; i += blockDim.x) qs[i] = q[qi * d + i];
    __syncthreads();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= qp.P(qi)) return;
    const int64_t o = qp.poff(qi) + j;
    const int l = lists[o];
    const float4* c4 = reinterpret_cast<const float4*>(ix.centroids + (int64_t)l * d);
    float s = 0.f;
    for (int i4 = 0; i4 < (d >> 2); ++i4) {
        const float4 c = __ldg(c4 + i4);
        s = __fmaf_rn(qs[4 * i4 + 0], c.x, s);
        s = __fmaf_rn(qs[4 * i4 + 1], c.y, s);
        s = __fmaf_rn(qs[4 * i4 + 2], c.z, s);
        s = __fmaf_rn(qs[4 * i4 + 3], c.w, s);
    }
    const float a = ix.metric == BBC_METRIC_L2 ? __fmaf_rn(-2.f, s, __ldg(ix.rcn2 + l)) : -s;
    base[o] = (int32_t)(1 << 30) + resid_units(a, inv[qi], 536870912.f);
}

cudaError_t launch_resid_base(const DevIndex& ix, const float* q, int64_t nq, const QueryParams& qp, int maxp,
                              const int32_t* lists, const float* inv, int32_t* base, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    if (!ix.rcn2 || (ix.d & 3) || maxp < 1) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((maxp + RB_THREADS - 1) / RB_THREADS), (unsigned)nq);
    resid_base_kernel<<<grid, RB_THREADS, sizeof(float) * ix.d, st>>>(ix, q, qp, lists, inv, base);
    return cudaGetLastError();
}

// Index build, one CTA per list: V_o of each object from its canonical code
// row (chain of fused multiply-adds over sub-spaces, then dimensions), and
// ||c_l||^2 (the same chain) by thread 0.
__global__ void resid_v_kernel(DevIndex ix, const uint8_t* __restrict__ canon, const int64_t* __restrict__ off,
                               float* __restrict__ rv, float* __restrict__ cn2) {
    const int l = blockIdx.x;
    const int d = ix.d, ds = ix.dsub, M = ix.M, bits = ix.bits, cb = ix.code_bytes;
    const float* c = ix.centroids + (int64_t)l * d;
    if (threadIdx.x == 0) {
        float n = 0.f;
        for (int i = 0; i < d; ++i) n = __fmaf_rn(c[i], c[i], n);
        cn2[l] = n;
    }
    const int64_t o0 = off[l];
    const int len = ix.list_len[l];
    const int64_t s0 = (int64_t)ix.list_blk[l] * 32;
    for (int p = threadIdx.x; p < len; p += blockDim.x) {
        const uint8_t* row = canon + (o0 + p) * cb;
        float t = 0.f;
        for (int m = 0; m < M; ++m) {
            const int code = bits == 8 ? row[m] : ((m & 1) ? (row[m >> 1] >> 4) : (row[m >> 1] & 0xF));
            const float* y = ix.books + ((int64_t)m * ix.K + code) * ds;
            for (int i = 0; i < ds; ++i) t = __fmaf_rn(c[m * ds + i], y[i], t);
        }
        rv[s0 + p] = ix.metric == BBC_METRIC_L2 ? 2.f * t : 0.f;
    }
}

cudaError_t launch_resid_v(const DevIndex& ix, const uint8_t* canon_codes, const int64_t* list_off, float* rv,
                           float* cn2, int64_t nslots, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(rv, 0, (size_t)nslots * sizeof(float), st);
    if (e != cudaSuccess) return e;
    resid_v_kernel<<<(unsigned)ix.nlist, 256, 0, st>>>(ix, canon_codes, list_off, rv, cn2);
    return cudaGetLastError();
}

}  // namespace bbc
