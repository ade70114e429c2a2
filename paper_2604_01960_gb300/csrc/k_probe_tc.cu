// S1 on the tensor cores: approximate probe scores from a BF16 GEMM with FP32
// accumulation in tensor memory (tcgen05), operands staged by TMA.
//
// Scores (as in k_probe.cu): a[q][l] = ||c_l||^2 - 2<q, c_l> (L2) or
// -<q, c_l> (IP).  To keep the pruning band narrow, each FP32 value x is split
// into two BF16 terms x = x_hi + x_lo + r with |r| <= 2^-16 |x|, and
//   <q, c> ~ <q_hi, c_hi> + <q_hi, c_lo> + <q_lo, c_hi>
// is one GEMM over K = 3d: A = [q_hi | q_hi | q_lo], B = [c_hi | c_lo | c_hi]
// (K padded with zeros to a multiple of 64).  Error bound: see probe_eps_tc.
//
// CTA tile 128 queries x 256 lists; K steps of 64 BF16 (one 128-byte swizzle
// row) in a 4-stage TMA ring; one elected thread issues TMA and tcgen05.mma
// (M = 128, N = 256, K = 16 per instruction) and commits to mbarriers; the
// four warps then read the 128 x 256 FP32 accumulator from tensor memory
// (warp w owns lanes 32w..32w+31) and write the scores.  Every mbarrier wait
// is bounded by a clock budget; on expiry the kernel latches a status bit,
// drains its own copies and MMAs (again bounded), frees its tensor memory and
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <mutex>

#include "bbc_internal.cuh"
#include "dev_util.cuh"
#include "tc_util.cuh"

namespace bbc {

constexpr int TC_BM = 128, TC_BN = 256, TC_BK = 64, TC_STAGES = 4;
constexpr int TC_A_BYTES = TC_BM * TC_BK * 2;
constexpr int TC_B_BYTES = TC_BN * TC_BK * 2;
constexpr int TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES;
constexpr int TC_THREADS = 128;
constexpr int TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 256 + TC_BN * 4 + 1024;
// tcgen05 instruction descriptor, kind::f16: FP32 accumulate, BF16 A and B,
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
                              ((uint32_t)(TC_BM >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    tc_mma_f16(tmem_d, adesc, bdesc, TC_IDESC, accumulate);
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    probe_gemm_tc_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                         const float* __restrict__ cnorm, int64_t nq, int L, int ktiles, int metric,
                         float* __restrict__ out, unsigned int* status) {
    extern __shared__ uint8_t tsm_raw[];
    const uint32_t raw = smem_u32(tsm_raw);
    const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
    uint8_t* tsm = tsm_raw + pad;
    const uint32_t sbase = raw + pad;
    uint64_t* bars = reinterpret_cast<uint64_t*>(tsm + TC_STAGES * TC_STAGE_BYTES);   // full[S], empty[S], done
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * TC_STAGES + 1);
    int* s_err = reinterpret_cast<int*>(tmem_slot + 1);
    float* cn = reinterpret_cast<float*>(tsm + TC_STAGES * TC_STAGE_BYTES + 256);
    const uint32_t bar0 = smem_u32(bars);
    auto full = [&](int s) { return bar0 + 8u * s; };
    auto empty = [&](int s) { return bar0 + 8u * (TC_STAGES + s); };
    const uint32_t done = bar0 + 8u * (2 * TC_STAGES);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t q0 = (int64_t)blockIdx.y * TC_BM;
    const int l0 = blockIdx.x * TC_BN;
    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) { mbar_init(full(s), 1); mbar_init(empty(s), 1); }
        mbar_init(done, 1);
        *s_err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)TC_BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    for (int j = tid; j < TC_BN; j += TC_THREADS) cn[j] = (l0 + j < L) ? cnorm[l0 + j] : 0.f;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (tid == 0) {
        bool ok = true;
        int issued = 0;                     // k tiles whose copies were issued
        const int pro = ktiles < TC_STAGES ? ktiles : TC_STAGES;
        for (int s = 0; s < pro; ++s) {
            const uint32_t a_s = sbase + s * TC_STAGE_BYTES, b_s = a_s + TC_A_BYTES;
            mbar_expect_tx(full(s), TC_STAGE_BYTES);
            tma_load_2d(a_s, &ta, full(s), s * TC_BK, (int)q0);
            tma_load_2d(b_s, &tb, full(s), s * TC_BK, l0);
            ++issued;
        }
        int consumed = 0;                   // k tiles whose copies were waited for
        for (int kt = 0; kt < ktiles && ok; ++kt) {
            const int s = kt % TC_STAGES;
            if (!mbar_wait(full(s), (uint32_t)((kt / TC_STAGES) & 1))) { ok = false; break; }
            ++consumed;
            tc_fence_after();
            const uint32_t a_s = sbase + s * TC_STAGE_BYTES, b_s = a_s + TC_A_BYTES;
#pragma unroll
            for (int k = 0; k < TC_BK / 16; ++k)
                tc_mma(tmem, sw128_desc(a_s + 32u * k), sw128_desc(b_s + 32u * k), (kt | k) != 0 ? 1u : 0u);
            tc_commit(empty(s));
            // refill the stage used one step earlier once its MMAs are done
            const int pk = kt - 1, nk = pk + TC_STAGES;
            if (pk >= 0 && nk < ktiles) {
                const int ps = pk % TC_STAGES;
                if (!mbar_wait(empty(ps), (uint32_t)((pk / TC_STAGES) & 1))) { ok = false; break; }
                const uint32_t a_p = sbase + ps * TC_STAGE_BYTES, b_p = a_p + TC_A_BYTES;
                mbar_expect_tx(full(ps), TC_STAGE_BYTES);
                tma_load_2d(a_p, &ta, full(ps), nk * TC_BK, (int)q0);
                tma_load_2d(b_p, &tb, full(ps), nk * TC_BK, l0);
                ++issued;
            }
        }
        if (!ok) {
            atomicOr(status, kStatusTimeout);
            *s_err = 1;
            // drain copies still in flight (bounded)
            for (int t = consumed; t < issued; ++t) mbar_wait(full(t % TC_STAGES), (uint32_t)((t / TC_STAGES) & 1));
        }
        tc_commit(done);                    // arrives when every MMA issued above has completed
    }
    __syncwarp();
    const bool done_ok = __all_sync(0xFFFFFFFFu, mbar_wait(done, 0u));
    if (!done_ok && lane == 0) atomicOr(status, kStatusTimeout);
    tc_fence_after();
    __syncthreads();
    if (done_ok && *s_err == 0) {
        const int64_t row = q0 + warp * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c = 0; c < TC_BN; c += 32) {
            uint32_t r[32];
            tmem_ld32(tl + (uint32_t)c, r);
            if (row < nq) {
                float* o = out + row * (int64_t)L + l0 + c;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    if (l0 + c + j < L) {
                        const float acc = __uint_as_float(r[j]);
                        o[j] = metric == BBC_METRIC_L2 ? fmaf(-2.f, acc, cn[c + j]) : -acc;
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)TC_BN));
}

// A = [q_hi | q_hi | q_lo | 0-pad] per query, BF16.
__global__ void split_queries_kernel(const float* __restrict__ q, int64_t nq, int d, int kp,
                                     __nv_bfloat16* __restrict__ a) {
    const int64_t qi = blockIdx.x;
    for (int k = threadIdx.x; k < kp; k += blockDim.x) {
        __nv_bfloat16 v = __float2bfloat16_rn(0.f);
        if (k < 3 * d) {
            const int i = k % d;
            const float x = q[qi * d + i];
            const __nv_bfloat16 hi = __float2bfloat16_rn(x);
            v = (k < 2 * d) ? hi : __float2bfloat16_rn(x - __bfloat162float(hi));
        }
        a[qi * kp + k] = v;
    }
}

namespace {
std::mutex g_tma_mu;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

cudaError_t encode_fn(PFN_cuTensorMapEncodeTiled_v12000* out) {
    std::lock_guard<std::mutex> lk(g_tma_mu);
    if (!g_encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult qr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr);
        if (e != cudaSuccess) return e;
        if (qr != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    *out = g_encode;
    return cudaSuccess;
}

cudaError_t make_map(CUtensorMap* map, const void* base, uint64_t inner, uint64_t rows, uint32_t box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc;
    cudaError_t e = encode_fn(&enc);
    if (e != cudaSuccess) return e;
    const cuuint64_t dims[2] = {inner, rows};
    const cuuint64_t strides[1] = {inner * 2};
    const cuuint32_t box[2] = {(cuuint32_t)TC_BK, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}
}  // namespace

size_t probe_tc_workspace(const DevIndex& ix, int64_t nq) { return (size_t)nq * ix.kp * 2; }

cudaError_t launch_probe_scores_tc(const DevIndex& ix, const float* q, int64_t nq, float* scores, void* abuf,
                                   cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    if (!ix.cent_b3 || ix.kp % TC_BK) return cudaErrorInvalidValue;
    __nv_bfloat16* a = static_cast<__nv_bfloat16*>(abuf);
    split_queries_kernel<<<(unsigned)nq, 128, 0, st>>>(q, nq, ix.d, ix.kp, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    CUtensorMap ta, tb;
    if ((e = make_map(&ta, a, (uint64_t)ix.kp, (uint64_t)nq, TC_BM)) != cudaSuccess) return e;
    if ((e = make_map(&tb, ix.cent_b3, (uint64_t)ix.kp, (uint64_t)ix.nlist, TC_BN)) != cudaSuccess) return e;
    if ((e = smem_attr_once((const void*)probe_gemm_tc_kernel, TC_SMEM)) != cudaSuccess) return e;
    dim3 grid((unsigned)((ix.nlist + TC_BN - 1) / TC_BN), (unsigned)((nq + TC_BM - 1) / TC_BM));
    probe_gemm_tc_kernel<<<grid, TC_THREADS, TC_SMEM, st>>>(ta, tb, ix.cnorm, nq, ix.nlist, ix.kp / TC_BK,
                                                            ix.metric, scores, ix.status);
    return cudaGetLastError();
}

}  // namespace bbc
