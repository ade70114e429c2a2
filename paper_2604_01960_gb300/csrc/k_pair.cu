// Pairing plan of the batched scan's pair form (k_scan.cu, scan_pair_kernel):
// which two queries of a batch share a CTA.  Two queries share most of the
// lists they probe when they are near each other; the plan pairs them so
// without reading the index:
//   1. pair_sort_kernel: sort the queries by (nearest list, second nearest
//      list, index), in blocks of kPairBlock queries (one CTA each);
//   2. pair_greedy_kernel: one warp per window of 32 consecutive sorted
//      queries; among the queries of a window that share their nearest list,
//      mutual nearest neighbours (squared L2 between the query vectors) are
//      paired, repeatedly, so the closest pairs form first;
//   3. pair_finalize_kernel: the output permutation, deterministic: first
//      the unpaired queries in sorted order, paired with each other two by
//      two (an odd one last), then the pairs in sorted order.
// perm[2i], perm[2i + 1] are the queries of CTA i; with an odd count the
// last entry is alone.  The plan only decides the schedule: the scan's
// results are the same under any pairing.
#include "bbc_internal.cuh"
#include "dev_util.cuh"

namespace bbc {

constexpr int kPairBlock = 16384;     // queries sorted by one CTA (keys in shared memory)
constexpr int kPairSortThreads = 1024;

__global__ void __launch_bounds__(kPairSortThreads) pair_sort_kernel(QueryParams qp, const int32_t* __restrict__ lists,
                                                                    int64_t nq, int32_t* sorted_q, int32_t* sorted_l) {
    extern __shared__ unsigned long long pkeys[];
    const int64_t base = (int64_t)blockIdx.x * kPairBlock;
    const int n = (int)min((int64_t)kPairBlock, nq - base);
    const int np2 = next_pow2(n);
    for (int i = threadIdx.x; i < np2; i += blockDim.x) {
        unsigned long long k = ~0ull;
        if (i < n) {
            const int64_t q = base + i;
            const int32_t* lq = lists + qp.poff(q);
            const unsigned long long l0 = (unsigned long long)lq[0] & 0xFFFFFull;
            const unsigned long long l1 = qp.P(q) > 1 ? (unsigned long long)lq[1] & 0xFFFFFull : 0ull;
            k = (l0 << 44) | (l1 << 24) | (unsigned long long)i;
        }
        pkeys[i] = k;
    }
    __syncthreads();
    cta_bitonic_u64(pkeys, np2);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const unsigned long long k = pkeys[i];
        sorted_q[base + i] = (int32_t)(base + (int64_t)(k & 0xFFFFFFull));
        sorted_l[base + i] = (int32_t)(k >> 44);
    }
}

// One warp per window of 32 sorted positions.  partner[p] = sorted position
// of p's partner, or -1.
__global__ void __launch_bounds__(256) pair_greedy_kernel(const float* __restrict__ q, int d, int64_t nq,
                                                          const int32_t* __restrict__ sorted_q,
                                                          const int32_t* __restrict__ sorted_l, int32_t* partner) {
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id();
    const int64_t p0 = w * 32;
    if (p0 >= nq) return;
    const unsigned ln = lane_id();
    const int64_t pos = p0 + ln;
    const bool valid = pos < nq;
    const int64_t qi = valid ? sorted_q[pos] : 0;
    const int li = valid ? sorted_l[pos] : -1;
    float D[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) D[j] = 0.f;
    const float* qv = q + qi * (int64_t)d;
    for (int c = 0; c < d; ++c) {
        const float x = valid ? __ldg(qv + c) : 0.f;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const float t = x - __shfl_sync(0xFFFFFFFFu, x, j);
            D[j] = fmaf(t, t, D[j]);
        }
    }
    // candidates: valid, not itself, same nearest list
    unsigned cand = 0;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const int lj = __shfl_sync(0xFFFFFFFFu, li, j);
        const bool vj = __shfl_sync(0xFFFFFFFFu, valid ? 1 : 0, j) != 0;
        if (valid && vj && j != (int)ln && lj == li) cand |= 1u << j;
    }
    unsigned open = __ballot_sync(0xFFFFFFFFu, valid);
    int mate = -1;
    for (int round = 0; round < 16; ++round) {
        int nn = -1;
        float best = 0.f;
        if ((open >> ln) & 1u) {
            const unsigned c = cand & open;
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (((c >> j) & 1u) && (nn < 0 || D[j] < best)) { nn = j; best = D[j]; }
        }
        const int back = __shfl_sync(0xFFFFFFFFu, nn, nn < 0 ? (int)ln : nn);
        const bool mutual = nn >= 0 && back == (int)ln;
        const unsigned mm = __ballot_sync(0xFFFFFFFFu, mutual);
        if (!mm) break;
        if (mutual) mate = nn;
        open &= ~mm;
    }
    if (valid) partner[pos] = mate >= 0 ? (int32_t)(p0 + mate) : -1;
}

// Exclusive CTA scan of v (blockDim.x <= 1024); *total = sum.
__device__ __forceinline__ uint32_t pair_cta_scan(uint32_t v, uint32_t* wsum, uint32_t* total) {
    const uint32_t inc = warp_incl_scan(v);
    if (lane_id() == 31) wsum[warp_id()] = inc;
    __syncthreads();
    if (warp_id() == 0) {
        const int nw = blockDim.x >> 5;
        const uint32_t x = (int)lane_id() < nw ? wsum[lane_id()] : 0u;
        const uint32_t xi = warp_incl_scan(x);
        if ((int)lane_id() < nw) wsum[lane_id()] = xi - x;
        if (lane_id() == 31) wsum[32] = xi;
    }
    __syncthreads();
    const uint32_t r = wsum[warp_id()] + inc - v;
    *total = wsum[32];
    __syncthreads();
    return r;
}

// One CTA per block of kPairBlock sorted queries; each thread takes a run of
// consecutive positions.
__global__ void __launch_bounds__(kPairSortThreads) pair_finalize_kernel(int64_t nq, const int32_t* __restrict__ sorted_q,
                                                                        const int32_t* __restrict__ partner,
                                                                        int32_t* perm) {
    __shared__ uint32_t wsum[33];
    const int64_t base = (int64_t)blockIdx.x * kPairBlock;
    const int n = (int)min((int64_t)kPairBlock, nq - base);
    const int per = (n + (int)blockDim.x - 1) / (int)blockDim.x;
    const int i0 = (int)threadIdx.x * per;
    uint32_t np = 0, nl = 0;
    for (int i = i0; i < min(n, i0 + per); ++i) {
        const int32_t m = partner[base + i];
        if (m < 0) ++nl;
        else if (m > base + i) ++np;
    }
    uint32_t tp, tl;
    const uint32_t op = pair_cta_scan(np, wsum, &tp);
    const uint32_t ol = pair_cta_scan(nl, wsum, &tl);
    // layout: leftovers [0, tl) (an odd last one moves to the very end), then pairs
    const uint32_t lead = tl & ~1u;
    uint32_t kp = op, kl = ol;
    for (int i = i0; i < min(n, i0 + per); ++i) {
        const int32_t m = partner[base + i];
        if (m < 0) {
            const uint32_t slot = kl < lead ? kl : (uint32_t)n - 1u;
            perm[base + slot] = sorted_q[base + i];
            ++kl;
        } else if (m > base + i) {
            perm[base + lead + 2 * kp] = sorted_q[base + i];
            perm[base + lead + 2 * kp + 1] = sorted_q[m];
            ++kp;
        }
    }
}

size_t pair_plan_bytes(int64_t nq) { return (size_t)nq * 4 * 4; }

cudaError_t launch_pair_plan(const float* q, int d, int64_t nq, const QueryParams& qp, const int32_t* lists,
                             void* scratch, int32_t* perm, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    int32_t* sorted_q = static_cast<int32_t*>(scratch);
    int32_t* sorted_l = sorted_q + nq;
    int32_t* partner = sorted_l + nq;
    const unsigned nb = (unsigned)((nq + kPairBlock - 1) / kPairBlock);
    const size_t smem = (size_t)kPairBlock * 8;
    cudaError_t e = smem_attr_once((const void*)pair_sort_kernel, (int)smem);
    if (e != cudaSuccess) return e;
    pair_sort_kernel<<<nb, kPairSortThreads, smem, st>>>(qp, lists, nq, sorted_q, sorted_l);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t windows = (nq + 31) / 32;
    pair_greedy_kernel<<<(unsigned)((windows + 7) / 8), 256, 0, st>>>(q, d, nq, sorted_q, sorted_l, partner);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    pair_finalize_kernel<<<nb, kPairSortThreads, 0, st>>>(nq, sorted_q, partner, perm);
    return cudaGetLastError();
}

}  // namespace bbc
