// S7: final collection (Algorithm 1, the last step of Collect) as its own
// kernel, one CTA per query, for the scan forms that do not run it in their
// tail (several CTAs per query, two queries per CTA) and for the
// allocation-free collect.  The per-query procedure is select_query
// (select_body.cuh).
#include "bbc_internal.cuh"
#include "dev_util.cuh"
#include "select_body.cuh"

namespace bbc {

constexpr int SELK_THREADS = 512;
constexpr int SELK_TCAP = 12288;   // threshold-bucket objects held in shared memory

__global__ void __launch_bounds__(SELK_THREADS) select_kernel(DevIndex ix, SelectArgs a) {
    extern __shared__ unsigned long long tkeys[];      // [SELK_TCAP]
    select_query(ix, a, blockIdx.x, tkeys, (uint32_t)SELK_TCAP);
}

cudaError_t launch_select(const DevIndex& ix, int64_t nq, const SelectArgs& a, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    const size_t smem = (size_t)SELK_TCAP * 8;
    cudaError_t e = smem_attr_once((const void*)select_kernel, (int)smem);
    if (e != cudaSuccess) return e;
    select_kernel<<<(unsigned)nq, SELK_THREADS, smem, st>>>(ix, a);
    return cudaGetLastError();
}

}  // namespace bbc
