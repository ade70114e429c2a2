// bbc_collect_static: the candidate-collection stage (lookup table, scan with
// the bucket-based result buffer, final selection) for callers that cannot
// allocate device memory.
//
// Who cannot allocate: a host program that budgets every byte of device
// memory itself -- for example a server that splits HBM between several
// models up front and forbids libraries from calling cudaMalloc behind its
// back -- and latency-critical threads, where a cudaMalloc can block in the
// driver and synchronise the device, stalling work other streams have in
// flight.  bbc_collect gets its scratch from a workspace that it grows with
// cudaMalloc; this entry point instead uses one fixed array compiled into the
// library, so it never allocates.
//
// The array lives in global memory of every GPU that loads the library and
// stays there until the process exits.  All calls share it: two calls whose
// kernels overlap on the GPU (on different streams, or from different
// threads without ordering) overwrite each other's scratch and race; order
// them on one stream.  No part of the array has to start at zero: each call
// writes every byte it later reads (the lookup tables, the per-query state and
// the appended (estimate, id) pairs) before reading it, so the contents left
// by the previous call are never used.
#include <cstdio>
#include <mutex>

#include "bbc_internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)BBC_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// The scratch itself.  In host code this name is only a host-side stand-in
// for the device symbol: its device address must come from
// cudaGetSymbolAddress (done once per device below), never from taking the
// address of the name here.
static __device__ __align__(256) unsigned char g_collect_scratch[kStaticScratchBytes];

namespace {

// Device address of the scratch on `device`, looked up on the first call for
// that device with the device current, then cached.
int scratch_address(int device, void** out) {
    if (device < 0 || device >= kMaxDevices) return bbc::api_error(BBC_ERR_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_collect_scratch);
        if (e != cudaSuccess || p == nullptr)
            return bbc::api_error(BBC_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return BBC_OK;
}

}  // namespace

extern "C" int bbc_collect_static(bbc_index* ix, const float* queries, int64_t nq, int32_t nprobe,
                                  const int32_t* probe_lists, int64_t kc, uint32_t* out_ids,
                                  int64_t* out_count, bbc_collector_state* out_state, void* stream) {
    using namespace bbc;
    int rc = api_check_search_args(ix, queries, nq, 1, nprobe, out_ids, out_count);
    if (rc) return rc;
    if (index_dev(ix).quant != 0) return api_error(BBC_ERR_UNSUPPORTED, "bbc_collect_static: not available on a sign-code index");
    if (nq > 0 && !probe_lists) return api_error(BBC_ERR_ARG, "null probe_lists");
    if (kc < 1 || kc > (int64_t)0x7FFFFFFF) return api_error(BBC_ERR_ARG, "kc must be in [1, 2^31)");
    if (nq == 0) return BBC_OK;
    const DevIndex& d = index_dev(ix);
    const int64_t cap = index_cap(ix, nprobe);
    const size_t lut_bytes = align256((size_t)nq * d.M * d.K * 2);
    const size_t state_bytes = out_state ? 0 : align256((size_t)nq * sizeof(bbc_collector_state));
    const size_t region_bytes = align256((size_t)nq * (size_t)cap * 8);
    // residual IVF-PQ: each query's table scale and its probed lists' bases
    const size_t resid_bytes = d.resid ? align256((size_t)nq * 4) + align256((size_t)nq * nprobe * 4) : 0;
    const size_t need = lut_bytes + state_bytes + region_bytes + resid_bytes;
    if (need > kStaticScratchBytes) {
        char msg[256];
        snprintf(msg, sizeof(msg),
                 "bbc_collect_static needs %zu bytes of scratch for nq=%lld, nprobe=%d but the static "
                 "scratch holds %zu bytes; pass fewer queries per call",
                 need, (long long)nq, nprobe, kStaticScratchBytes);
        return api_error(BBC_ERR_ARG, msg);
    }
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return api_error(BBC_ERR_CUDA, "cudaGetDevice failed");
    const int dev = index_device(ix);
    if (cudaSetDevice(dev) != cudaSuccess) return api_error(BBC_ERR_CUDA, "cudaSetDevice failed");
    void* base = nullptr;
    rc = scratch_address(dev, &base);
    cudaError_t e = cudaSuccess;
    if (rc == BBC_OK) {
        char* p = static_cast<char*>(base);
        uint16_t* lut = reinterpret_cast<uint16_t*>(p);
        bbc_collector_state* state =
            out_state ? out_state : reinterpret_cast<bbc_collector_state*>(p + lut_bytes);
        uint2* region = reinterpret_cast<uint2*>(p + lut_bytes + state_bytes);
        char* rp = p + lut_bytes + state_bytes + region_bytes;
        float* qinv = d.resid ? reinterpret_cast<float*>(rp) : nullptr;
        int32_t* lbase = d.resid ? reinterpret_cast<int32_t*>(rp + align256((size_t)nq * 4)) : nullptr;
        cudaStream_t st = (cudaStream_t)stream;
        const QueryParams qp = uniform_params(nprobe, kc, 1, cap);
        e = launch_lut16(d, queries, nq, lut, st, qinv, index_lut_levels(ix));
        if (e == cudaSuccess && d.resid) e = launch_resid_base(d, queries, nq, qp, nprobe, probe_lists, qinv, lbase, st);
        if (e == cudaSuccess) {
            ScanArgs sa{lut, probe_lists, nprobe, kc, index_buckets(ix), index_sample_lists(ix), region, cap, state, qp};
            sa.qinv = qinv;
            sa.lbase = lbase;
            e = launch_scan(d, nq, sa, st);
        }
        if (e == cudaSuccess) {
            SelectArgs se{region, cap, state, kc, out_ids, out_count, nullptr, uniform_params(nprobe, kc, 1, cap)};
            e = launch_select(d, nq, se, st);
        }
        if (e != cudaSuccess) rc = api_error(BBC_ERR_CUDA, cudaGetErrorString(e));
    }
    cudaSetDevice(prev);
    return rc;
}
