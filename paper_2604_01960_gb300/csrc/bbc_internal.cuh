// Internal declarations shared by the CUDA translation units of libbbc.
//
// Device data layout of an IVF-PQ index (all resident in HBM):
//   centroids  f32 [nlist][d]          probe operand (row-major)
//   cnorm      f32 [nlist]             ||c_l||^2 for the probe epilogue
//   list_blk   i32 [nlist]             first 32-vector block of list l
//   list_len   i32 [nlist]             vectors in list l
//   codes      u8  [nblocks][CBP/16][32][16]
//              one block = 32 consecutive list positions ("lanes"); the code
//              row of lane t is split in 16-byte chunks, chunk c of all 32
//              lanes contiguous, so a warp reads each chunk with one fully
//              coalesced 512-byte access.  Inside a row, code slot s of lane t
//              holds sub-space (s + t) mod M (rotated rows), which makes the
//              shared-memory lookup-table reads of a warp bank-conflict free.
//   ids        u32 [nblocks*32]        vector id per position, 0xFFFFFFFF = pad
//   books      f32 [M][K][d/M]         PQ codebooks
//   vectors    f32 [n][d]              by id, for the exact re-rank
//   vec_u8     u8  [n][d]              exact copy when all components are
//                                      integers in [0,255] (else null)
//   vec_lp     bf16 or e4m3 [n][dpad]  low-precision copy for the precision
//                                      re-rank (null until requested); rows
//                                      zero-padded to dpad = d rounded up to 16
//   vec_meta   f32x4 [n]               {FP8 scale s (1 for BF16), e_v =
//                                      ||v - v~||_2 rounded up, ||v||_2 rounded
//                                      up, 0} per vector
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bbc.h"

namespace bbc {

constexpr int kLanes = 32;                 // vectors per code block (one per lane)
constexpr uint32_t kPadId = 0xFFFFFFFFu;   // id of padding slots in a block
constexpr int kMaxBuckets = 256;

// Status bits latched in the index's device status word.
constexpr unsigned kStatusRegionOverrun = 1u;
constexpr unsigned kStatusSelectOverrun = 2u;
constexpr unsigned kStatusTopkOverrun = 4u;
constexpr unsigned kStatusTimeout = 8u;
constexpr unsigned kStatusPrecBound = 16u;   // a precision re-rank bound failed its self-check

struct DevIndex {
    int d, nlist, metric, M, bits, K, dsub;
    int code_bytes;      // bytes of one canonical code row
    int cbp;             // code row bytes padded to a multiple of 16
    int W;               // words per row of the shared-memory LUT
    int64_t n;
    float cmax;          // max_l ||c_l||_2
    const float* centroids;
    const float* cnorm;
    const int32_t* list_blk;
    const int32_t* list_len;
    const uint8_t* codes;
    const uint32_t* ids;
    const float* books;
    const float* vectors;
    const uint8_t* vec_u8;
    unsigned int* status;
    const uint16_t* cent_b3;   // BF16 [nlist][kp]: [c_hi | c_lo | c_hi | 0-pad] for the tensor-core probe
    int kp;                    // 3d rounded up to a multiple of 64
    int num_sms;               // streaming multiprocessors of the device
    const void* vec_lp;        // low-precision copy (see above) or null
    const float4* vec_meta;    // per-vector scale / error / norm, or null
    int prec;                  // 0 none, 1 BF16 copy, 2 FP8-E4M3 copy
    int dpad;                  // row length of the low-precision copy
    // 1-bit sign quantizer (quant = 1); codes and ids share the block layout of the PQ codes
    int quant;                 // 0 PQ, 1 sign codes
    const uint32_t* sgn;       // [nblocks][d/32][32] code words, word w of lane t at (b*W + w)*32 + t
    const float4* sfac;        // [nblocks*32] {alpha, e (rounded up), ||o - c||^2, popcount}
    const double* crot;        // [nlist][d] P c_l in FP64
    const float* rot;          // [d][d] rotation P, row-major (r = P u)
    double eps_p;              // ||P^T P - I||_F
    // early re-rank (Algorithm 4): the exact u8 copy in code-block slot order,
    // so a warp's 32-vector block has its rows contiguous, and ||v||^2 per slot
    const uint8_t* vec_lo;     // [nblocks * 32][d] or null
    const uint32_t* vnorm2;    // [nblocks * 32] or null
    // residual IVF-PQ: the codes quantise o - c_l; per code-block slot the
    // object's term V_o = 2 <c_l, y_o> (L2; 0 for IP and padding slots)
    int resid;                 // 1: residual codes
    const float* rv;           // [nblocks * 32] or null
    const float* rcn2;         // [nlist] ||c_l||^2 in FP32 (chain of fused multiply-adds), or null
};

// Words per LUT row in shared memory: lane t at code slot s reads word t + s
// of the row of its code value, so a row needs M + 31 words; a multiple of 32
// keeps bank(t, s) = (t + s) mod 32 for every row (k_scan.cu rounds up to a
// power of two where that costs little, to turn the row offset into a shift).
inline int lut_row_words(int M) { return M <= 32 ? 64 : (M <= 96 ? 128 : M + 32); }

// Per-query shape of a batch.  Uniform batches leave the arrays null and use
// the scalar values; mixed batches (different k and nprobe per query) give
// per-query values and exclusive prefix offsets into the packed buffers.
struct QueryParams {
    int nprobe;                     // uniform values
    int64_t kc;
    int k;
    int64_t cap;                    // region entries per query (uniform)
    const int32_t* nprobe_q;        // [nq] or null
    const int64_t* kc_q;            // [nq] or null
    const int32_t* k_q;             // [nq] or null
    const int64_t* probe_off;       // [nq + 1] offsets into probe lists, or null
    const int64_t* region_off;      // [nq + 1] offsets into the region, or null
    const int64_t* cand_off;        // [nq + 1] offsets into candidates, or null
    const int64_t* out_off;         // [nq + 1] offsets into results, or null
    __host__ __device__ int P(int64_t q) const { return nprobe_q ? nprobe_q[q] : nprobe; }
    __host__ __device__ int64_t KC(int64_t q) const { return kc_q ? kc_q[q] : kc; }
    __host__ __device__ int K(int64_t q) const { return k_q ? k_q[q] : k; }
    __host__ __device__ int64_t poff(int64_t q) const { return probe_off ? probe_off[q] : q * (int64_t)nprobe; }
    __host__ __device__ int64_t roff(int64_t q) const { return region_off ? region_off[q] : q * cap; }
    __host__ __device__ int64_t rcap(int64_t q) const {
        return region_off ? region_off[q + 1] - region_off[q] : cap;
    }
    __host__ __device__ int64_t coff(int64_t q) const { return cand_off ? cand_off[q] : q * kc; }
    __host__ __device__ int64_t ooff(int64_t q) const { return out_off ? out_off[q] : q * (int64_t)k; }
};

inline QueryParams uniform_params(int nprobe, int64_t kc, int k, int64_t cap) {
    QueryParams p{};
    p.nprobe = nprobe;
    p.kc = kc;
    p.k = k;
    p.cap = cap;
    return p;
}

// Raises a kernel's dynamic shared-memory limit to `bytes` on the current
// device, once per (kernel, device, bytes): the attribute belongs to the
// kernel on one device, so a process that searches on several devices sets
// it on each.  Thread-safe.
cudaError_t smem_attr_once(const void* kernel, int bytes);

// ---- launchers (one per translation unit) ----

// S1: approximate probe scores a[q][l] = ||c_l||^2 - 2<q,c_l> (L2) or -<q,c_l> (IP).
cudaError_t launch_probe_scores(const DevIndex& ix, const float* q, int64_t nq, float* scores,
                                cudaStream_t st);
// S1 on the tensor cores (tcgen05 BF16 GEMM, 3-term split); abuf holds
// probe_tc_workspace(ix, nq) bytes for the split queries.
size_t probe_tc_workspace(const DevIndex& ix, int64_t nq);
cudaError_t launch_probe_scores_tc(const DevIndex& ix, const float* q, int64_t nq, float* scores, void* abuf,
                                   cudaStream_t st);
// S2: exact probe selection (FP64 decides where the approximations cannot).
// tc = 1 when the scores come from the tensor-core GEMM (wider error bound).
cudaError_t launch_probe_select(const DevIndex& ix, const float* q, int64_t nq, const QueryParams& qp,
                                int max_nprobe, const float* scores, int32_t* lists, int tc, cudaStream_t st);
// S3: uint16 PQ lookup tables [nq][M][K] with entries in [0, levels]; inv
// (may be null): each query's scale levels / span, the table's integer units
// per unit of distance; lut_f16 (may be null, levels <= 2048): the same
// entries as FP16 bit patterns.
cudaError_t launch_lut16(const DevIndex& ix, const float* q, int64_t nq, uint16_t* lut16,
                         cudaStream_t st, float* inv = nullptr, int levels = 65535, uint16_t* lut_f16 = nullptr);
// Residual IVF-PQ, per (query, probed list): base = 2^30 + rint(clamp(A_ql *
// inv_q, +-2^29)), A_ql = ||c_l||^2 - 2 <q, c_l> (L2) or -<q, c_l> (IP) in FP32
// (fused multiply-adds over ascending dimension); packed like the probe lists
// (maxp: the largest nprobe of the batch).
cudaError_t launch_resid_base(const DevIndex& ix, const float* q, int64_t nq, const QueryParams& qp, int maxp,
                              const int32_t* lists, const float* inv, int32_t* base, cudaStream_t st);
// Residual IVF-PQ index build: rv[slot] = 2 <c_l, y> (L2) or 0 (IP) for each
// slot of list l's code blocks, y the reconstruction of the canonical code
// row codes[off_l + p] (p = the slot's position in the list); 0 for padding;
// cn2[l] = ||c_l||^2 in FP32.
cudaError_t launch_resid_v(const DevIndex& ix, const uint8_t* canon_codes, const int64_t* list_off, float* rv,
                           float* cn2, int64_t nslots, cudaStream_t st);

struct SelectArgs {
    const uint2* region;
    int64_t cap;
    bbc_collector_state* state;
    int64_t kc;
    uint32_t* cand;               // candidates, per QueryParams::coff
    int64_t* cand_count;          // [nq]
    uint2* spill;                 // unused
    QueryParams qp;
    uint32_t tcap = 0;            // set by the fused launch: threshold-bucket keys in shared memory
    const float* rdist = nullptr; // early re-rank: exact distance per region entry (< 0: none), per roff
    float* cand_early = nullptr;  // and per candidate, per coff
};
struct ScanArgs {
    const uint16_t* lut16;        // [nq][M][K]
    const int32_t* lists;         // probe lists, packed per QueryParams::poff
    int nprobe;                   // largest nprobe in the batch (shared-memory sizing)
    int64_t kc;                   // uniform K_c (per-query values in qp)
    int m;                        // buckets
    int sample_min;               // minimum sampled lists
    uint2* region;                // appended (e, list position) pairs, per QueryParams::roff
    int64_t cap;                  // uniform region capacity (per-query values in qp)
    bbc_collector_state* state;   // [nq]
    QueryParams qp;
    int fuse_select;              // 1: the one-CTA-per-query scan runs S7 in its tail (outputs in sel)
    SelectArgs sel;
    int early = 0;                // 1: Algorithm 4's early re-rank in the one-CTA-per-query scan
    const float* q = nullptr;     // [nq][d] queries (the early re-rank's exact distances)
    float* rdist = nullptr;       // exact distance per region entry (< 0: none), per roff
    unsigned long long* early_totals = nullptr;   // [2]: objects scored early, early distances used
    // residual IVF-PQ: each query's table scale and per-(query, list) base, packed like lists
    const float* qinv = nullptr;
    const int32_t* lbase = nullptr;
    int sample_only = 0;          // 1: the one-CTA-per-query scan stops after the codebook (sampled
                                  // objects appended, state written; the tensor-core scan continues)
};
// S4-S6: sample + codebook + scan + push/update, one CTA per query (and S7
// in its tail when fuse_select is set).
cudaError_t launch_scan(const DevIndex& ix, int64_t nq, const ScanArgs& a, cudaStream_t st);
// Same result with G CTAs per query (persistent CTAs over (query, part) items);
// counters: 2 u32 of device scratch.  The state array must be zeroed first.
cudaError_t launch_scan_split(const DevIndex& ix, int64_t nq, const ScanArgs& a, int G, unsigned int* counters,
                              cudaStream_t st);

// Pair form of the scan (batched, two queries per CTA sharing one packed
// table and the union of their lists); perm from launch_pair_plan.  Same
// results as launch_scan.  Supported for 8-bit tables with M <= 32 and 4-bit
// tables with M <= 64 when its shared memory allows two CTAs per SM.
bool scan_pair_supported(const DevIndex& ix, int nprobe);
cudaError_t launch_scan_pair(const DevIndex& ix, int64_t nq, const ScanArgs& a, const int32_t* perm,
                             cudaStream_t st);
// Baseline collectors in place of the result buffer (the comparison of
// Section 4, Exp-3), one CTA per query, the K_c candidates written to
// a.sel.cand / a.sel.cand_count: mode 1 a lazily updated linear buffer, mode
// 2 a binary max-heap in shared memory (stage_cap >= the longest list).
bool scan_collect_supported(const DevIndex& ix, int mode, int nprobe, int64_t kc, uint32_t stage_cap);
cudaError_t launch_scan_collect(const DevIndex& ix, int64_t nq, const ScanArgs& a, int mode, uint32_t stage_cap,
                                cudaStream_t st);
// Pairing plan (k_pair.cu): perm[nq] (query of CTA i at 2i and 2i + 1), from
// the probe lists and the query vectors; scratch holds pair_plan_bytes(nq)
// bytes, perm included (the last quarter).
size_t pair_plan_bytes(int64_t nq);
cudaError_t launch_pair_plan(const float* q, int d, int64_t nq, const QueryParams& qp, const int32_t* lists,
                             void* scratch, int32_t* perm, cudaStream_t st);

// List-grouped form on the tensor cores (k_scan_tc.cu): 4-bit codes, tables
// with entries <= 2047 (a.lut16, and the same entries as FP16 in lut_f16
// [nq][16 M]), plain PQ, m <= 64 buckets.  Runs the one-query scan over the
// sampled lists first (codebooks), then the list-grouped pass.  The same
// candidates and collector state (codebook, tau*, counts of the buckets <=
// tau*) as the one-query scan on the same table; the region may hold more
// appended pairs (tau is refreshed once per item).  The state array must be
// zeroed first; scratch holds scan_tc_plan_bytes(ix, sum of nprobe) bytes.
// The selection (S7) runs after it.
bool scan_tc_supported(const DevIndex& ix, int m);
size_t scan_tc_plan_bytes(const DevIndex& ix, int64_t sum_probe);
cudaError_t launch_scan_tc(const DevIndex& ix, int64_t nq, const ScanArgs& a, const uint16_t* lut_f16,
                           void* scratch, int64_t sum_probe, cudaStream_t st);

// S7: exact threshold bucket, compaction, top-s of the threshold bucket.
cudaError_t launch_select(const DevIndex& ix, int64_t nq, const SelectArgs& a, cudaStream_t st);

struct RerankArgs {
    const float* q;               // [nq][d]
    const uint32_t* cand;         // candidates, per QueryParams::coff
    const int64_t* cand_count;    // [nq]
    int64_t kc;                   // largest K_c in the batch (grid sizing)
    int use_u8;
    float* cdist;                 // per QueryParams::coff
    int k;
    int64_t* out_ids;             // per QueryParams::ooff
    float* out_dists;             // per QueryParams::ooff
    unsigned long long* keys;     // per QueryParams::coff, scratch for large top-k
    QueryParams qp;
    const float* early = nullptr; // per QueryParams::coff: a candidate's exact distance from the scan (< 0: none)
    unsigned long long* early_totals = nullptr;
};
// S8: exact distances of the candidates; S9: k smallest (dist, id), sorted.
cudaError_t launch_rerank(const DevIndex& ix, int64_t nq, const RerankArgs& a, cudaStream_t st);
cudaError_t launch_topk(const DevIndex& ix, int64_t nq, const RerankArgs& a, cudaStream_t st);
// S8 + S9 in one kernel per query (distances kept in shared memory), when
// rerank_topk_fits: the batch's largest K_c distances and ids and the k - 1 +
// 1,024 kept keys fit in one CTA's shared memory.  Same results as the two.
bool rerank_topk_fits(const DevIndex& ix, const RerankArgs& a);
cudaError_t launch_rerank_topk(const DevIndex& ix, int64_t nq, const RerankArgs& a, cudaStream_t st);
// The early re-rank's copy: rows[slot] = vec_u8[ids[slot]] (zero for padding
// slots), norms[slot] = ||row||^2, for nslots = 32 * blocks slots.
cudaError_t launch_early_copy(const DevIndex& ix, int64_t nslots, uint8_t* rows, uint32_t* norms, cudaStream_t st);

// S8, precision form: scores from the low-precision copy with a bound rho per
// candidate, classification against the k-th place, FP32 recheck of the
// uncertain candidates, FP64 for those the FP32 bound cannot place.  All
// arrays are per QueryParams::coff unless noted.
struct PrecArgs {
    float* rho;                   // bound of each score in RerankArgs::cdist
    uint32_t* unc;                // uncertain candidates (ids), compacted
    float* unc_d;                 // FP32 distance of each uncertain candidate (finalize input)
    float* unc_r;                 // its FP32 bound
    int copy_unc;                 // classify copies cdist / rho of the uncertain ones to unc_d / unc_r
    const uint32_t* rc_ids;       // ids the FP32 recheck scores, per coff
    const int64_t* rc_from;       // [nq] first position to score (null: 0)
    const int64_t* sc_from;       // [nq] first candidate the copy scores (pass 1; null: 0)
    const int64_t* rc_count;      // [nq] end position
    float* rc_d;                  // FP32 distances written by the recheck
    float* rc_r;                  // and their bounds
    uint32_t* fin_id;             // final members, compacted
    float* fin_d;                 // their reported distances
    uint32_t* band_id;            // members left to FP64
    double* band_d;               // their FP64 distances
    int64_t* n_fin;               // [nq] final members so far
    int64_t* n_unc;               // [nq] uncertain candidates
    int64_t* item_off;            // [nq + 1] recheck work items (prefix)
    float* qnorm;                 // [nq] ||q||_2 rounded up (may be null for pass 1 alone)
    unsigned long long* totals;   // [4] running totals: candidates, uncertain after the
                                  // low-precision pass, FP64-scored, final members
};
constexpr int kPrecItem = 512;    // candidates per recheck work item
// Builds the copy (prec 1 BF16, 2 FP8-E4M3) and the per-vector metadata.
cudaError_t launch_prec_copy(const DevIndex& ix, int prec, void* rows, float4* meta, cudaStream_t st);
// Scores and bounds of the candidates (pass 1), written to a.cdist and p.rho.
cudaError_t launch_prec_score(const DevIndex& ix, int64_t nq, const RerankArgs& a, const PrecArgs& p,
                              cudaStream_t st);
// Classification (pass 2), the recheck plan and the FP32 recheck (pass 3),
// the FP32 classification with the FP64 decision (pass 4).  Afterwards
// p.fin_id / p.fin_d / p.n_fin hold the min(k, count) final members.
cudaError_t launch_prec_classify(const DevIndex& ix, int64_t nq, const RerankArgs& a, const PrecArgs& p,
                                 cudaStream_t st);
cudaError_t launch_prec_plan(int64_t nq, const PrecArgs& p, cudaStream_t st);
cudaError_t launch_prec_recheck(const DevIndex& ix, int64_t nq, const RerankArgs& a, const PrecArgs& p,
                                cudaStream_t st);
cudaError_t launch_prec_finalize(const DevIndex& ix, int64_t nq, const RerankArgs& a, const PrecArgs& p,
                                 cudaStream_t st);

// ---- 1-bit sign quantizer and the bounded re-rank (S9b) ----
// out[i][r] = sum_j P[r][j] (A[row(i)][j] - sub(i)[j]) in FP64 for rows i < n,
// row(i) = rows ? rows[i] : i (rows < 0 are skipped), sub(i) = centroid of
// lists[i] when lists is given.
cudaError_t launch_rotate_f64(const float* A, const int64_t* rows, const int32_t* lists, const float* centroids,
                              const float* P, int64_t n, int d, double* out, cudaStream_t st);
// Codes and factors of slots [s0, s0 + n) from their rotated residuals R (FP64
// [n][d]); rows / lists: vector id (-1 for padding) and list of every slot.
cudaError_t launch_sign_factors(const double* R, int64_t s0, int64_t n, int d, const int64_t* rows,
                                const int32_t* lists, const float* vec, const float* cent, uint32_t* codes,
                                float4* fac, cudaStream_t st);

struct SignArgs {
    const double* qrot;           // [nq][d] P q in FP64
    const float* q;               // [nq][d]
    const int32_t* lists;         // probe lists, per QueryParams::poff
    int nprobe;
    int k;                        // uniform k (per-query values in qp)
    int m;                        // buckets
    int sample_min;               // minimum sampled lists
    float scale;                  // scale of the residual term (1 = hard bounds)
    int est;                      // 0: hard bounds; 1: the RaBitQ estimator's probabilistic bounds
    float eps0;                   // its confidence parameter epsilon_0
    uint4* region;                // {lb key, ub key, slot, 0}, per QueryParams::roff
    int64_t cap;
    int64_t* pushed;              // [nq]
    int64_t* scanned;             // [nq]
    float* dbg_lb;                // bounds of every scanned object (debug form), per roff, or null
    float* dbg_ub;
    uint32_t* prep;               // per (query, probed list) records, sign_prep_bytes(ix, sum of nprobe)
    QueryParams qp;
};
size_t sign_prep_bytes(const DevIndex& ix, int64_t sum_probe);
// Query preparation per (query, probed list), then the scan with the result buffer.
cudaError_t launch_sign_scan(const DevIndex& ix, int64_t nq, const SignArgs& a, cudaStream_t st);

struct SignSelectArgs {
    const uint4* region;
    const int64_t* pushed;
    const int64_t* scanned;
    uint32_t* clist;              // ids to re-rank, per coff (capacity cap)
    int64_t* n_b;                 // [nq] size of the first round
    int64_t* n_c;                 // [nq] ids in clist
    uint32_t* rest_key;           // lb keys of S minus the first round, per coff
    uint32_t* rest_id;
    int64_t* n_rest;              // [nq]
    const float* cd;              // FP32 distances of clist (after the first recheck)
    const float* cr;              // and bounds
    unsigned long long* totals;   // [4]
    QueryParams qp;
    float first = 2.f;            // first-round size, a multiple of k
};
cudaError_t launch_sign_select(const DevIndex& ix, int64_t nq, const SignSelectArgs& a, cudaStream_t st);
cudaError_t launch_sign_filter(const DevIndex& ix, int64_t nq, const SignSelectArgs& a, cudaStream_t st);

}  // namespace bbc

// Accessors into the host-side index object (defined in api.cu).
namespace bbc {
int api_error(int code, const char* msg);
int api_check_search_args(const bbc_index* ix, const void* queries, int64_t nq, int k, int nprobe,
                          const void* out_ids, const void* out_dists);
const DevIndex& index_dev(const bbc_index* ix);
int index_device(const bbc_index* ix);
int64_t index_cap(const bbc_index* ix, int nprobe);
int index_buckets(const bbc_index* ix);
int index_lut_levels(const bbc_index* ix);
int index_sample_lists(const bbc_index* ix);
}  // namespace bbc
