/*
 * bbc.h -- C ABI of the GB300 (sm_103a) search path for large-k ANN queries
 * on IVF indexes with a bucket-based result collector (BBC, arxiv 2604.01960).
 *
 * Problem (Section 2, "Problem Statement"): given N d-dimensional vectors, an
 * indexing phase builds a structure; a query q asks for the k nearest vectors
 * under a metric.  Here the structure is an IVF partition with PQ codes, and
 * the query path is: coarse probe -> PQ lookup table -> quantised-distance
 * scan with the bucket-based result buffer (Algorithm 1) -> exact re-rank of
 * the collected candidates -> final top-k.
 *
 * Conventions shared by every entry point
 *  - Every function returns an int status: BBC_OK (0) or a negative BBC_ERR_*.
 *    bbc_last_error() returns a thread-local message for the last failure.
 *  - Argument errors are reported before anything is enqueued on the stream.
 *  - "device" pointers are CUDA device (or managed) memory on the index's
 *    device; "host" pointers are ordinary host memory.  The caller owns every
 *    buffer it passes; the library owns the index and its workspaces.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device-pointer entry points are asynchronous: they return
 *    after enqueuing work on `stream`.  Device-side faults that the kernels
 *    detect (a collector region overrun) are latched in a per-index status
 *    word that bbc_stream_status() reads after synchronising the stream.
 *  - Distances are squared L2 (metric L2) or the negated inner product
 *    -<q, v> (metric IP); results are ascending by (distance, id).  When fewer
 *    than k vectors are scanned the tail is padded with id -1 and +inf
 *    (Algorithm 1's Update returns "infinity" when fewer than k are buffered).
 *  - Ties are broken by the smaller id everywhere: list id in the probe,
 *    vector id among equal estimated distances and among equal exact ones.
 */
#ifndef BBC_H
#define BBC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BBC_OK 0
#define BBC_ERR_ARG (-1)        /* invalid argument (null pointer, k <= 0, nprobe out of range, ...) */
#define BBC_ERR_IO (-2)         /* index file cannot be opened or read */
#define BBC_ERR_FORMAT (-3)     /* index file or arrays are malformed */
#define BBC_ERR_OOM (-4)        /* host or device allocation failed */
#define BBC_ERR_CUDA (-5)       /* a CUDA runtime call failed */
#define BBC_ERR_CAPACITY (-6)   /* a device-side capacity check tripped */
#define BBC_ERR_TIMEOUT (-7)    /* a bounded device-side wait ran out */
#define BBC_ERR_BUSY (-8)       /* resource in use */
#define BBC_ERR_UNSUPPORTED (-9) /* configuration this build does not handle */

#define BBC_METRIC_L2 0
#define BBC_METRIC_IP 1
#define BBC_QUANT_PQ 0
#define BBC_QUANT_SIGN 1
#define BBC_QUANT_PQ_RESIDUAL 2   /* PQ codes of each object's residual o - c_l */

typedef struct bbc_index bbc_index;   /* opaque, owned by the library */

/* Host-side description of an IVF-PQ index (Section 2, "Quantization"):
 * nlist k-means centroids, inverted lists of vector ids, PQ with pq_m
 * sub-spaces of d/pq_m dimensions and 2^pq_bits codewords each, of the
 * vectors themselves or (residual = 1) of each vector's residual o - c_l to
 * its list's centroid.  For a residual index the estimated distance of an
 * object is its distance from the query to c_l + y (y the code's
 * reconstruction): the query's table sum, plus per (query, list) ||c_l||^2 -
 * 2 <q, c_l> (L2) or -<q, c_l> (IP), plus per object 2 <c_l, y> (L2), the
 * last computed on the device at creation.  All pointers are HOST pointers;
 * bbc_index_create copies what it needs. */
typedef struct {
    int64_t n;                 /* number of vectors, 1 <= n < 2^32 - 1 */
    int32_t d;                 /* dimension, multiple of pq_m */
    int32_t nlist;             /* number of inverted lists */
    int32_t metric;            /* BBC_METRIC_L2 or BBC_METRIC_IP */
    int32_t pq_m;              /* sub-spaces: 8, 16, 32, 64, 96 or 128 (multiple of 32 above 32) */
    int32_t pq_bits;           /* 8, or 4 with pq_m a multiple of 32 */
    const float* centroids;    /* [nlist * d] row-major */
    const int64_t* list_offsets; /* [nlist + 1], list l = positions [off[l], off[l+1]) */
    const int64_t* ids;        /* [n] vector id at each list position */
    const uint8_t* codes;      /* [n * pq_m * pq_bits / 8] one row per list position; 8-bit:
                                  byte m = code of sub-space m; 4-bit: byte m/2, low nibble
                                  for even m, high nibble for odd m */
    const float* codebooks;    /* [pq_m * 2^pq_bits * (d/pq_m)], [m][j][i] */
    const float* vectors;      /* [n * d] row-major by id (for the exact re-rank) */
    int32_t residual;          /* 0: PQ of the vectors; 1: PQ of o - c_l (residual IVF-PQ) */
} bbc_index_host;

typedef struct {
    int64_t n;
    int32_t d, nlist, metric, pq_m, pq_bits;
    int32_t max_list_len;      /* longest inverted list */
    int32_t vectors_u8_exact;  /* 1 if every component is an integer in [0,255] (exact u8 copy kept) */
    int32_t device;
    int64_t device_bytes;      /* bytes of device memory the index holds */
    int32_t quantizer;         /* BBC_QUANT_PQ, BBC_QUANT_SIGN or BBC_QUANT_PQ_RESIDUAL */
    int32_t reserved;
} bbc_index_info_t;

/* Build a device-resident index from host arrays (copied to `device`).
 * Validates the arrays (offsets monotone and ending at n, ids in [0,n) and a
 * permutation, pq shape supported): BBC_ERR_FORMAT / BBC_ERR_ARG otherwise. */
int bbc_index_create(const bbc_index_host* h, int device, bbc_index** out);

/* Read an index file and create the device index (the paper's indexing
 * phase, Section 2, done offline; this call only loads its result).  Format
 * "BBCIDX01", little-endian: a 64-byte header {magic[8], u32 version = 1,
 * u32 quantizer, u32 metric, u32 d, u64 n, u32 nlist, u32 pq_m, u32 pq_bits},
 * then arrays each starting on a 64-byte boundary.  Quantizer BBC_QUANT_PQ
 * (or BBC_QUANT_PQ_RESIDUAL, the same arrays with codes of o - c_l):
 * centroids, list_offsets, ids, codes, codebooks, vectors, laid out as in
 * bbc_index_host.  Quantizer BBC_QUANT_SIGN (pq_m = pq_bits = 0):
 * centroids, list_offsets, ids, rotation, vectors, as in bbc_sign_host.
 * BBC_ERR_IO when the file cannot be opened, BBC_ERR_FORMAT on a bad or
 * truncated file, and the errors of bbc_index_create(_sign). */
int bbc_index_load(const char* path, int device, bbc_index** out);

/* Host-side description of an IVF index with the 1-bit sign quantizer of the
 * bounded re-rank (Section 3.4; the paper cites RaBitQ without stating its
 * estimator, so the bounds are this library's hard bounds, see bbc_search).
 * The library derives, on the device, for every vector o of list l the codes
 * s = sign(P (o - c_l)) and the factors alpha = mean |P (o - c_l)|_i,
 * e = ||P (o - c_l) - alpha s||, ||o - c_l||^2.  HOST pointers, copied. */
typedef struct {
    int64_t n;                 /* number of vectors, 1 <= n < 2^32 - 1 */
    int32_t d;                 /* dimension, a multiple of 32, at most 2048 */
    int32_t nlist;
    int32_t metric;            /* BBC_METRIC_L2 */
    const float* centroids;    /* [nlist * d] */
    const int64_t* list_offsets; /* [nlist + 1] */
    const int64_t* ids;        /* [n] vector id at each list position */
    const float* rotation;     /* [d * d] row-major P (orthonormal rows); r = P u */
    const float* vectors;      /* [n * d] row-major by id */
} bbc_sign_host;

/* Build a device index with sign codes.  BBC_ERR_UNSUPPORTED for inner
 * product or d not a multiple of 32 / above 2048.  On such an index
 * bbc_search, bbc_search_host and bbc_search_ex run the bounded re-rank; the
 * other per-step calls return BBC_ERR_UNSUPPORTED. */
int bbc_index_create_sign(const bbc_sign_host* h, int device, bbc_index** out);

int bbc_index_free(bbc_index* ix);
int bbc_index_info(const bbc_index* ix, bbc_index_info_t* out);

/* Search parameters, settable per index.  Keys:
 *   "kc_ratio"     K_c = ceil(kc_ratio * k) candidates are collected by
 *                  estimated distance and re-ranked (the paper's n_cand,
 *                  Section 2 and Table 4).  Default 1.5; must be >= 1.
 *   "buckets"      m, buckets of the result buffer (Section 3.2), 2..256.  Default 64.
 *   "sample_lists" minimum number of nearest lists sampled to build the
 *                  codebook (Section 3.2: "5-10 nearest clusters").  Default 8.
 *   "rerank"       0 = FP32 vectors, 1 = exact u8 copy (only when
 *                  vectors_u8_exact).  Default: 1 when available.
 *   "workspace_mb" device workspace budget per call; queries are processed in
 *                  chunks that fit.  Default 8192.
 *   "profile"      1 = record per-stage CUDA events (see bbc_profile_read).  Default 0.
 *   "split"        CTAs per query in the scan: 1 = one CTA owns each query, G >= 2 =
 *                  G CTAs share each query (persistent CTAs over (query, part)
 *                  items, collector state in global memory), 0 = automatic (split
 *                  when the batch is too small to fill the GPU).  Same results
 *                  either way.  Default 0.
 *   "pair"         1 = the scan runs two queries per CTA where the table shape
 *                  allows it (8-bit codes with pq_m <= 32, 4-bit with pq_m <= 64):
 *                  queries are paired by nearest list and vector distance, the
 *                  two uint16 tables share one shared-memory table (one in the
 *                  low, one in the high half of each word) and the union of
 *                  their probed lists is streamed once, so a code row serves
 *                  both queries.  0 = one query per CTA.  Applies when "split"
 *                  gives one CTA per query.  Same results either way.  Default 0.
 *   "collector"    the top-K_c collector of the scan: 0 (default) = the
 *                  bucket-based result buffer (Section 3.2, Algorithm 1); the
 *                  baselines it is compared with (Section 4, Exp-3): 1 = a
 *                  lazily updated linear buffer (objects below the current
 *                  threshold appended; after each list the threshold becomes
 *                  the K_c-th smallest buffered estimate and the buffer is
 *                  compacted), 2 = a binary max-heap of the K_c smallest
 *                  (estimate, id) in shared memory.  Same candidates with
 *                  every collector; 1 and 2 run one CTA per query and take
 *                  8-bit tables with pq_m <= 32 or 4-bit tables with pq_m <= 64
 *                  (2 also needs the heap in shared memory: K_c up to about
 *                  18,000), else BBC_ERR_UNSUPPORTED at search time.
 *   "early_rerank" 1 = the early re-ranking of Algorithm 4 (Section 3.3,
 *                  "Integrating with IVF+PQ"): while a list is scanned, an
 *                  appended object whose bucket lies below the predicted
 *                  threshold bucket tau_pred (the bucket of the ceil(f n_cand)-th
 *                  smallest estimate so far, f the scanned share of the probed
 *                  objects) gets its exact distance at once, from a copy of
 *                  the u8 vectors in list order (the code and vector of an
 *                  object stored alike, read while the list is hot); the
 *                  re-rank then skips the candidates that have one.  Setting
 *                  it builds that copy (waits for all work on the device).
 *                  Needs an L2 index with the exact u8 copy, d a multiple of
 *                  16 up to 256 and a table of at most 64 KB, else
 *                  BBC_ERR_UNSUPPORTED; applies with one CTA per query and the
 *                  result buffer.  Candidates and results are unchanged (the
 *                  exact distances are the u8 re-rank's, bit for bit); see
 *                  bbc_early_stats.  Default 0.
 *   "graphs"       1 = bbc_search captures the launch sequence of each call shape
 *                  (pointers, sizes, parameters, stream) into a CUDA graph the
 *                  first time and replays it afterwards (not on the legacy
 *                  default stream).  Default 0.
 *   "probe_gemm"   1 = approximate probe scores on the tensor cores (tcgen05 BF16
 *                  GEMM with a 3-term split), 0 = FP32 SIMT.  Either way the
 *                  probe result is exact (see bbc_probe).  Default 1.
 *   "precision"    precision form of the re-rank (step S8 with a low-precision
 *                  copy; the paper re-ranks "with exact distances", Section 2,
 *                  and leaves their precision open): 0 = FP32 rows (default),
 *                  1 = BF16 copy, 2 = FP8-E4M3 copy with one scale per vector.
 *                  Setting 1 or 2 builds the copy on the device (waits for all
 *                  work on the device first; not to be called while other
 *                  threads search this index).  Candidates are scored from the
 *                  copy with a rigorous per-candidate bound; only those whose
 *                  interval straddles the k-th place are re-scored from the
 *                  FP32 rows, and FP64 decides what FP32 cannot.  The result
 *                  set is the same as with the FP32 re-rank decided in FP64;
 *                  reported distances of members placed by the copy's bound
 *                  are the copy's scores (see bbc_rerank_bounds).  Applies when
 *                  the exact u8 re-rank is not in use.
 *   "lut_levels"   top level T of the integer lookup tables (step S3): entry =
 *                  min(T, floor((L - lo_m) T / span + 0.5)), 1..65535.
 *                  Default 65535 (the uint16 table).
 *   "scan_tc"      1 = the list-grouped form of the scan on the tensor cores
 *                  (plain, not residual, 4-bit PQ with pq_m = 32, 64 or 128;
 *                  buckets <= 64): a batch's (query, probed list) pairs
 *                  are grouped by list on the device, and a CTA stages a tile
 *                  of 256 code rows of one list once, as one-hot FP16 rows,
 *                  for up to 128 of the queries that probe it; tcgen05.mma
 *                  contracts them with the queries' tables (FP32
 *                  accumulation in tensor memory), and the result buffer's
 *                  Push runs on the accumulators.  Setting 1 lowers
 *                  "lut_levels" to 2047 when it is larger: such entries are
 *                  integers FP16 holds exactly and every sum of them stays
 *                  below 2^24, so the estimated distances equal the integer
 *                  table sums and the candidates equal those of the one-query
 *                  scan on the same table.  Applies with the result buffer
 *                  ("collector" 0) and without "early_rerank"; a search whose
 *                  index or buckets do not fit returns BBC_ERR_UNSUPPORTED.
 *                  Default 0.
 *   "rerank_fused" 1 = the exact re-rank (step S8) and the top-k (step S9) run
 *                  as one kernel, a CTA per query keeping its candidates'
 *                  distances in shared memory, when the largest K_c of the
 *                  batch and k fit there (8 K_c + 8 (k + 1024) + 5 d bytes <=
 *                  215 KB; K_c = 15,000 with k = 10,000 does); otherwise, and
 *                  with 0, two kernels with the distances in the workspace.
 *                  Same results either way; with "profile" the fused kernel's
 *                  time is the re-rank stage's.  Default 0: at K_c = 15,000
 *                  the kernel holds one CTA per SM, so each query's top-k
 *                  phase (bound by instructions and barriers) runs with no
 *                  other query beside it and no row loads in flight
 *                  (measured 4.6 ms against 3.1 ms for the two kernels per
 *                  10,000 queries on 1M x 128).
 *   "region_cap"   entries of each query's collector region (the buffer the
 *                  scan appends (estimated distance, position) pairs to).
 *                  0 (default) = the total length of the nprobe longest lists,
 *                  which holds every scanned object.  A smaller value bounds
 *                  the workspace; appends past it are dropped and latch
 *                  BBC_ERR_CAPACITY in the status word (bbc_stream_status),
 *                  and that call's results are then incomplete.
 *   "bound_scale"  sign-code indexes: factor on the residual term ||q'|| e of
 *                  the bounds, in (0, 1].  1 (default) gives hard bounds and
 *                  results equal to the exact top-k of the probed lists;
 *                  smaller values narrow the intervals in the spirit of
 *                  RaBitQ's probabilistic bound and may drop true members.
 *   "estimator"    sign-code indexes: 0 (default) = hard bounds (above); 1 =
 *                  the RaBitQ estimator of <q', r> (Section 3.4 builds on it;
 *                  Section 4.1 runs it with epsilon_0 = 1.9): the estimate
 *                  ||r||^2 / (d alpha) <s, q~> with the probabilistic bound
 *                  epsilon_0 / sqrt(d - 1) ||q'|| ||r|| sqrt(1 - <o_bar, o_r>^2)
 *                  / <o_bar, o_r> plus the 4-bit query's share at the same
 *                  confidence.  The true distance lies inside with high
 *                  probability, not always; the result is the two-round
 *                  bounded re-rank on these bounds (exact distances returned).
 *   "epsilon0"     epsilon_0 of the estimator mode, in (0, 100].  Default 1.9.
 *   "first_round"  sign-code indexes: the bounded re-rank's first round
 *                  re-ranks the first_round * k objects of S = {lb <= U_k}
 *                  with the smallest interval centres, in [1, 64]; the second
 *                  round takes the rest of S whose lb is <= the k-th smallest
 *                  upper bound of the first round's distances.  Default 2.
 *                  Results never depend on it (with hard bounds), only the
 *                  number of exact distances computed.
 * Unknown key or out-of-range value: BBC_ERR_ARG. */
int bbc_set_param(bbc_index* ix, const char* key, double value);
int bbc_get_param(const bbc_index* ix, const char* key, double* value);

/* Full search for nq queries (the hot path of Algorithms 1 and 4 with the
 * sort-free re-rank of the collected candidates).
 *   queries   device f32 [nq * d], row-major
 *   k         results per query, >= 1
 *   nprobe    lists probed per query, 1..nlist
 *   out_ids   device i64 [nq * k], ascending by (dist, id); -1 padding
 *   out_dists device f32 [nq * k]; +inf padding
 * Asynchronous on `stream`.  The first call with a given shape may allocate
 * the index's workspace (cudaMalloc); later calls of equal or smaller shape
 * do not. */
int bbc_search(bbc_index* ix, const float* queries, int64_t nq, int32_t k, int32_t nprobe,
               int64_t* out_ids, float* out_dists, void* stream);

/* Mixed batch (batched form with uneven shapes): query q has its own k[q]
 * and nprobe[q] (HOST arrays of nq int32, k[q] >= 1, 1 <= nprobe[q] <= nlist)
 * and K_c = max(k[q], ceil(kc_ratio * k[q])).  Results are packed in query
 * order: query q's k[q] results start at sum_{j<q} k[j] in out_ids / out_dists
 * (device arrays holding sum k entries).  Each query's results are identical
 * to those of a bbc_search call for that query alone.  Asynchronous on
 * `stream` (the small per-query tables are copied from host memory). */
int bbc_search_ex(bbc_index* ix, const float* queries, int64_t nq, const int32_t* k, const int32_t* nprobe,
                  int64_t* out_ids, float* out_dists, void* stream);

/* Same as bbc_search with HOST query and output buffers: copies the queries
 * to the device, searches, copies the results back, and synchronises
 * `stream` before returning. */
int bbc_search_host(bbc_index* ix, const float* queries, int64_t nq, int32_t k, int32_t nprobe,
                    int64_t* out_ids, float* out_dists, void* stream);

/* Autotuner for the batched form: times the scan schedules ("split", CTAs
 * per query, and "pair", two queries per CTA) and then "buckets" (m, the
 * result buffer's bucket count) for this call shape on `nq` device queries,
 * and keeps the fastest
 * on the index.  With cache_path (may be NULL) the choice is looked up in,
 * or appended to, a JSON-lines file keyed by the index shape and the call
 * shape, so later processes skip the timing.  Allocates its own output
 * buffers and synchronises `stream`.  out_ms (host, may be NULL) receives
 * the best time per call (0 when taken from the cache).  The results of a
 * search never depend on these settings, only its speed. */
int bbc_autotune(bbc_index* ix, const float* queries, int64_t nq, int32_t k, int32_t nprobe,
                 const char* cache_path, double* out_ms, void* stream);

/* ---- stage entry points (each one row of the hot path; device pointers) ---- */

/* Approximate probe scores (the pruning step of the coarse probe):
 * out_scores device f32 [nq * nlist], a[q][l] = ||c_l||^2 - 2<q, c_l> (L2) or
 * -<q, c_l> (IP), from the tensor-core GEMM ("probe_gemm" = 1) or FP32 SIMT.
 * |a + ||q||^2 - s| stays within the bound bbc_probe uses, s = the FP64 score. */
int bbc_probe_scores(bbc_index* ix, const float* queries, int64_t nq, float* out_scores, void* stream);

/* Coarse probe (Section 2: route q to the n_probe nearest clusters;
 * Algorithm 4 scans them nearest first).  out_lists: device i32
 * [nq * nprobe], ascending by (FP64 score, list id), where the score is
 * sum_i (q_i - c_i)^2 (L2) or -sum_i q_i c_i (IP) evaluated in FP64 in
 * ascending dimension order. */
int bbc_probe(bbc_index* ix, const float* queries, int64_t nq, int32_t nprobe,
              int32_t* out_lists, void* stream);

/* PQ lookup table (Section 2, step (1)) quantised to uint16:
 * out_lut16 device u16 [nq * pq_m * 2^pq_bits], [q][m][j].
 * FP32 entry L[m][j] = sum_i (q_i - y_i)^2 (or -sum_i q_i y_i) in ascending i,
 * lo_m = min_j L[m][j], span = max_m (max_j L[m][j] - lo_m),
 * entry = min(65535, floor((L - lo_m) * (65535 / span) + 0.5)), 0 when span = 0. */
int bbc_lut(bbc_index* ix, const float* queries, int64_t nq, uint16_t* out_lut16, void* stream);

/* Per-query state of the bucket-based result buffer after the scan. */
typedef struct {
    uint32_t d_min, d_max;     /* codebook range from the sampled lists */
    int32_t sh;                /* equal-width bin width delta = 2^sh */
    int32_t m;                 /* buckets */
    int32_t sample_lists;      /* lists in the codebook sample */
    int32_t tau;               /* final threshold bucket (m = infinity) */
    int64_t sample_size;       /* objects in the sample */
    int64_t scanned;           /* S_q, objects scanned */
    int64_t pushed;            /* objects appended to the buffer */
    int64_t below;             /* objects in buckets < tau */
    int64_t kc;                /* candidates requested */
    uint32_t hist[256];        /* per-bucket counts of appended objects */
    uint8_t map[256];          /* equal-width bin -> equal-depth bucket */
} bbc_collector_state;

/* Probe + LUT + scan with the bucket-based result buffer + final selection
 * (Algorithm 1: Push / Update / Collect).  Produces the K_c candidates with
 * the smallest (estimated distance, id) among the scanned objects.
 *   probe_lists   device i32 [nq * nprobe] from bbc_probe
 *   kc            candidates per query (K_c >= 1)
 *   out_ids       device u32 [nq * kc], unordered within a query
 *   out_count     device i64 [nq], min(kc, S_q)
 *   out_state     device bbc_collector_state [nq], or NULL */
int bbc_collect(bbc_index* ix, const float* queries, int64_t nq, int32_t nprobe,
                const int32_t* probe_lists, int64_t kc, uint32_t* out_ids, int64_t* out_count,
                bbc_collector_state* out_state, void* stream);

/* Allocation-free variant of bbc_collect.  The paper has no counterpart:
 * it exists for callers that cannot call cudaMalloc -- programs that budget
 * every byte of device memory themselves and forbid libraries to allocate
 * (for example a server that splits HBM between models up front), and
 * latency-critical threads, where a cudaMalloc can block in the driver and
 * synchronise the device.  Same arguments and results as bbc_collect.  Its
 * scratch (lookup tables, the collector state when out_state is NULL, and
 * the appended (estimate, id) pairs) is one static device array of
 * BBC_STATIC_SCRATCH_BYTES, which every GPU that loads the library holds
 * until the process exits; the call allocates nothing.  A call that needs
 * more scratch than that -- about nq * (2 * pq_m * 2^pq_bits + 1344 +
 * 8 * cap) bytes, cap = total length of the nprobe longest lists, plus
 * nq * 4 * (1 + nprobe) on a residual index -- returns
 * BBC_ERR_ARG before launching anything.  The first call on a device looks
 * up the array's device address with that device current and keeps it for
 * the life of the process; make that first call before any stream capture,
 * and do not use this entry point after cudaDeviceReset (the array may move).
 * All calls share the array, so calls whose kernels overlap on the GPU race:
 * order them on one stream.  The scan always runs one CTA per query (the
 * split form needs zeroed counters), so small batches run slower than with
 * bbc_collect, and these calls are not recorded by bbc_profile_read. */
#define BBC_STATIC_SCRATCH_BYTES (64u * 1024u * 1024u)
int bbc_collect_static(bbc_index* ix, const float* queries, int64_t nq, int32_t nprobe,
                       const int32_t* probe_lists, int64_t kc, uint32_t* out_ids, int64_t* out_count,
                       bbc_collector_state* out_state, void* stream);

/* Exact re-rank of candidates and final top-k (Algorithm 4, last two lines).
 *   cand_ids   device u32 [nq * kc]; cand_count device i64 [nq]
 *   out_ids / out_dists as in bbc_search.
 * With "precision" set, the precision form of the re-rank runs instead. */
int bbc_rerank_topk(bbc_index* ix, const float* queries, int64_t nq, const uint32_t* cand_ids,
                    const int64_t* cand_count, int64_t kc, int32_t k, int64_t* out_ids,
                    float* out_dists, void* stream);

/* First pass of the precision re-rank alone: for each candidate i < count of
 * each query, the score d^ from the low-precision copy (squared L2, or minus
 * the inner product) and a bound rho with |d^ - d64| <= rho, d64 being the
 * FP64 distance of the FP32-stored vector.
 *   cand_ids  device u32 [nq * kc]; cand_count device i64 [nq]
 *   out_dist, out_rho  device f32 [nq * kc] (entries past count untouched)
 * BBC_ERR_ARG when no copy has been built ("precision" 0). */
int bbc_rerank_bounds(bbc_index* ix, const float* queries, int64_t nq, const uint32_t* cand_ids,
                      const int64_t* cand_count, int64_t kc, float* out_dist, float* out_rho,
                      void* stream);

/* The low-precision copy itself, for inspection: out_rows device buffer of
 * n * dpad elements (dpad = d rounded up to a multiple of 16; BF16 bits as
 * u16 for "precision" 1, E4M3 bytes for 2; row i = vector id i, zero padded),
 * out_meta device f32 [n * 4] = {scale s (1 for BF16), e_v = ||v - s v~||_2
 * rounded up, ||v||_2 rounded up, 0}.  BBC_ERR_ARG without a copy. */
int bbc_precision_copy(bbc_index* ix, void* out_rows, float* out_meta, void* stream);

/* Bounds of the sign quantizer for every object of the probed lists, in probe
 * order (list by list, list positions ascending): the debug form of the
 * bounded scan.  probe_lists device i32 [nq * nprobe]; out_lb / out_ub device
 * f32 [nq * stride]; out_count device i64 [nq] = objects scanned (entries
 * past stride are dropped and latch a region overrun).  Bounds enclose
 * ||q - o||^2 (with "bound_scale" 1). */
int bbc_sign_bounds(bbc_index* ix, const float* queries, int64_t nq, int32_t nprobe,
                    const int32_t* probe_lists, int64_t stride, float* out_lb, float* out_ub,
                    int64_t* out_count, void* stream);

/* Running totals of the bounded re-rank since the last reset (synchronises
 * the device): out4[0] objects scanned, [1] objects in S = {lb <= U_k},
 * [2] exact distances computed (both rounds), [3] queries. */
int bbc_bounded_stats(bbc_index* ix, int64_t* out4, int reset);

/* Running totals of the early re-rank ("early_rerank") since the last reset
 * (synchronises the device): out2[0] objects given their exact distance
 * during the scan, [1] candidates whose re-rank used one. */
int bbc_early_stats(bbc_index* ix, int64_t* out2, int reset);

/* Running totals of the precision re-rank since the last reset (synchronises
 * the device): out4[0] candidates scored from the copy, [1] candidates
 * re-scored in FP32, [2] candidates scored in FP64, [3] final members. */
int bbc_precision_stats(bbc_index* ix, int64_t* out4, int reset);

/* ---- serving: continuous batching of single-query requests ----
 * A server owns one worker thread and `streams` CUDA streams.  Requests
 * (one query, its own k and nprobe) queue on the host; whenever a stream is
 * free the worker admits waiting requests, oldest first, into one mixed batch
 * (bbc_search_ex) while the batch has fewer than max_batch requests and the
 * candidate-buffer bytes of all admitted, unfinished requests stay within
 * cand_bytes_budget (a lone request larger than the budget is admitted when
 * nothing else is in flight).  Batches on different streams overlap on the
 * GPU, so requests that arrive while others run start as soon as a stream
 * and memory free up.  Each request's result equals bbc_search on that query
 * alone.  Candidate-buffer bytes of a request = 8 * (total length of its
 * nprobe longest lists) + 8 * K_c. */
typedef struct bbc_server bbc_server;
typedef struct {
    int32_t max_batch;            /* requests per batch, >= 1 */
    int32_t streams;              /* batches in flight, 1..16 */
    int64_t cand_bytes_budget;    /* admission budget in bytes, >= 1 */
} bbc_serve_config;
typedef struct {
    int64_t submitted, completed, batches;
    int64_t inflight_bytes_peak;  /* largest admitted total observed */
    double p50_ms, p99_ms;        /* submit -> result ready, over completed requests */
    double mean_batch;            /* requests per batch */
    double wall_s;                /* time since start */
} bbc_serve_stats_t;
int bbc_serve_start(bbc_index* ix, const bbc_serve_config* cfg, bbc_server** out);
/* host_query: d floats (copied).  Returns a ticket for bbc_serve_poll. */
int bbc_serve_submit(bbc_server* sv, const float* host_query, int32_t k, int32_t nprobe, uint64_t* ticket);
/* Wait up to timeout_ms (< 0: forever) for the ticket; on success copies its
 * k ids and distances into the HOST buffers and forgets the ticket.
 * BBC_ERR_TIMEOUT if not ready in time, BBC_ERR_ARG for an unknown ticket. */
int bbc_serve_poll(bbc_server* sv, uint64_t ticket, int64_t* ids, float* dists, int32_t timeout_ms);
int bbc_serve_stats(bbc_server* sv, bbc_serve_stats_t* out);
/* Finishes in-flight batches, stops the worker and frees the server. */
int bbc_serve_stop(bbc_server* sv);

/* Per-stage timing (the GPU counterpart of the paper's time breakdown,
 * Figure 2).  With parameter "profile" = 1 the library records a CUDA event
 * pair on the launch stream around every kernel it launches.  This call
 * waits for the recorded events, adds their elapsed times per stage into
 * stage_ms[BBC_NUM_STAGES] (host array, may be NULL), writes the number of
 * kernels launched since the last reset into *launches (may be NULL; counted
 * whether or not profiling is on), and clears both when reset != 0.
 * Stages: 0 probe scores, 1 probe selection, 2 lookup table, 3 scan +
 * result buffer, 4 final selection, 5 re-rank (the copy's scores in the
 * precision form), 6 top-k, 7 precision classification and FP64 decision,
 * 8 precision FP32 recheck. */
#define BBC_NUM_STAGES 9
int bbc_profile_read(bbc_index* ix, double* stage_ms, int64_t* launches, int reset);

/* Synchronise `stream`, then read and clear the index's device status word.
 * Returns BBC_OK, or BBC_ERR_CAPACITY if a kernel latched an overrun. */
int bbc_stream_status(bbc_index* ix, void* stream);

/* Thread-local message describing the last error returned on this thread. */
const char* bbc_last_error(void);

/* Library version string. */
const char* bbc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* BBC_H */
