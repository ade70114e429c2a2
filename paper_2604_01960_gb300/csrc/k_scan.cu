// S4-S6: quantised-distance scan of the probed lists fused with the
// bucket-based result buffer (Section 3.2, Algorithm 1), one CTA per query.
//
// Phase A  stage the query's uint16 lookup table in shared memory and lay out
//          its probed lists (nearest first) as a sequence of 32-vector blocks.
// Phase B  sample: scan the first lists in probe order -- at least
//          min(sample_min, nprobe) of them, extended until they hold
//          min(K_c, S_q) vectors -- and append every (estimated distance, id)
//          to the query's region (threshold = infinity, as Algorithm 1 starts).
// Phase C  codebook (Section 3.2, "Codebook Generation Based on Estimated
//          Distance"): d_min = smallest, d_max = t-th smallest sampled
//          distance with t = min(K_c, sample size); n_ew = 256 equal-width
//          bins of width 2^sh over [d_min, d_max]; bin(e) = clamp((e - d_min)
//          >> sh, 0, 255) (Eq. remap); an equal-depth remap map[256] -> [0, m)
//          from the bins' cumulative counts; counts of the sample and the
//          threshold bucket tau (Update, Algorithm 1: first bucket whose
//          running count reaches K_c).  d_max comes from a coarse histogram
//          of e counted while sampling plus one pass for the low bits.
// Phase D  scan the remaining lists: per vector, estimated distance
//          e = sum_m LUT[m][code_m], bucket a = map[bin(e)], and Push
//          (Algorithm 1): append (e, id) and count it when a <= tau.  The
//          counts are kept per bin (a bucket is a union of consecutive bins,
//          so Update on them gives the same tau), and a <= tau is tested as
//          e <= the largest estimate whose bucket is <= tau.  Warps refresh
//          tau after every eighth chunk (the paper updates once per cluster;
//          tau only moves down, and a stale tau only admits extra objects,
//          never drops a needed one).
// The final selection (the last step of Algorithm 1's Collect) runs in k_select.cu.
//
// GPU mapping: one lane per vector; the lane's code row sits in registers
// (coalesced 512-byte chunk loads); each LUT read goes to bank (lane + slot)
// mod 32, so the 32 reads of a warp never conflict.  The region stores
// (estimated distance, list position); positions become ids in k_select.cu,
// so the hot loop never waits on an id load.  Appends are warp-
// aggregated (ballots + one shared atomic per warp and chunk) into a
// contiguous region.
#include <algorithm>
#include <climits>
#include <type_traits>

#include "bbc_internal.cuh"
#include "dev_util.cuh"
#include "select_body.cuh"

namespace bbc {

constexpr int SCAN_THREADS = 512;
// A warp runs Update after every kUpdateEvery-th chunk of its main scan (a
// power of two).  A staler tau only admits extra objects; fewer Updates
// leave more issue slots to the lookups.
constexpr int kUpdateEvery = 8;

template <int M, int BITS>
struct ScanCfg {
    static constexpr int K = 1 << BITS;
    // words per LUT row: >= M + 31 and a multiple of 32 (a power of two where that costs little)
    static constexpr int W = M <= 32 ? 64 : (M <= 96 ? 128 : M + 32);
    static constexpr int ROWB = W * 4;
    static constexpr int CB = M * BITS / 8;
    static constexpr int CBP = (CB + 15) / 16 * 16;
    static constexpr int NCH = CBP / 16;
    static constexpr int LUT_WORDS = K * W;
    // CTAs per SM the shared-memory table allows (the launch bound for registers)
    static constexpr int MIN_CTAS = K * W * 4 <= 100 * 1024 ? 2 : 1;
    // threads of the one-CTA-per-query kernel: a table too large for two
    // CTAs per SM gets 32 warps in one CTA
    static constexpr int THREADS = MIN_CTAS == 2 ? 512 : 1024;
    // 32-vector blocks per warp iteration (their code loads in flight together)
    static constexpr int CHUNK = NCH <= 2 ? 3 : (NCH <= 6 && THREADS == 512 ? 2 : 1);
    // the same for the pair form, which keeps two estimates per vector
    static constexpr int PCHUNK = NCH <= 2 ? 2 : 1;
    // estimates are below M * 65535 < 2^EB; the sample's coarse histogram
    // counts e >> SHC (2^11 bins), the fine one e mod 2^SHC
    static constexpr int EB = M <= 8 ? 19 : (M <= 16 ? 20 : (M <= 32 ? 21 : (M <= 64 ? 22 : 23)));
    static constexpr int SHC = EB - 11;
};

__device__ __forceinline__ uint32_t word_of(const uint4& v, int wi) {
    return wi == 0 ? v.x : (wi == 1 ? v.y : (wi == 2 ? v.z : v.w));
}

// Shared-memory byte address of the LUT entry for code slot S of this lane,
// without the slot's own offset 4 * S (added as the load's immediate):
// LUT base + code * ROWB + 4 * lane (lane4 = 4 * lane, base = LUT base,
// warp-uniform).  For 8-bit codes with 256-byte rows one byte permute yields
// code << 8 | 4 * lane directly.
template <int M, int BITS, int S>
__device__ __forceinline__ uint32_t slot_addr(const uint4 (&r)[ScanCfg<M, BITS>::NCH], uint32_t lane4, uint32_t base) {
    using C = ScanCfg<M, BITS>;
    if (BITS == 8) {
        const uint32_t w = word_of(r[S >> 4], (S >> 2) & 3);
        if (C::ROWB == 256) {
            // one byte permute yields code << 8 | 4 * lane (bytes 2, 3 of lane4 are zero)
            const uint32_t x = __byte_perm(w, lane4, 0x7604u | ((uint32_t)(S & 3) << 4));
            return x + base;
        }
        const uint32_t x = __byte_perm(w, 0u, 0x4404u | ((uint32_t)(S & 3) << 4));   // code << 8
        const uint32_t lane_base = base + lane4;
        if (C::ROWB == 512) return (x << 1) + lane_base;
        return (x >> 8) * (uint32_t)C::ROWB + lane_base;
    } else {
        const int byte = S >> 1;
        const uint32_t w = word_of(r[byte >> 4], (byte >> 2) & 3);
        const uint32_t code = (w >> (8 * (byte & 3) + 4 * (S & 1))) & 0xFu;
        return code * (uint32_t)C::ROWB + base + lane4;
    }
}

template <int OFF>
__device__ __forceinline__ uint32_t lds(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1+%2];" : "=r"(v) : "r"(addr), "n"(OFF));
    return v;
}

template <int M, int BITS, int S>
struct AdcUnroll {
    static __device__ __forceinline__ uint32_t run(const uint4 (&r)[ScanCfg<M, BITS>::NCH], uint32_t lane4,
                                                   uint32_t base) {
        // two lookups per step, summed with one three-input add
        const uint32_t v0 = lds<4 * S>(slot_addr<M, BITS, S>(r, lane4, base));
        const uint32_t v1 = lds<4 * (S + 1)>(slot_addr<M, BITS, S + 1>(r, lane4, base));
        return v0 + v1 + AdcUnroll<M, BITS, S + 2>::run(r, lane4, base);
    }
};
template <int M, int BITS>
struct AdcUnroll<M, BITS, M> {
    static __device__ __forceinline__ uint32_t run(const uint4 (&)[ScanCfg<M, BITS>::NCH], uint32_t, uint32_t) {
        return 0u;
    }
};

// Estimated distance of this lane's vector: sum over sub-spaces of its LUT entries.
template <int M, int BITS>
__device__ __forceinline__ uint32_t adc_lane(const uint4 (&r)[ScanCfg<M, BITS>::NCH], uint32_t lane4, uint32_t base) {
    return AdcUnroll<M, BITS, 0>::run(r, lane4, base);
}

// Packed table of the pair form: word (code j, column c) holds query a's
// entry LUT_a[c mod M][j] in its low and query b's LUT_b[c mod M][j] in its
// high 16 bits.  With A = the sum of a lane's words (mod 2^32) and B = the
// sum of their high halves, e_b = B and e_a = A - 2^16 B exactly: both true
// sums are below M * 65535 < 2^32.  B takes one two-way dot product per
// word (dp2a.lo with weights (0, 1): B + the word's high half); the scan is
// issue-bound, and this saves the separate shift per lookup.
template <int M, int BITS, int S>
struct AdcPairUnroll {
    static __device__ __forceinline__ void run(const uint4 (&r)[ScanCfg<M, BITS>::NCH], uint32_t lane4,
                                               uint32_t base, uint32_t& A, uint32_t& B) {
        const uint32_t v0 = lds<4 * S>(slot_addr<M, BITS, S>(r, lane4, base));
        const uint32_t v1 = lds<4 * (S + 1)>(slot_addr<M, BITS, S + 1>(r, lane4, base));
        A += v0 + v1;
        B = __dp2a_lo(v0, 0x100u, B);
        B = __dp2a_lo(v1, 0x100u, B);
        AdcPairUnroll<M, BITS, S + 2>::run(r, lane4, base, A, B);
    }
};
template <int M, int BITS>
struct AdcPairUnroll<M, BITS, M> {
    static __device__ __forceinline__ void run(const uint4 (&)[ScanCfg<M, BITS>::NCH], uint32_t, uint32_t,
                                               uint32_t&, uint32_t&) {}
};

// Estimated distances of this lane's vector for both queries of a packed table.
template <int M, int BITS>
__device__ __forceinline__ void adc_pair(const uint4 (&r)[ScanCfg<M, BITS>::NCH], uint32_t lane4, uint32_t base,
                                         uint32_t& ea, uint32_t& eb) {
    uint32_t A = 0u, B = 0u;
    AdcPairUnroll<M, BITS, 0>::run(r, lane4, base, A, B);
    eb = B;
    ea = A - (B << 16);
}

// Update on the shared bucket counts by one warp: first bucket whose running
// count reaches kc, or m.
__device__ __forceinline__ uint32_t warp_update(const uint32_t* hist, int m, int64_t kc) {
    const unsigned ln = lane_id();
    uint32_t h[8];
    uint32_t s = 0;
    // two 16-byte loads per lane where hist is 16-byte aligned (it is zero past m)
    uint32_t raw[8];
    if ((reinterpret_cast<uintptr_t>(hist) & 15u) == 0) {
        asm volatile("ld.volatile.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(raw[0]), "=r"(raw[1]), "=r"(raw[2]), "=r"(raw[3]) : "l"(hist + ln * 8));
        asm volatile("ld.volatile.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(raw[4]), "=r"(raw[5]), "=r"(raw[6]), "=r"(raw[7]) : "l"(hist + ln * 8 + 4));
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) raw[i] = *(volatile const uint32_t*)&hist[ln * 8 + i];
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        h[i] = (int)ln * 8 + i < m ? raw[i] : 0u;
        s += h[i];
    }
    unsigned long long inc = warp_incl_scan64(s);
    unsigned hit = __ballot_sync(0xFFFFFFFFu, inc >= (unsigned long long)kc);
    if (!hit) return (uint32_t)m;
    unsigned src = __ffs(hit) - 1;
    uint32_t bk = 0;
    if (ln == src) {
        unsigned long long c = inc - s;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            c += h[i];
            if (c >= (unsigned long long)kc) { bk = ln * 8 + i; break; }
        }
    }
    return __shfl_sync(0xFFFFFFFFu, bk, src);
}

// Update on bin counts by one warp.  Buckets are unions of consecutive bins
// (the map is monotone), so the first bin b whose running count reaches kc
// lies in the first bucket whose running count reaches kc: tau = map[b];
// m when the total is below kc.  bh is 16-byte aligned shared memory.
__device__ __forceinline__ uint32_t warp_update_bins(const uint32_t* bh, const uint8_t* bmap, int m, int64_t kc) {
    const unsigned ln = lane_id();
    uint32_t h[8];
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(bh + ln * 8);
    asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(h[0]), "=r"(h[1]), "=r"(h[2]), "=r"(h[3]) : "r"(sa));
    asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4+16];"
                 : "=r"(h[4]), "=r"(h[5]), "=r"(h[6]), "=r"(h[7]) : "r"(sa));
    const uint32_t k32 = kc >= 0xFFFFFFFFll ? 0xFFFFFFFFu : (kc < 0 ? 0u : (uint32_t)kc);
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += h[i];
    const uint32_t inc = warp_incl_scan(s);
    const unsigned hit = __ballot_sync(0xFFFFFFFFu, inc >= k32);
    if (!hit) return (uint32_t)m;
    const unsigned src = __ffs(hit) - 1;
    uint32_t b = 0;
    if (ln == src) {
        // smallest i with (count before this lane) + h[0] + ... + h[i] >= kc
        uint32_t run = inc - s;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            run += h[i];
            if (run >= k32) { b = (uint32_t)i; break; }
        }
        b += ln * 8;
    }
    b = __shfl_sync(0xFFFFFFFFu, b, src);
    return bmap[b];
}

__device__ __forceinline__ uint32_t bin_of(uint32_t e, uint32_t dmin, int sh) {
    if (e <= dmin) return 0u;
    uint32_t b = (e - dmin) >> sh;
    return b > 255u ? 255u : b;
}

struct ScanShared {
    alignas(16) uint32_t hist[kMaxBuckets];   // bucket counts (state in / out)
    alignas(16) uint32_t bh[256];             // counts of pushed objects per bin
    uint32_t ehist[256];
    alignas(16) uint8_t bmap[256];
    uint32_t sc[2];
    uint32_t count;
    uint32_t dmin, dmax;
    uint32_t tau;
    uint32_t etau;      // largest estimate whose bucket is <= tau (the map is monotone)
    uint32_t eearly;    // early re-rank: estimates below this are scored exactly in the scan
    int sh;
    int nsl;
    int gs;             // layout blocks of the sampled lists
    int gtot;           // layout blocks of all probed lists
    long long sq;
};

// Per-query view of the batch: this query's probe count, K_c and region.
struct QCtx {
    int P;
    int64_t kc;
    int64_t cap;
    uint2* region;
    const int32_t* lists;
    float* rdist;       // early re-rank: exact distance per region entry, or null
    const int32_t* lbase = nullptr;   // residual IVF-PQ: base of each list (indexed like lists)
    float inv = 0.f;                  // residual IVF-PQ: the table's scale
};

// Residual IVF-PQ: the object term w_o = rint(clamp(V_o * inv, +-2^28)) in
// the table's integer units (the per-list base is added with it).
__device__ __forceinline__ int32_t resid_w(float v, float inv) {
    float u = __fmul_rn(v, inv);
    u = fminf(fmaxf(u, -268435456.f), 268435456.f);
    return __float2int_rn(u);
}

// Early re-rank (Algorithm 4): ||q - v||^2 of the object in code-block slot
// `slot` from the slot-ordered u8 copy, in 32-bit integers (q8: the query's
// components as bytes; exact for integer data as the u8 re-rank).
__device__ __forceinline__ float early_dist(const DevIndex& ix, const uint4* q8, uint32_t qn2, uint32_t slot) {
    const int nc = ix.d >> 4;
    const uint4* row = reinterpret_cast<const uint4*>(ix.vec_lo + (size_t)slot * ix.d);
    uint32_t qv = 0;
    for (int c = 0; c < nc; ++c) {
        const uint4 v = __ldg(row + c);
        const uint4 qq = q8[c];
        qv = __dp4a(v.x, qq.x, qv); qv = __dp4a(v.y, qq.y, qv);
        qv = __dp4a(v.z, qq.z, qv); qv = __dp4a(v.w, qq.w, qv);
    }
    return __uint2float_rn(qn2 + __ldg(ix.vnorm2 + slot) - 2u * qv);
}

// Early threshold after the objects before layout block g of S_q scanned:
// tau_pred = the bucket of the ceil(f K_c)-th smallest estimate counted so
// far (f = 32 g / S_q), and objects with a bucket below it, i.e. with an
// estimate below the returned bound, are scored early.  Warp-collective.
template <typename SS>
__device__ __forceinline__ uint32_t early_bound(const SS& S, int m, int64_t kc, long long scanned) {
    const long long sq = S.sq > 0 ? S.sq : 1;
    if (scanned > sq) scanned = sq;
    long long r = (scanned * (long long)kc + sq - 1) / sq;
    if (r < 1) r = 1;
    const uint32_t tp = warp_update_bins(S.bh, S.bmap, m, r);
    if (tp == 0) return 0u;
    const uint32_t et = etau_of(S, tp - 1);
    return et == 0xFFFFFFFFu ? et : et + 1u;
}

// Push test without the map: buckets are monotone in the bin, so bucket(e) <= t
// holds exactly for bins 0 .. c-1, c = number of bins whose bucket is <= t,
// i.e. for e <= d_min + (c << sh) - 1.  Warp-collective.
__device__ __forceinline__ uint32_t etau_of(const ScanShared& S, uint32_t t) {
    const unsigned ln = lane_id();
    const uint2 w = *(const uint2*)&S.bmap[ln * 8];             // 8 map entries of this lane
    const uint32_t tt = t > 255u ? 0xFFFFFFFFu : t * 0x01010101u;
    // bytes <= t: per-byte unsigned compare (0xFF where true)
    uint32_t c = t > 255u ? 8u : (uint32_t)(__popc(__vcmpleu4(w.x, tt)) + __popc(__vcmpleu4(w.y, tt))) / 8u;
    c = __reduce_add_sync(0xFFFFFFFFu, c);
    if (c >= 256u) return 0xFFFFFFFFu;
    const unsigned long long v = (unsigned long long)S.dmin + ((unsigned long long)c << S.sh) - 1ull;
    return v > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)v;
}

// Split mode: move this CTA's per-bin count deltas into the query's global
// bucket counts, then Update on the global counts (one warp).
__device__ __forceinline__ void flush_and_update(ScanShared& S, bbc_collector_state* st, int m, int64_t kc) {
    for (int b = (int)lane_id(); b < 256; b += 32) {
        const uint32_t v = atomicExch(&S.bh[b], 0u);
        if (v) atomicAdd(&st->hist[S.bmap[b]], v);
    }
    __syncwarp();
    const uint32_t t = warp_update(st->hist, m, kc);
    const uint32_t e = etau_of(S, t);
    if (lane_id() == 0) {
        atomicMin(&st->tau, (int)t);
        atomicMin(&S.tau, t);
        atomicMin(&S.etau, e);
    }
}

// Bucket counts from the per-bin counts: hist[map[b]] += bh[b] (whole CTA;
// S.hist is overwritten).
__device__ void bins_to_buckets(ScanShared& S) {
    for (int i = threadIdx.x; i < kMaxBuckets; i += blockDim.x) S.hist[i] = 0u;
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += blockDim.x)
        if (S.bh[b]) atomicAdd(&S.hist[S.bmap[b]], S.bh[b]);
    __syncthreads();
}

// Load of list descriptor j from the descriptor array at shared address d0.
__device__ __forceinline__ int4 ld_desc(uint32_t d0, int j) {
    int4 v;
    asm volatile("ld.shared.v4.s32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(d0 + 16u * (uint32_t)j));
    return v;
}

// Warp-collective: lay out lists[0..nl) in probe order as consecutive
// 32-vector blocks.  ldesc[j] = {first layout block, end layout block,
// code block minus layout block, 32 * first layout block + list length}, so
// layout block g of list j is code block g + ldesc[j].z and its lane t holds
// a vector when 32 g + t < ldesc[j].w.  Returns the number of layout blocks;
// *nvec = the number of vectors.
__device__ int build_layout(const DevIndex& ix, const int32_t* lists, int nl, int4* ldesc, long long* nvec) {
    const unsigned ln = lane_id();
    int carry = 0;
    long long carryv = 0;
    for (int base = 0; base < nl; base += 32) {
        const int j = base + (int)ln;
        int nb = 0, nv = 0, blk = 0;
        if (j < nl) {
            const int l = lists[j];
            nv = ix.list_len[l];
            nb = (nv + 31) >> 5;
            blk = ix.list_blk[l];
        }
        const uint32_t inc = warp_incl_scan((uint32_t)nb);
        const unsigned long long incv = warp_incl_scan64((unsigned long long)nv);
        if (j < nl) {
            const int lo = carry + (int)inc - nb;
            ldesc[j] = make_int4(lo, lo + nb, blk - lo, 32 * lo + nv);
        }
        carry += (int)__shfl_sync(0xFFFFFFFFu, inc, 31);
        carryv += (long long)__shfl_sync(0xFFFFFFFFu, incv, 31);
    }
    *nvec = carryv;
    return carry;
}

// Phase A's table staging: the query's uint16 table [M][K] from global
// memory into the scan layout (row = code, word c = entry of sub-space
// c mod M).  A thread moves 8 consecutive codes of one sub-space (one 16-byte
// load); consecutive threads take consecutive sub-spaces, so each row store
// of a warp covers consecutive words.
template <int M, int BITS>
__device__ __forceinline__ void stage_lut(const uint16_t* lq, uint32_t* lut) {
    using C = ScanCfg<M, BITS>;
    constexpr int K8 = C::K / 8;
    for (int t = threadIdx.x; t < M * K8; t += blockDim.x) {
        const int j8 = t / M, c = t - j8 * M;
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(lq + c * C::K + j8 * 8));
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint32_t wd = word_of(v, i >> 1);
            const uint32_t val = (i & 1) ? (wd >> 16) : (wd & 0xFFFFu);
            uint32_t* row = lut + (j8 * 8 + i) * C::W;
#pragma unroll
            for (int cc = c; cc < C::W; cc += M) row[cc] = val;
        }
    }
}

// Scans blocks [g0, g1) of the lists laid out in ldesc (nl lists).
// MAIN = false: sampling (append everything); MAIN = true: Push with the
// codebook and tau.  GLOBAL = false: the CTA owns the query (counts and
// region cursor in shared memory); GLOBAL = true: several CTAs share the
// query (region cursor and counts in the global state, tau cached per CTA).
//
// Warps take chunks of CHUNK consecutive blocks in turn, so the CTA moves
// through the lists in probe order.  A warp keeps the descriptor of its
// current list in registers and walks forward (its chunks ascend); the
// appends of a chunk take one cursor atomic.
// HALF = -1: the table holds one query; HALF = 0 / 1: a packed pair table,
// of which this pass scores query a (low halves) or query b (high halves).
// EARLY (one CTA per query): Algorithm 4's early re-rank -- an appended
// object whose estimate is below S.eearly gets its exact distance now, from
// the slot-ordered u8 copy (q8: the query as bytes, null when it is not
// integer-valued), in Q.rdist; the other appended objects get -1 there.
// RES: residual IVF-PQ -- each estimate is the table sum plus the list's base
// (Q.lbase) and the object's term from V_o (ix.rv); the sampling pass then
// keeps no coarse histogram (the estimates are not bounded by M * 65535).
template <int M, int BITS, bool MAIN, bool GLOBAL, int HALF = -1, bool EARLY = false, bool RES = false>
__device__ __forceinline__ void scan_blocks(const DevIndex& ix, const ScanArgs& a, const QCtx& Q,
                                            bbc_collector_state* st, int nl, int g0, int g1,
                                            const uint32_t* lut, const int4* ldesc, ScanShared& S,
                                            uint32_t* cf = nullptr, const uint4* q8 = nullptr,
                                            uint32_t qn2 = 0) {
    using C = ScanCfg<M, BITS>;
    using Pos = typename std::conditional<GLOBAL, unsigned long long, uint32_t>::type;
    static_assert(!(EARLY && RES), "the early re-rank takes plain PQ codes");
    // the early re-rank's row loads need registers: two blocks per step there
    constexpr int CH = EARLY && C::CHUNK > 2 ? 2 : C::CHUNK;
    const unsigned ln = lane_id();
    const int nw = blockDim.x >> 5;
    const uint32_t lut_s = (uint32_t)__cvta_generic_to_shared(lut);   // warp-uniform
    const uint32_t lane4 = 4u * ln;
    uint2* region = Q.region;
    const unsigned lt_mask = (1u << ln) - 1u;
    const Pos cap = GLOBAL ? (Pos)Q.cap : (Pos)(Q.cap < 0xFFFFFFFFll ? Q.cap : 0xFFFFFFFFll);
    const uint4* codes = reinterpret_cast<const uint4*>(ix.codes) + ln;
    const uint32_t dmin = S.dmin;                             // fixed once the codebook exists
    const int sh = S.sh;
    // current list j of this warp (descriptor fields in registers)
    const uint32_t d0 = (uint32_t)__cvta_generic_to_shared(ldesc);
    int j = -1, jhi = 0, jb = 0, jend = 0;
    int32_t jbase = 0;                                        // RES: base of list j
    auto seek = [&](int g) {
        int4 d;
        if (j < 0) {
            int lo = 0, hi = nl - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (ld_desc(d0, mid).x <= g) lo = mid; else hi = mid - 1;
            }
            j = lo;
            d = ld_desc(d0, j);
        } else {
            do { d = ld_desc(d0, ++j); } while (g >= d.y);
        }
        jhi = d.y;
        jb = d.z;
        jend = d.w;
        if (RES) jbase = __ldg(Q.lbase + j);
    };
    int it = 0;
    uint32_t nearly = 0;                                      // EARLY: objects this lane scored
    for (int cb = g0 + (int)warp_id() * CH; cb < g1; cb += nw * CH, ++it) {
        const int nb = min(CH, g1 - cb);                      // blocks in this chunk (warp-uniform)
        int gbk[CH];
        uint32_t vbits = 0;                                   // bit u: this lane holds a vector of block u
        uint4 r[CH][C::NCH];
        int32_t radd[CH];                                     // RES: list base (then + the object's term)
        float rvv[CH];                                        // RES: V_o of this lane's object
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            gbk[u] = 0;
            radd[u] = 0;
            rvv[u] = 0.f;
            if (u < nb) {
                const int g = cb + u;
                if (g >= jhi) seek(g);
                gbk[u] = jb + g;
                vbits |= (uint32_t)((int)ln < jend - 32 * g) << u;
                const uint4* cp = codes + (size_t)gbk[u] * (32 * C::NCH);
#pragma unroll
                for (int c = 0; c < C::NCH; ++c) r[u][c] = __ldg(cp + c * 32);
                if (RES) {
                    radd[u] = jbase;
                    rvv[u] = __ldg(ix.rv + (size_t)gbk[u] * 32u + ln);
                }
            }
        }
        const uint32_t etau = MAIN ? *(volatile uint32_t*)&S.etau : 0u;
        const uint32_t eearly = (EARLY && MAIN && q8) ? *(volatile uint32_t*)&S.eearly : 0u;
        uint32_t e[CH];
        unsigned bal[CH];
        uint32_t tot = 0;
        uint32_t mn = 0xFFFFFFFFu;
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            e[u] = 0;
            bal[u] = 0;
            if (u < nb) {
                if (HALF < 0) {
                    e[u] = adc_lane<M, BITS>(r[u], lane4, lut_s);
                } else {
                    uint32_t ea, eb;
                    adc_pair<M, BITS>(r[u], lane4, lut_s, ea, eb);
                    e[u] = HALF ? eb : ea;
                }
                if (RES) e[u] += (uint32_t)(radd[u] + resid_w(rvv[u], Q.inv));
                const bool valid = (vbits >> u) & 1u;
                const bool push = MAIN ? (valid && e[u] <= etau) : valid;    // bucket(e) <= tau
                bal[u] = __ballot_sync(0xFFFFFFFFu, push);
                tot += (uint32_t)__popc(bal[u]);
                if (!MAIN && valid) mn = min(mn, e[u]);
            }
        }
        if (!MAIN && !GLOBAL) {
            mn = __reduce_min_sync(0xFFFFFFFFu, mn);
            if (ln == 0 && mn != 0xFFFFFFFFu) atomicMin(&S.dmin, mn);
        }
        uint32_t epos[CH];                                    // EARLY: region slot of each appended object
        uint32_t ebits = 0;                                   // EARLY: bit u: block u's object is scored now
#pragma unroll
        for (int u = 0; u < CH; ++u) epos[u] = 0xFFFFFFFFu;
        if (tot) {
            Pos base = 0;
            if (ln == 0) {
                if (GLOBAL)
                    base = (Pos)atomicAdd(reinterpret_cast<unsigned long long*>(&st->pushed),
                                          (unsigned long long)tot);
                else
                    base = (Pos)atomicAdd(&S.count, tot);
            }
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                if ((bal[u] >> ln) & 1u) {
                    const Pos pos = base + (Pos)__popc(bal[u] & lt_mask);
                    if (pos < cap) {
                        region[pos] = make_uint2(e[u], (uint32_t)gbk[u] * 32u + ln);
                        if constexpr (EARLY) {
                            epos[u] = (uint32_t)pos;
                            if (e[u] < eearly) ebits |= 1u << u;
                        }
                    } else {
                        atomicOr(ix.status, kStatusRegionOverrun);
                    }
                    if (MAIN) atomicAdd(&S.bh[bin_of(e[u], dmin, sh)], 1u);
                    else if (!GLOBAL && !RES) atomicAdd(&cf[e[u] >> C::SHC], 1u);   // coarse histogram of the sample
                }
                base += (Pos)__popc(bal[u]);
            }
        }
        if (EARLY) {
            // Algorithm 4: the appended objects below the predicted threshold get their exact distance
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                if (epos[u] != 0xFFFFFFFFu) {
                    float rd = -1.f;
                    if ((ebits >> u) & 1u) {
                        rd = early_dist(ix, q8, qn2, (uint32_t)gbk[u] * 32u + ln);
                        ++nearly;
                    }
                    Q.rdist[epos[u]] = rd;
                }
            }
        }
        if (MAIN && (it & (kUpdateEvery - 1)) == 0) {
            if (GLOBAL) {
                if (warp_id() == 0) flush_and_update(S, st, a.m, Q.kc);
            } else {
                const uint32_t t = warp_update_bins(S.bh, S.bmap, a.m, Q.kc);
                const uint32_t et = etau_of(S, t);
                if (ln == 0) {
                    atomicMin(&S.tau, t);
                    atomicMin(&S.etau, et);
                }
                if (EARLY && q8) {
                    // tau_pred from the fraction of S_q scanned through this chunk
                    const uint32_t ee = early_bound(S, a.m, Q.kc, 32ll * (cb + CH));
                    if (ln == 0) S.eearly = ee;
                }
            }
        }
    }
    if (EARLY && a.early_totals) {
        const uint32_t w = __reduce_add_sync(0xFFFFFFFFu, nearly);
        if (ln == 0 && w) atomicAdd(&a.early_totals[0], (unsigned long long)w);
    }
}

// CTA-wide: the bin holding rank r (0-based) of the counts h[0..nb), nb <=
// 8 * blockDim.x: res[0] = that bin, res[1] = r minus the count of the bins
// before it.  Requires sum(h) > r.  wsum: 32 words of shared scratch.
__device__ void cta_rank_bin(const uint32_t* h, int nb, uint32_t r, uint32_t* wsum, uint32_t* res) {
    const int tid = threadIdx.x, bs = blockDim.x;
    const int per = (nb + bs - 1) / bs;
    uint32_t loc[8], tot = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int b = tid * per + j;
        loc[j] = (j < per && b < nb) ? h[b] : 0u;
        tot += loc[j];
    }
    const uint32_t winc = warp_incl_scan(tot);
    if (lane_id() == 31) wsum[warp_id()] = winc;
    __syncthreads();
    if (warp_id() == 0) {
        const int nw = bs >> 5;
        const uint32_t v = (int)lane_id() < nw ? wsum[lane_id()] : 0u;
        const uint32_t x = warp_incl_scan(v) - v;
        if ((int)lane_id() < nw) wsum[lane_id()] = x;
    }
    __syncthreads();
    uint32_t c = wsum[warp_id()] + winc - tot;
    if (c <= r && r < c + tot) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (j < per && r < c + loc[j]) {
                res[0] = (uint32_t)(tid * per + j);
                res[1] = r - c;
                break;
            }
            c += loc[j];
        }
    }
    __syncthreads();
}

// Phase C of Algorithm 1's Collect (Section 3.2, "Codebook Generation Based
// on Estimated Distance") over the ns sampled objects at the start of the
// region, by the whole CTA, given d_max (the t-th smallest sampled estimate,
// t = min(K_c, ns)).  On entry S.dmin holds the smallest sampled estimate and
// S.bh is zero; on exit S holds d_max, the shift, the equal-depth map, the
// sample's counts per bin and tau.  One pass over the sample counts both the
// bins of the objects at or below d_max (for the map) and the bins of all of
// them (the counts Update works on).
__device__ void codebook_from_dmax(const uint2* region, int64_t ns, int64_t kc, int m, uint32_t dmax,
                                   ScanShared& S) {
    const int tid = threadIdx.x, bs = blockDim.x;
    if (tid == 0) {
        S.dmax = dmax;
        int sh = 0;
        while (((dmax - S.dmin) >> sh) > 255u) ++sh;
        S.sh = sh;
    }
    for (int i = tid; i < 256; i += bs) S.ehist[i] = 0;
    __syncthreads();
    const uint32_t dmin = S.dmin;
    const int sh = S.sh;
    for (int64_t i = tid; i < ns; i += 4 * bs) {
        uint32_t e[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) e[u] = i + u * bs < ns ? region[i + u * bs].x : 0xFFFFFFFFu;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (i + u * bs < ns) {
                const uint32_t b = bin_of(e[u], dmin, sh);
                atomicAdd(&S.bh[b], 1u);
                if (e[u] <= dmax) atomicAdd(&S.ehist[b], 1u);
            }
        }
    }
    __syncthreads();
    if (warp_id() == 0) {
        const unsigned ln = lane_id();
        uint32_t h[8], s = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) { h[i] = S.ehist[ln * 8 + i]; s += h[i]; }
        const unsigned long long inc = warp_incl_scan64(s);
        const unsigned long long T = __shfl_sync(0xFFFFFFFFu, inc, 31);
        unsigned long long cum = inc - s;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            unsigned long long v = T ? ((unsigned long long)m * cum) / T : 0ull;
            S.bmap[ln * 8 + i] = (uint8_t)(v > (unsigned long long)(m - 1) ? m - 1 : v);
            cum += h[i];
        }
    }
    __syncthreads();
    if (warp_id() == 0) {
        const uint32_t t0 = warp_update_bins(S.bh, S.bmap, m, kc);
        const uint32_t e0 = etau_of(S, t0);
        if (lane_id() == 0) { S.tau = t0; S.etau = e0; }
    }
    __syncthreads();
}

// Codebook when the sampling pass counted e >> shc into cf[0..2048): d_max
// from that coarse histogram and one pass for the low shc bits.  cf (at least
// max(2048, 2^shc) words) is overwritten.
__device__ void build_codebook_hist(const uint2* region, int64_t ns, int64_t kc, int m, ScanShared& S,
                                    uint32_t* cf, int shc) {
    const int tid = threadIdx.x, bs = blockDim.x;
    if (ns <= 0) {
        if (tid == 0) { S.dmin = 0; S.dmax = 0; S.sh = 0; S.tau = (uint32_t)m; S.etau = 0xFFFFFFFFu; }
        for (int i = tid; i < 256; i += bs) S.bmap[i] = 0;
        __syncthreads();
        return;
    }
    const int64_t t = ns < kc ? ns : kc;
    __shared__ uint32_t wsum[32];
    cta_rank_bin(cf, 2048, (uint32_t)(t - 1), wsum, S.sc);
    const uint32_t hi = S.sc[0], r1 = S.sc[1];
    const int nf = 1 << shc;
    for (int i = tid; i < nf; i += bs) cf[i] = 0u;
    __syncthreads();
    for (int64_t i = tid; i < ns; i += 4 * bs) {
        uint32_t e[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) e[u] = i + u * bs < ns ? region[i + u * bs].x : 0xFFFFFFFFu;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (i + u * bs < ns && (e[u] >> shc) == hi) atomicAdd(&cf[e[u] & (uint32_t)(nf - 1)], 1u);
    }
    __syncthreads();
    cta_rank_bin(cf, nf, r1, wsum, S.sc);
    codebook_from_dmax(region, ns, kc, m, (hi << shc) | S.sc[0], S);
}

// Codebook when d_max is found by a radix select over the sample (no
// histogram gathered while sampling).  wide: the estimates may use all 32
// bits (residual IVF-PQ); otherwise they are below M * 65535 < 2^24.
__device__ void build_codebook(const uint2* region, int64_t ns, int64_t kc, int m, ScanShared& S,
                               bool wide = false) {
    const int tid = threadIdx.x, bs = blockDim.x;
    if (ns > 0) {
        const int64_t t = ns < kc ? ns : kc;
        const uint32_t dmax = cta_select_u32(ns, (uint32_t)(t - 1), [&](int64_t i) { return region[i].x; },
                                             S.ehist, S.sc, wide ? 24 : 16);
        codebook_from_dmax(region, ns, kc, m, dmax, S);
        return;
    } else {
        if (tid == 0) { S.dmin = 0; S.dmax = 0; S.sh = 0; S.tau = (uint32_t)m; S.etau = 0xFFFFFFFFu; }
        for (int i = tid; i < 256; i += bs) S.bmap[i] = 0;
    }
    __syncthreads();
}

// Largest dimension of the early re-rank's in-register query bytes.
constexpr int kEarlyMaxD = 256;

template <int M, int BITS, bool EARLY = false, bool RES = false>
__global__ void __launch_bounds__(ScanCfg<M, BITS>::THREADS, ScanCfg<M, BITS>::MIN_CTAS) scan_kernel(DevIndex ix, ScanArgs a) {
    using C = ScanCfg<M, BITS>;
    extern __shared__ uint4 dsm[];
    uint32_t* lut = reinterpret_cast<uint32_t*>(dsm);
    int4* ldesc = reinterpret_cast<int4*>(lut + C::LUT_WORDS);         // [nprobe]
    __shared__ ScanShared S;
    __shared__ uint32_t cf[2048 > (1 << C::SHC) ? 2048 : (1 << C::SHC)];   // sample histograms
    __shared__ uint4 sq8[EARLY ? kEarlyMaxD / 16 : 1];                   // EARLY: the query as bytes
    __shared__ uint32_t s_qn2;
    __shared__ int s_intq;
    const int64_t qi = blockIdx.x;
    const QCtx Q{a.qp.P(qi), a.qp.KC(qi), a.qp.rcap(qi), a.region + a.qp.roff(qi), a.lists + a.qp.poff(qi),
                 EARLY ? a.rdist + a.qp.roff(qi) : nullptr, RES ? a.lbase + a.qp.poff(qi) : nullptr,
                 RES ? a.qinv[qi] : 0.f};
    const int P = Q.P;
    const int tid = threadIdx.x, bs = blockDim.x;

    // ---- Phase A: LUT staging and list layout ----
    stage_lut<M, BITS>(a.lut16 + qi * (int64_t)M * C::K, lut);
    if (EARLY) {
        // the query's components as bytes when they are all integers in [0, 255]
        if (tid == 0) { s_qn2 = 0u; s_intq = 1; S.eearly = 0u; }
        __syncthreads();
        uint8_t* qb = reinterpret_cast<uint8_t*>(sq8);
        for (int i = tid; i < ix.d; i += bs) {
            const float v = a.q[qi * ix.d + i];
            const bool ok = v >= 0.f && v <= 255.f && v == floorf(v);
            if (!ok) s_intq = 0;
            qb[i] = ok ? (uint8_t)v : 0;
            if (ok) atomicAdd(&s_qn2, (uint32_t)v * (uint32_t)v);
        }
    }
    for (int i = tid; i < 256; i += bs) S.bh[i] = 0;
    for (int i = tid; i < 2048; i += bs) cf[i] = 0;
    if (tid == 0) {
        S.count = 0;
        S.dmin = 0xFFFFFFFFu;
        S.tau = (uint32_t)a.m;
        S.etau = 0xFFFFFFFFu;
        S.sh = 0;
    }
    if (warp_id() == 0) {
        const unsigned ln = lane_id();
        long long carryv;
        const int gtot = build_layout(ix, Q.lists, P, ldesc, &carryv);
        __syncwarp();
        // sample lists: at least min(sample_min, P), extended until min(K_c, S_q) vectors
        const long long want = Q.kc < carryv ? Q.kc : carryv;
        const int smin = a.sample_min < P ? a.sample_min : P;
        long long cum = 0;
        int nsl = P;
        for (int base = 0; base < P; base += 32) {
            const int j = base + (int)ln;
            int nv = 0;
            if (j < P) {
                const int4 d = ldesc[j];
                nv = d.w - 32 * d.x;
            }
            const unsigned long long incv = warp_incl_scan64((unsigned long long)nv);
            const bool ok = j < P && (j + 1) >= smin && (long long)(cum + (long long)incv) >= want;
            const unsigned hit = __ballot_sync(0xFFFFFFFFu, ok);
            if (hit) { nsl = base + (int)(__ffs(hit) - 1) + 1; break; }
            cum += (long long)__shfl_sync(0xFFFFFFFFu, incv, 31);
        }
        if (ln == 0) {
            S.nsl = nsl;
            S.sq = carryv;
            S.gs = nsl > 0 ? ldesc[nsl - 1].y : 0;
            S.gtot = gtot;
        }
    }
    __syncthreads();

    // ---- Phase B: sample ----
    const int gs = S.gs;
    const uint4* q8 = (EARLY && s_intq) ? sq8 : nullptr;
    scan_blocks<M, BITS, false, false, -1, EARLY, RES>(ix, a, Q, a.state + qi, P, 0, gs, lut, ldesc, S, cf, q8,
                                                        s_qn2);
    __syncthreads();

    // ---- Phase C: codebook ----
    const int64_t ns = (int64_t)min((long long)S.count, (long long)Q.cap);
    if (RES) build_codebook(Q.region, ns, Q.kc, a.m, S, true);
    else build_codebook_hist(Q.region, ns, Q.kc, a.m, S, cf, C::SHC);
    if (EARLY && q8) {
        // Algorithm 4: the first predicted threshold from the sample's share of S_q
        if (warp_id() == 0) {
            const uint32_t ee = early_bound(S, a.m, Q.kc, (long long)ns);
            if (lane_id() == 0) S.eearly = ee;
        }
        __syncthreads();
    }
    if (a.sample_only) {
        // the sampled objects are appended and the codebook built: the state
        // as the list-grouped scan (k_scan_tc.cu) takes it over
        bbc_collector_state* st = a.state + qi;
        bins_to_buckets(S);
        for (int i = tid; i < kMaxBuckets; i += bs) st->hist[i] = i < a.m ? S.hist[i] : 0u;
        for (int i = tid; i < 256; i += bs) st->map[i] = S.bmap[i];
        if (tid == 0) {
            st->d_min = S.dmin;
            st->d_max = S.dmax;
            st->sh = S.sh;
            st->m = a.m;
            st->sample_lists = S.nsl;
            st->tau = (int32_t)S.tau;
            st->sample_size = ns;
            st->scanned = S.sq;
            st->pushed = (int64_t)S.count;
            st->below = 0;
            st->kc = Q.kc;
        }
        return;
    }
    // ---- Phase D: main scan ----
    scan_blocks<M, BITS, true, false, -1, EARLY, RES>(ix, a, Q, a.state + qi, P, gs, S.gtot, lut, ldesc, S, nullptr,
                                                       q8, s_qn2);
    __syncthreads();

    // ---- state out ----
    bbc_collector_state* st = a.state + qi;
    bins_to_buckets(S);
    for (int i = tid; i < kMaxBuckets; i += bs) st->hist[i] = i < a.m ? S.hist[i] : 0u;
    for (int i = tid; i < 256; i += bs) st->map[i] = S.bmap[i];
    if (warp_id() == 0) {
        const uint32_t t1 = warp_update_bins(S.bh, S.bmap, a.m, Q.kc);
        if (lane_id() == 0) {
            st->d_min = S.dmin;
            st->d_max = S.dmax;
            st->sh = S.sh;
            st->m = a.m;
            st->sample_lists = S.nsl;
            st->tau = (int32_t)t1;
            st->sample_size = ns;
            st->scanned = S.sq;
            st->pushed = (int64_t)S.count;
            st->below = 0;
            st->kc = Q.kc;
        }
    }
    // ---- S7 in the tail: the query's region is still in L2; the table's
    // shared memory (dead now) holds the threshold bucket's keys ----
    if (a.fuse_select) {
        __syncthreads();
        select_query(ix, a.sel, qi, reinterpret_cast<unsigned long long*>(dsm), a.sel.tcap);
    }
}

// ---------------------------------------------------------------------------
// Split form: several CTAs per query.  Work items (query q, part g) come from
// a device counter (persistent CTAs); part g of G covers a contiguous range
// of the query's lists.  Used when a batch has too few queries to fill the
// GPU with one CTA per query.
//   pass 1 (MAIN = false): the sampled lists, every object appended;
//   codebook_kernel: the codebook, counts and tau from the sampled objects;
//   pass 2 (MAIN = true): the remaining lists with Push against tau.
// ---------------------------------------------------------------------------

// Warp 0: sampled list count (as in the fused kernel) and S_q of a query.
__device__ void sample_plan(const DevIndex& ix, const QCtx& Q, int sample_min, int* nsl_out, long long* sq_out) {
    const unsigned ln = lane_id();
    const int P = Q.P;
    long long tot = 0;
    for (int base = 0; base < P; base += 32) {
        const int j = base + (int)ln;
        const unsigned long long inc = warp_incl_scan64(j < P ? (unsigned long long)ix.list_len[Q.lists[j]] : 0ull);
        tot += (long long)__shfl_sync(0xFFFFFFFFu, inc, 31);
    }
    const long long want = Q.kc < tot ? Q.kc : tot;
    const int smin = sample_min < P ? sample_min : P;
    long long cum = 0;
    int nsl = P;
    for (int base = 0; base < P; base += 32) {
        const int j = base + (int)ln;
        const unsigned long long inc = warp_incl_scan64(j < P ? (unsigned long long)ix.list_len[Q.lists[j]] : 0ull);
        const bool ok = j < P && (j + 1) >= smin && (long long)(cum + (long long)inc) >= want;
        const unsigned hit = __ballot_sync(0xFFFFFFFFu, ok);
        if (hit) { nsl = base + (int)(__ffs(hit) - 1) + 1; break; }
        cum += (long long)__shfl_sync(0xFFFFFFFFu, inc, 31);
    }
    *nsl_out = nsl;
    *sq_out = tot;
}

struct SplitArgs {
    int G;                    // parts per query
    unsigned int* counter;    // work counter, zero before the launch
};

template <int M, int BITS, bool MAIN, bool RES = false>
__global__ void __launch_bounds__(SCAN_THREADS, ScanCfg<M, BITS>::MIN_CTAS) scan_split_kernel(DevIndex ix, ScanArgs a, SplitArgs sp, int64_t nq) {
    using C = ScanCfg<M, BITS>;
    extern __shared__ uint4 dsm[];
    uint32_t* lut = reinterpret_cast<uint32_t*>(dsm);
    int4* ldesc = reinterpret_cast<int4*>(lut + C::LUT_WORDS);
    __shared__ ScanShared S;
    __shared__ long long s_item, s_q;
    __shared__ int s_nsl;
    const int tid = threadIdx.x, bs = blockDim.x;
    const long long total = nq * (long long)sp.G;
    if (tid == 0) s_q = -1;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = (long long)atomicAdd(sp.counter, 1u);
        __syncthreads();
        const long long item = s_item;
        if (item >= total) break;
        const int64_t qi = item / sp.G;
        const int g = (int)(item % sp.G);
        const QCtx Q{a.qp.P(qi), a.qp.KC(qi), a.qp.rcap(qi), a.region + a.qp.roff(qi), a.lists + a.qp.poff(qi)};
        bbc_collector_state* st = a.state + qi;
        const int P = Q.P;
        if (MAIN) {
            if (tid == 0) s_nsl = st->sample_lists;
        } else if (warp_id() == 0) {
            int nsl;
            long long sq;
            sample_plan(ix, Q, a.sample_min, &nsl, &sq);
            if (lane_id() == 0) {
                s_nsl = nsl;
                if (g == 0) { st->sample_lists = nsl; st->scanned = sq; }
            }
        }
        __syncthreads();
        const int nsl = s_nsl;
        int j0, j1;
        if (MAIN) {
            const int per = (P - nsl + sp.G - 1) / sp.G;
            j0 = nsl + g * per;
            j1 = min(P, j0 + per);
        } else {
            const int per = (nsl + sp.G - 1) / sp.G;
            j0 = g * per;
            j1 = min(nsl, j0 + per);
        }
        if (j0 >= j1) continue;
        const int nl = j1 - j0;
        if (s_q != qi) stage_lut<M, BITS>(a.lut16 + qi * (int64_t)M * C::K, lut);
        if (warp_id() == 0) {
            long long nv;
            const int nb = build_layout(ix, Q.lists + j0, nl, ldesc, &nv);
            if (lane_id() == 0) S.gtot = nb;
        }
        if (MAIN) {
            for (int i = tid; i < 256; i += bs) {
                S.bmap[i] = st->map[i];
                S.bh[i] = 0u;                                    // this CTA's count deltas per bin
            }
            if (tid == 0) {
                S.dmin = st->d_min;
                S.sh = st->sh;
                S.tau = (uint32_t)*(volatile int*)&st->tau;
            }
            __syncthreads();
            if (warp_id() == 0) {
                const uint32_t e0 = etau_of(S, S.tau);
                if (lane_id() == 0) S.etau = e0;
            }
        }
        __syncthreads();
        if (tid == 0) s_q = qi;
        if (RES) {
            // this part's lists start at probe rank j0
            QCtx Qr = Q;
            Qr.lbase = a.lbase + a.qp.poff(qi) + j0;
            Qr.inv = a.qinv[qi];
            scan_blocks<M, BITS, MAIN, true, -1, false, true>(ix, a, Qr, st, nl, 0, S.gtot, lut, ldesc, S);
        } else {
            scan_blocks<M, BITS, MAIN, true>(ix, a, Q, st, nl, 0, S.gtot, lut, ldesc, S);
        }
        __syncthreads();
        if (MAIN && warp_id() == 0) flush_and_update(S, st, a.m, Q.kc);
    }
}

// Per query: smallest sampled estimate, then the codebook of the sample.
__global__ void __launch_bounds__(SCAN_THREADS) codebook_kernel(ScanArgs a) {
    __shared__ ScanShared S;
    const int64_t qi = blockIdx.x;
    bbc_collector_state* st = a.state + qi;
    const int64_t cap = a.qp.rcap(qi);
    const int64_t kc = a.qp.KC(qi);
    const uint2* region = a.region + a.qp.roff(qi);
    const int64_t ns = st->pushed < cap ? st->pushed : cap;
    const int tid = threadIdx.x, bs = blockDim.x;
    if (tid == 0) S.dmin = 0xFFFFFFFFu;
    for (int i = tid; i < 256; i += bs) S.bh[i] = 0u;
    __syncthreads();
    uint32_t mn = 0xFFFFFFFFu;
    for (int64_t i = tid; i < ns; i += bs) mn = min(mn, region[i].x);
    mn = __reduce_min_sync(0xFFFFFFFFu, mn);
    if (lane_id() == 0 && mn != 0xFFFFFFFFu) atomicMin(&S.dmin, mn);
    __syncthreads();
    build_codebook(region, ns, kc, a.m, S, a.lbase != nullptr);
    bins_to_buckets(S);
    for (int i = tid; i < kMaxBuckets; i += bs) st->hist[i] = i < a.m ? S.hist[i] : 0u;
    for (int i = tid; i < 256; i += bs) st->map[i] = S.bmap[i];
    if (tid == 0) {
        st->d_min = S.dmin;
        st->d_max = S.dmax;
        st->sh = S.sh;
        st->m = a.m;
        st->tau = (int32_t)S.tau;
        st->sample_size = ns;
        st->below = 0;
        st->kc = kc;
    }
}

// ---------------------------------------------------------------------------
// Pair form of the batched scan: one CTA owns two queries whose probe sets
// overlap (paired by the plan in k_pair.cu).  Their uint16 tables share one
// shared-memory table (query a in the low, query b in the high half of each
// word), so a code row is loaded once for both and one shared load serves
// both queries' lookups of a vector.  Each query keeps its own sample,
// codebook, bin counts, threshold and region; the main pass streams the
// union of the two queries' remaining lists, each list tagged with the
// queries that scan it there.  Candidate sets, thresholds and the counts of
// buckets up to the threshold are those of the one-CTA-per-query form.
// ---------------------------------------------------------------------------

// Phase A's table staging for a pair (lb null: no second query, high halves 0).
template <int M, int BITS>
__device__ __forceinline__ void stage_lut_pair(const uint16_t* la, const uint16_t* lb, uint32_t* lut) {
    using C = ScanCfg<M, BITS>;
    constexpr int K8 = C::K / 8;
    for (int t = threadIdx.x; t < M * K8; t += blockDim.x) {
        const int j8 = t / M, c = t - j8 * M;
        const uint4 va = __ldg(reinterpret_cast<const uint4*>(la + c * C::K + j8 * 8));
        const uint4 vb = lb ? __ldg(reinterpret_cast<const uint4*>(lb + c * C::K + j8 * 8)) : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint32_t wa = word_of(va, i >> 1), wb = word_of(vb, i >> 1);
            const uint32_t val = (i & 1) ? ((wa >> 16) | (wb & 0xFFFF0000u)) : ((wa & 0xFFFFu) | (wb << 16));
            uint32_t* row = lut + (j8 * 8 + i) * C::W;
#pragma unroll
            for (int cc = c; cc < C::W; cc += M) row[cc] = val;
        }
    }
}

// Warp 0: the union of the two queries' main lists (probe ranks at or after
// their sampled lists) laid out as consecutive 32-vector blocks, with the
// descriptors of build_layout and lfl[j] = bit 0: query a scans list j here,
// bit 1: query b does.  Ranks go in steps of 16 (lanes 0-15 query a, 16-31
// query b), so the union keeps both probe orders, nearest first.  A list of
// query b that is also one of a's main lists is laid out once, from a's side
// (bm: the main-list bitmaps of a and b, nlw words each).  Returns the
// number of blocks; *nlists = the number of lists.
__device__ int build_union_layout(const DevIndex& ix, const QCtx (&Q)[2], const int (&nsl)[2], bool hb,
                                  const uint32_t* bm, int nlw, int4* ldesc, uint8_t* lfl, int* nlists) {
    const unsigned ln = lane_id();
    const int h = (int)(ln >> 4), r0 = (int)(ln & 15u);
    const unsigned lt_mask = (1u << ln) - 1u;
    const int pmax = max(Q[0].P, hb ? Q[1].P : 0);
    // this lane's query, selected without indexing Q by a run-time value
    const int Ph = h ? Q[1].P : Q[0].P;
    const int32_t* lh = h ? Q[1].lists : Q[0].lists;
    const int nslh = h ? nsl[1] : nsl[0];
    int carry = 0, cnt = 0;
    for (int base = 0; base < pmax; base += 16) {
        const int r = base + r0;
        bool take = false;
        int nb = 0, nv = 0, blk = 0;
        uint32_t fl = 0;
        if ((h == 0 || hb) && r >= nslh && r < Ph) {
            const int l = lh[r];
            const bool in0 = (bm[l >> 5] >> (l & 31)) & 1u;
            const bool in1 = (bm[nlw + (l >> 5)] >> (l & 31)) & 1u;
            take = h == 0 || !in0;
            fl = h == 0 ? (1u | (in1 ? 2u : 0u)) : 2u;
            if (take) {
                nv = ix.list_len[l];
                nb = (nv + 31) >> 5;
                blk = ix.list_blk[l];
            }
        }
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, take);
        const uint32_t inc = warp_incl_scan((uint32_t)nb);
        if (take) {
            const int pos = cnt + __popc(bal & lt_mask);
            const int lo = carry + (int)inc - nb;
            ldesc[pos] = make_int4(lo, lo + nb, blk - lo, 32 * lo + nv);
            lfl[pos] = (uint8_t)fl;
        }
        cnt += __popc(bal);
        carry += (int)__shfl_sync(0xFFFFFFFFu, inc, 31);
    }
    *nlists = cnt;
    return carry;
}

// Appends the pushed objects of one query for a chunk (see scan_blocks).
template <int CH>
__device__ __forceinline__ void pair_append(const DevIndex& ix, ScanShared& S, uint2* region, uint32_t cap,
                                            const uint32_t (&e)[CH], const unsigned (&bal)[CH], const int (&gbk)[CH],
                                            uint32_t tot, uint32_t dmin, int sh) {
    const unsigned ln = lane_id();
    const unsigned lt_mask = (1u << ln) - 1u;
    uint32_t base = 0;
    if (ln == 0) base = atomicAdd(&S.count, tot);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
#pragma unroll
    for (int u = 0; u < CH; ++u) {
        if ((bal[u] >> ln) & 1u) {
            const uint32_t pos = base + (uint32_t)__popc(bal[u] & lt_mask);
            if (pos < cap) region[pos] = make_uint2(e[u], (uint32_t)gbk[u] * 32u + ln);
            else atomicOr(ix.status, kStatusRegionOverrun);
            atomicAdd(&S.bh[bin_of(e[u], dmin, sh)], 1u);
        }
        base += (uint32_t)__popc(bal[u]);
    }
}

// Main pass of the pair form over blocks [0, g1) of the union layout.
template <int M, int BITS>
__device__ __forceinline__ void scan_pair_main(const DevIndex& ix, const ScanArgs& a, const QCtx (&Q)[2], bool hb,
                                               int nl, int g1, const uint32_t* lut, const int4* ldesc,
                                               const uint8_t* lfl, ScanShared (&S)[2]) {
    using C = ScanCfg<M, BITS>;
    constexpr int CH = C::PCHUNK;
    const unsigned ln = lane_id();
    const int nw = blockDim.x >> 5;
    const uint32_t lut_s = (uint32_t)__cvta_generic_to_shared(lut);
    const uint32_t lane4 = 4u * ln;
    const uint32_t cap0 = (uint32_t)(Q[0].cap < 0xFFFFFFFFll ? Q[0].cap : 0xFFFFFFFFll);
    const uint32_t cap1 = (uint32_t)(Q[1].cap < 0xFFFFFFFFll ? Q[1].cap : 0xFFFFFFFFll);
    const uint4* codes = reinterpret_cast<const uint4*>(ix.codes) + ln;
    const uint32_t dmin0 = S[0].dmin, dmin1 = S[1].dmin;
    const int sh0 = S[0].sh, sh1 = S[1].sh;
    const uint32_t d0 = (uint32_t)__cvta_generic_to_shared(ldesc);
    int j = -1, jhi = 0, jb = 0, jend = 0;
    uint32_t jfl = 0;
    auto seek = [&](int g) {
        int4 d;
        if (j < 0) {
            int lo = 0, hi = nl - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (ld_desc(d0, mid).x <= g) lo = mid; else hi = mid - 1;
            }
            j = lo;
            d = ld_desc(d0, j);
        } else {
            do { d = ld_desc(d0, ++j); } while (g >= d.y);
        }
        jhi = d.y;
        jb = d.z;
        jend = d.w;
        jfl = lfl[j];
    };
    int it = 0;
    for (int cb = (int)warp_id() * CH; cb < g1; cb += nw * CH, ++it) {
        const int nb = min(CH, g1 - cb);
        int gbk[CH];
        uint32_t v0 = 0, v1 = 0;                        // bit u: block u's lane holds a vector query a / b scans
        uint4 r[CH][C::NCH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            gbk[u] = 0;
            if (u < nb) {
                const int g = cb + u;
                if (g >= jhi) seek(g);
                gbk[u] = jb + g;
                const uint32_t has = (uint32_t)((int)ln < jend - 32 * g);
                v0 |= (has & jfl) << u;
                v1 |= (has & (jfl >> 1)) << u;
                const uint4* cp = codes + (size_t)gbk[u] * (32 * C::NCH);
#pragma unroll
                for (int c = 0; c < C::NCH; ++c) r[u][c] = __ldg(cp + c * 32);
            }
        }
        const uint32_t et0 = *(volatile uint32_t*)&S[0].etau;
        const uint32_t et1 = *(volatile uint32_t*)&S[1].etau;
        uint32_t e0[CH], e1[CH];
        unsigned b0[CH], b1[CH];
        uint32_t t0 = 0, t1 = 0;
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            e0[u] = 0; e1[u] = 0; b0[u] = 0; b1[u] = 0;
            if (u < nb) {
                adc_pair<M, BITS>(r[u], lane4, lut_s, e0[u], e1[u]);
                b0[u] = __ballot_sync(0xFFFFFFFFu, ((v0 >> u) & 1u) && e0[u] <= et0);
                b1[u] = __ballot_sync(0xFFFFFFFFu, ((v1 >> u) & 1u) && e1[u] <= et1);
                t0 += (uint32_t)__popc(b0[u]);
                t1 += (uint32_t)__popc(b1[u]);
            }
        }
        if (t0) pair_append<CH>(ix, S[0], Q[0].region, cap0, e0, b0, gbk, t0, dmin0, sh0);
        if (t1) pair_append<CH>(ix, S[1], Q[1].region, cap1, e1, b1, gbk, t1, dmin1, sh1);
        if ((it & (kUpdateEvery - 1)) == 0) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (h == 1 && !hb) break;
                const uint32_t t = warp_update_bins(S[h].bh, S[h].bmap, a.m, Q[h].kc);
                const uint32_t et = etau_of(S[h], t);
                if (ln == 0) {
                    atomicMin(&S[h].tau, t);
                    atomicMin(&S[h].etau, et);
                }
            }
        }
    }
}

// Bytes of dynamic shared memory of the pair form: the table, 2 nprobe list
// descriptors and flags, and the two main-list bitmaps.
__host__ __device__ inline size_t pair_smem_bytes(int lut_words, int nprobe, int nlist) {
    const size_t fl = ((size_t)2 * nprobe + 15) / 16 * 16;
    return (size_t)lut_words * 4 + (size_t)2 * nprobe * 16 + fl + (size_t)2 * ((nlist + 31) / 32) * 4;
}

template <int M, int BITS>
__global__ void __launch_bounds__(SCAN_THREADS, ScanCfg<M, BITS>::MIN_CTAS)
scan_pair_kernel(DevIndex ix, ScanArgs a, const int32_t* __restrict__ perm, int64_t nq) {
    using C = ScanCfg<M, BITS>;
    extern __shared__ uint4 dsm[];
    uint32_t* lut = reinterpret_cast<uint32_t*>(dsm);
    int4* ldesc = reinterpret_cast<int4*>(lut + C::LUT_WORDS);                       // [2 nprobe]
    uint8_t* lfl = reinterpret_cast<uint8_t*>(ldesc + 2 * a.nprobe);                  // [2 nprobe]
    const int nlw = (ix.nlist + 31) / 32;
    uint32_t* bm = reinterpret_cast<uint32_t*>(lfl + ((2 * a.nprobe + 15) / 16) * 16);  // [2][nlw]
    __shared__ ScanShared S[2];
    __shared__ uint32_t cf[2048 > (1 << C::SHC) ? 2048 : (1 << C::SHC)];
    __shared__ int s_nsl[2], s_gu, s_nu;
    __shared__ long long s_ns[2];
    const int tid = threadIdx.x, bs = blockDim.x;
    const bool hb = 2 * (int64_t)blockIdx.x + 1 < nq;
    const int64_t qid[2] = {perm[2 * (int64_t)blockIdx.x], hb ? perm[2 * (int64_t)blockIdx.x + 1] : perm[2 * (int64_t)blockIdx.x]};
    QCtx Q[2];
#pragma unroll
    for (int h = 0; h < 2; ++h)
        Q[h] = QCtx{a.qp.P(qid[h]), a.qp.KC(qid[h]), a.qp.rcap(qid[h]), a.region + a.qp.roff(qid[h]),
                    a.lists + a.qp.poff(qid[h])};

    // ---- Phase A: the packed table, per-query state ----
    stage_lut_pair<M, BITS>(a.lut16 + qid[0] * (int64_t)M * C::K, hb ? a.lut16 + qid[1] * (int64_t)M * C::K : nullptr,
                            lut);
    for (int i = tid; i < 2 * nlw; i += bs) bm[i] = 0u;
    for (int i = tid; i < 256; i += bs) { S[0].bh[i] = 0u; S[1].bh[i] = 0u; }
    if (tid < 2) {
        S[tid].count = 0;
        S[tid].dmin = 0xFFFFFFFFu;
        S[tid].tau = (uint32_t)a.m;
        S[tid].etau = 0xFFFFFFFFu;
        S[tid].sh = 0;
    }
    // ---- Phases B and C per query: sample of its nearest lists, codebook ----
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (h == 1 && !hb) break;
        for (int i = tid; i < (int)(sizeof(cf) / 4); i += bs) cf[i] = 0u;
        __syncthreads();
        if (warp_id() == 0) {
            const unsigned ln = lane_id();
            long long carryv;
            const int P = Q[h].P;
            const int gtot = build_layout(ix, Q[h].lists, P, ldesc, &carryv);
            __syncwarp();
            const long long want = Q[h].kc < carryv ? Q[h].kc : carryv;
            const int smin = a.sample_min < P ? a.sample_min : P;
            long long cum = 0;
            int nsl = P;
            for (int base = 0; base < P; base += 32) {
                const int j = base + (int)ln;
                int nv = 0;
                if (j < P) {
                    const int4 d = ldesc[j];
                    nv = d.w - 32 * d.x;
                }
                const unsigned long long incv = warp_incl_scan64((unsigned long long)nv);
                const bool ok = j < P && (j + 1) >= smin && (long long)(cum + (long long)incv) >= want;
                const unsigned hit = __ballot_sync(0xFFFFFFFFu, ok);
                if (hit) { nsl = base + (int)(__ffs(hit) - 1) + 1; break; }
                cum += (long long)__shfl_sync(0xFFFFFFFFu, incv, 31);
            }
            if (ln == 0) {
                S[h].nsl = nsl;
                S[h].sq = carryv;
                S[h].gs = nsl > 0 ? ldesc[nsl - 1].y : 0;
                S[h].gtot = gtot;
                s_nsl[h] = nsl;
            }
        }
        __syncthreads();
        if (h == 0)
            scan_blocks<M, BITS, false, false, 0>(ix, a, Q[0], a.state + qid[0], Q[0].P, 0, S[0].gs, lut, ldesc, S[0], cf);
        else
            scan_blocks<M, BITS, false, false, 1>(ix, a, Q[1], a.state + qid[1], Q[1].P, 0, S[1].gs, lut, ldesc, S[1], cf);
        __syncthreads();
        const int64_t ns = (int64_t)min((long long)S[h].count, (long long)Q[h].cap);
        if (tid == 0) s_ns[h] = ns;
        build_codebook_hist(Q[h].region, ns, Q[h].kc, a.m, S[h], cf, C::SHC);
    }
    // ---- Phase D: the union of the main lists, both queries per lookup ----
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (h == 1 && !hb) break;
        for (int j = s_nsl[h] + tid; j < Q[h].P; j += bs) {
            const int l = Q[h].lists[j];
            atomicOr(&bm[h * nlw + (l >> 5)], 1u << (l & 31));
        }
    }
    __syncthreads();
    if (warp_id() == 0) {
        int nu;
        const int gu = build_union_layout(ix, Q, s_nsl, hb, bm, nlw, ldesc, lfl, &nu);
        if (lane_id() == 0) { s_gu = gu; s_nu = nu; }
    }
    __syncthreads();
    if (s_nu > 0) scan_pair_main<M, BITS>(ix, a, Q, hb, s_nu, s_gu, lut, ldesc, lfl, S);
    __syncthreads();

    // ---- state out ----
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (h == 1 && !hb) break;
        bbc_collector_state* st = a.state + qid[h];
        bins_to_buckets(S[h]);
        for (int i = tid; i < kMaxBuckets; i += bs) st->hist[i] = i < a.m ? S[h].hist[i] : 0u;
        for (int i = tid; i < 256; i += bs) st->map[i] = S[h].bmap[i];
        if (warp_id() == 0) {
            const uint32_t t1 = warp_update_bins(S[h].bh, S[h].bmap, a.m, Q[h].kc);
            if (lane_id() == 0) {
                st->d_min = S[h].dmin;
                st->d_max = S[h].dmax;
                st->sh = S[h].sh;
                st->m = a.m;
                st->sample_lists = S[h].nsl;
                st->tau = (int32_t)t1;
                st->sample_size = s_ns[h];
                st->scanned = S[h].sq;
                st->pushed = (int64_t)S[h].count;
                st->below = 0;
                st->kc = Q[h].kc;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Baseline collectors (the comparison of Section 4, Exp-3: a binary heap and
// a lazily updated linear buffer in place of the bucket-based result buffer),
// one CTA per query, lists in probe order.  Both return the same candidate
// set as the result buffer -- the K_c smallest (estimated distance, id) of
// the scanned objects -- and exist to measure what the collector costs.
//   LAZY (mode 1): objects with e <= the current threshold are appended to a
//     linear buffer; after each list, when the buffer holds more than K_c,
//     the K_c-th smallest buffered e becomes the threshold (a CTA radix
//     select) and the buffer is compacted to the objects at or below it.
//   HEAP (mode 2): a binary max-heap of the K_c smallest (e, id) keys in
//     shared memory; per list, the warps stage the objects that can enter
//     (heap not full, or e <= the top's e) and one thread inserts them in
//     order (replace-top and sift-down once full).
// ---------------------------------------------------------------------------

__device__ __forceinline__ void heap_sift_down(unsigned long long* h, uint32_t n, uint32_t i) {
    const unsigned long long x = h[i];
    for (;;) {
        uint32_t c = 2 * i + 1;
        if (c >= n) break;
        if (c + 1 < n && h[c + 1] > h[c]) ++c;
        if (h[c] <= x) break;
        h[i] = h[c];
        i = c;
    }
    h[i] = x;
}

__device__ __forceinline__ void heap_sift_up(unsigned long long* h, uint32_t i) {
    const unsigned long long x = h[i];
    while (i > 0) {
        const uint32_t p = (i - 1) / 2;
        if (h[p] >= x) break;
        h[i] = h[p];
        i = p;
    }
    h[i] = x;
}

template <int M, int BITS, int MODE>
__global__ void __launch_bounds__(SCAN_THREADS, 1)
scan_collect_kernel(DevIndex ix, ScanArgs a, uint32_t stage_cap) {
    using C = ScanCfg<M, BITS>;
    extern __shared__ uint4 dsm[];
    uint32_t* lut = reinterpret_cast<uint32_t*>(dsm);
    int4* ldesc = reinterpret_cast<int4*>(lut + C::LUT_WORDS);                         // [nprobe]
    unsigned long long* heap = reinterpret_cast<unsigned long long*>(ldesc + a.nprobe); // MODE 2: [K_c]
    unsigned long long* stage = heap + (MODE == 2 ? a.kc : 0);                          // MODE 2: [stage_cap]
    __shared__ uint32_t hist[256], sc[2];
    __shared__ uint32_t s_count, s_stage, s_keep, s_heapn, s_over;
    __shared__ uint32_t s_thr;                 // LAZY: buffer threshold on e
    __shared__ unsigned long long s_top;      // HEAP: current largest key (max when not full)
    __shared__ long long s_sq;
    __shared__ int s_gtot;
    const int64_t qi = blockIdx.x;
    const QCtx Q{a.qp.P(qi), a.qp.KC(qi), a.qp.rcap(qi), a.region + a.qp.roff(qi), a.lists + a.qp.poff(qi)};
    const int tid = threadIdx.x, bs = blockDim.x, nw = bs >> 5;
    const unsigned ln = lane_id(), lt_mask = (1u << ln) - 1u;
    const uint32_t cap = (uint32_t)(Q.cap < 0xFFFFFFFFll ? Q.cap : 0xFFFFFFFFll);
    stage_lut<M, BITS>(a.lut16 + qi * (int64_t)M * C::K, lut);
    if (tid == 0) { s_count = 0; s_stage = 0; s_heapn = 0; s_over = 0; s_thr = 0xFFFFFFFFu; s_top = ~0ull; }
    if (warp_id() == 0) {
        long long nv;
        const int g = build_layout(ix, Q.lists, Q.P, ldesc, &nv);
        if (ln == 0) { s_gtot = g; s_sq = nv; }
    }
    __syncthreads();
    const uint32_t lut_s = (uint32_t)__cvta_generic_to_shared(lut);
    const uint4* codes = reinterpret_cast<const uint4*>(ix.codes) + ln;
    const uint32_t kc32 = (uint32_t)min(Q.kc, (int64_t)0xFFFFFFFF);
    for (int j = 0; j < Q.P; ++j) {
        const int4 dj = ldesc[j];
        const uint32_t thr = s_thr;
        const unsigned long long top = s_top;
        for (int g = dj.x + (int)warp_id(); g < dj.y; g += nw) {
            const int gb = dj.z + g;
            uint4 r[C::NCH];
            const uint4* cp = codes + (size_t)gb * (32 * C::NCH);
#pragma unroll
            for (int c = 0; c < C::NCH; ++c) r[c] = __ldg(cp + c * 32);
            const uint32_t e = adc_lane<M, BITS>(r, 4u * ln, lut_s);
            const bool valid = (int)ln < dj.w - 32 * g;
            const uint32_t pos = (uint32_t)gb * 32u + ln;
            if (MODE == 1) {
                const bool push = valid && e <= thr;
                const unsigned bal = __ballot_sync(0xFFFFFFFFu, push);
                if (bal) {
                    uint32_t base = 0;
                    if (ln == 0) base = atomicAdd(&s_count, (uint32_t)__popc(bal));
                    base = __shfl_sync(0xFFFFFFFFu, base, 0) + (uint32_t)__popc(bal & lt_mask);
                    if (push) {
                        if (base < cap) Q.region[base] = make_uint2(e, pos);
                        else atomicOr(ix.status, kStatusRegionOverrun);
                    }
                }
            } else {
                const bool push = valid && e <= (uint32_t)(top >> 32);
                const unsigned bal = __ballot_sync(0xFFFFFFFFu, push);
                if (bal) {
                    uint32_t base = 0;
                    if (ln == 0) base = atomicAdd(&s_stage, (uint32_t)__popc(bal));
                    base = __shfl_sync(0xFFFFFFFFu, base, 0) + (uint32_t)__popc(bal & lt_mask);
                    if (push) {
                        if (base < stage_cap) stage[base] = ((unsigned long long)e << 32) | ix.ids[pos];
                        else s_over = 1;
                    }
                }
            }
        }
        __syncthreads();
        if (MODE == 1) {
            const uint32_t n = min(s_count, cap);
            if (n > kc32) {
                // threshold = the K_c-th smallest buffered e; keep e <= threshold
                const uint32_t t = cta_select_u32(n, kc32 - 1, [&](int64_t i) { return Q.region[i].x; }, hist, sc, 24);
                if (tid == 0) { s_keep = 0; s_thr = t; }
                __syncthreads();
                for (uint32_t i0 = 0; i0 < n; i0 += (uint32_t)bs) {
                    const uint32_t i = i0 + (uint32_t)tid;
                    const uint2 v = i < n ? Q.region[i] : make_uint2(0xFFFFFFFFu, 0u);
                    const bool keep = i < n && v.x <= t;
                    __syncthreads();                            // every read of this tile before any write
                    const unsigned bal = __ballot_sync(0xFFFFFFFFu, keep);
                    uint32_t base = 0;
                    if (ln == 0 && bal) base = atomicAdd(&s_keep, (uint32_t)__popc(bal));
                    base = __shfl_sync(0xFFFFFFFFu, base, 0) + (uint32_t)__popc(bal & lt_mask);
                    if (keep) Q.region[base] = v;               // base <= i: the tile's own or earlier slots
                    __syncthreads();
                }
                if (tid == 0) s_count = s_keep;
                __syncthreads();
            }
        } else {
            if (tid == 0) {
                const uint32_t ns = min(s_stage, stage_cap);
                uint32_t hn = s_heapn;
                for (uint32_t i = 0; i < ns; ++i) {
                    const unsigned long long key = stage[i];
                    if (hn < kc32) {
                        heap[hn] = key;
                        heap_sift_up(heap, hn);
                        ++hn;
                    } else if (key < heap[0]) {
                        heap[0] = key;
                        heap_sift_down(heap, hn, 0);
                    }
                }
                s_heapn = hn;
                s_top = hn < kc32 ? ~0ull : heap[0];
                s_stage = 0;
            }
            __syncthreads();
        }
    }
    // ---- the K_c candidates ----
    uint32_t* cand = a.sel.cand + a.qp.coff(qi);
    bbc_collector_state* st = a.state + qi;
    if (MODE == 1) {
        const uint32_t n = min(s_count, cap);
        const uint32_t want = min(n, kc32);
        unsigned long long kth = ~0ull;
        if (want > 0 && want < n)
            kth = cta_select_u64(n, want - 1, [&](int64_t i) {
                const uint2 v = Q.region[i];
                return ((unsigned long long)v.x << 32) | ix.ids[v.y];
            }, hist, sc, 56);
        if (tid == 0) s_keep = 0;
        __syncthreads();
        for (uint32_t i0 = 0; i0 < n; i0 += (uint32_t)bs) {
            const uint32_t i = i0 + (uint32_t)tid;
            uint32_t id = 0;
            bool take = false;
            if (i < n) {
                const uint2 v = Q.region[i];
                id = ix.ids[v.y];
                take = (((unsigned long long)v.x << 32) | id) <= kth;
            }
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, take);
            uint32_t base = 0;
            if (ln == 0 && bal) base = atomicAdd(&s_keep, (uint32_t)__popc(bal));
            base = __shfl_sync(0xFFFFFFFFu, base, 0) + (uint32_t)__popc(bal & lt_mask);
            if (take && base < kc32) cand[base] = id;
        }
        __syncthreads();
        if (tid == 0) a.sel.cand_count[qi] = min(s_keep, kc32);
    } else {
        const uint32_t hn = s_heapn;
        for (uint32_t i = tid; i < hn; i += bs) cand[i] = (uint32_t)(heap[i] & 0xFFFFFFFFull);
        if (tid == 0) {
            a.sel.cand_count[qi] = hn;
            if (s_over) atomicOr(ix.status, kStatusRegionOverrun);
        }
    }
    for (int i = tid; i < kMaxBuckets; i += bs) st->hist[i] = 0u;
    for (int i = tid; i < 256; i += bs) st->map[i] = 0u;
    if (tid == 0) {
        st->d_min = 0; st->d_max = 0; st->sh = 0; st->m = 0; st->sample_lists = 0; st->tau = -1;
        st->sample_size = 0; st->scanned = s_sq; st->pushed = MODE == 1 ? (int64_t)s_count : (int64_t)s_heapn;
        st->below = 0; st->kc = Q.kc;
    }
}

// Largest dynamic shared memory a kernel can take next to its static shared
// memory (227 KB per block in all).
template <typename F>
static int max_dyn_smem(F kernel) {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return 0;
    return 227 * 1024 - (int)fa.sharedSizeBytes;
}

template <int M, int BITS>
static cudaError_t launch_split_t(const DevIndex& ix, int64_t nq, const ScanArgs& a, int G, unsigned int* counters,
                                  cudaStream_t st) {
    using C = ScanCfg<M, BITS>;
    const size_t smem = (size_t)C::LUT_WORDS * 4 + (size_t)a.nprobe * sizeof(int4);
    // a property of the compiled kernels (the same on every device); thread-safe initialisation
    static const int lim = std::min(std::min(max_dyn_smem(scan_split_kernel<M, BITS, false>),
                                             max_dyn_smem(scan_split_kernel<M, BITS, true>)),
                                    std::min(max_dyn_smem(scan_split_kernel<M, BITS, false, true>),
                                             max_dyn_smem(scan_split_kernel<M, BITS, true, true>)));
    cudaError_t e;
    if (ix.resid) {
        e = smem_attr_once((const void*)scan_split_kernel<M, BITS, false, true>, lim);
        if (e == cudaSuccess) e = smem_attr_once((const void*)scan_split_kernel<M, BITS, true, true>, lim);
    } else {
        e = smem_attr_once((const void*)scan_split_kernel<M, BITS, false>, lim);
        if (e == cudaSuccess) e = smem_attr_once((const void*)scan_split_kernel<M, BITS, true>, lim);
    }
    if (e != cudaSuccess) return e;
    if (smem > (size_t)lim) return cudaErrorInvalidValue;
    const long long items = nq * (long long)G;
    const unsigned grid = (unsigned)std::min<long long>(items, (long long)ix.num_sms * C::MIN_CTAS);
    e = cudaMemsetAsync(counters, 0, 2 * sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    if (ix.resid) {
        if (!a.lbase || !a.qinv) return cudaErrorInvalidValue;
        scan_split_kernel<M, BITS, false, true><<<grid, SCAN_THREADS, smem, st>>>(ix, a, SplitArgs{G, counters}, nq);
    } else {
        scan_split_kernel<M, BITS, false><<<grid, SCAN_THREADS, smem, st>>>(ix, a, SplitArgs{G, counters}, nq);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    codebook_kernel<<<(unsigned)nq, SCAN_THREADS, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ix.resid)
        scan_split_kernel<M, BITS, true, true><<<grid, SCAN_THREADS, smem, st>>>(ix, a, SplitArgs{G, counters + 1}, nq);
    else
        scan_split_kernel<M, BITS, true><<<grid, SCAN_THREADS, smem, st>>>(ix, a, SplitArgs{G, counters + 1}, nq);
    return cudaGetLastError();
}

// Threshold-bucket keys the fused selection holds in shared memory at least.
constexpr size_t kFusedSelectKeys = 8192;

template <int M, int BITS>
static cudaError_t launch_scan_t(const DevIndex& ix, int64_t nq, const ScanArgs& a0, cudaStream_t st) {
    using C = ScanCfg<M, BITS>;
    ScanArgs a = a0;
    size_t smem = (size_t)C::LUT_WORDS * 4 + (size_t)a.nprobe * sizeof(int4);
    if (a.fuse_select) {
        smem = std::max(smem, kFusedSelectKeys * 8);
        a.sel.tcap = (uint32_t)(smem / 8);
    }
    if (a.early && ix.resid) return cudaErrorInvalidValue;    // the early re-rank takes plain PQ codes
    if (a.early) {
        // Algorithm 4's early re-rank: tables of up to 64 KB (8-bit, M <= 32; 4-bit, M <= 64), d <= 256
        if constexpr (C::LUT_WORDS * 4 <= 64 * 1024 && M <= 64) {
            if (ix.d > kEarlyMaxD || ix.d % 16 || !ix.vec_lo || !a.rdist || !a.q) return cudaErrorInvalidValue;
            static const int lim_e = max_dyn_smem(scan_kernel<M, BITS, true>);
            cudaError_t e = smem_attr_once((const void*)scan_kernel<M, BITS, true>, lim_e);
            if (e != cudaSuccess) return e;
            if (smem > (size_t)lim_e) return cudaErrorInvalidValue;
            scan_kernel<M, BITS, true><<<(unsigned)nq, C::THREADS, smem, st>>>(ix, a);
            return cudaGetLastError();
        } else {
            return cudaErrorInvalidValue;
        }
    }
    if (ix.resid) {
        // residual IVF-PQ: the table sum plus the per-list base and the per-object term
        if (!a.lbase || !a.qinv || !ix.rv) return cudaErrorInvalidValue;
        static const int lim_r = max_dyn_smem(scan_kernel<M, BITS, false, true>);
        cudaError_t e = smem_attr_once((const void*)scan_kernel<M, BITS, false, true>, lim_r);
        if (e != cudaSuccess) return e;
        if (smem > (size_t)lim_r) return cudaErrorInvalidValue;
        scan_kernel<M, BITS, false, true><<<(unsigned)nq, C::THREADS, smem, st>>>(ix, a);
        return cudaGetLastError();
    }
    static const int lim = max_dyn_smem(scan_kernel<M, BITS>);   // a property of the compiled kernel
    cudaError_t e = smem_attr_once((const void*)scan_kernel<M, BITS>, lim);
    if (e != cudaSuccess) return e;
    if (smem > (size_t)lim) return cudaErrorInvalidValue;
    scan_kernel<M, BITS><<<(unsigned)nq, C::THREADS, smem, st>>>(ix, a);
    return cudaGetLastError();
}

template <int M, int BITS>
static cudaError_t launch_pair_t(const DevIndex& ix, int64_t nq, const ScanArgs& a, const int32_t* perm,
                                 cudaStream_t st) {
    using C = ScanCfg<M, BITS>;
    const size_t smem = pair_smem_bytes(C::LUT_WORDS, a.nprobe, ix.nlist);
    static const int lim = max_dyn_smem(scan_pair_kernel<M, BITS>);   // a property of the compiled kernel
    cudaError_t e = smem_attr_once((const void*)scan_pair_kernel<M, BITS>, lim);
    if (e != cudaSuccess) return e;
    if (smem > (size_t)lim) return cudaErrorInvalidValue;
    scan_pair_kernel<M, BITS><<<(unsigned)((nq + 1) / 2), SCAN_THREADS, smem, st>>>(ix, a, perm, nq);
    return cudaGetLastError();
}

// The pair form runs for tables that allow two 512-thread CTAs per SM, and
// only when its shared memory (table, list descriptors, bitmaps) still does.
bool scan_pair_supported(const DevIndex& ix, int nprobe) {
    if (ix.resid) return false;            // the pair form takes plain PQ codes
    int lut_words = 0;
    if (ix.bits == 8 && (ix.M == 8 || ix.M == 16 || ix.M == 32)) lut_words = 256 * 64;
    else if (ix.bits == 4 && (ix.M == 32 || ix.M == 64)) lut_words = 16 * (ix.M <= 32 ? 64 : 128);
    else return false;
    return pair_smem_bytes(lut_words, nprobe, ix.nlist) + 24 * 1024 <= 110 * 1024;
}

cudaError_t launch_scan_pair(const DevIndex& ix, int64_t nq, const ScanArgs& a, const int32_t* perm,
                             cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    if (!scan_pair_supported(ix, a.nprobe)) return cudaErrorInvalidValue;
    if (ix.bits == 8) {
        switch (ix.M) {
            case 8: return launch_pair_t<8, 8>(ix, nq, a, perm, st);
            case 16: return launch_pair_t<16, 8>(ix, nq, a, perm, st);
            case 32: return launch_pair_t<32, 8>(ix, nq, a, perm, st);
        }
    } else if (ix.bits == 4) {
        switch (ix.M) {
            case 32: return launch_pair_t<32, 4>(ix, nq, a, perm, st);
            case 64: return launch_pair_t<64, 4>(ix, nq, a, perm, st);
        }
    }
    return cudaErrorInvalidValue;
}

template <int M, int BITS, int MODE>
static size_t collect_smem(int nprobe, int64_t kc, uint32_t stage_cap) {
    using C = ScanCfg<M, BITS>;
    size_t smem = (size_t)C::LUT_WORDS * 4 + (size_t)nprobe * sizeof(int4);
    if (MODE == 2) smem += ((size_t)kc + stage_cap) * 8;
    return smem;
}

template <int M, int BITS, int MODE>
static cudaError_t launch_collect_t(const DevIndex& ix, int64_t nq, const ScanArgs& a, uint32_t stage_cap,
                                    cudaStream_t st) {
    const size_t smem = collect_smem<M, BITS, MODE>(a.nprobe, a.kc, stage_cap);
    static const int lim = max_dyn_smem(scan_collect_kernel<M, BITS, MODE>);   // a property of the compiled kernel
    cudaError_t e = smem_attr_once((const void*)scan_collect_kernel<M, BITS, MODE>, lim);
    if (e != cudaSuccess) return e;
    if (smem > (size_t)lim) return cudaErrorInvalidValue;
    scan_collect_kernel<M, BITS, MODE><<<(unsigned)nq, SCAN_THREADS, smem, st>>>(ix, a, stage_cap);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_collect_m(const DevIndex& ix, int64_t nq, const ScanArgs& a, uint32_t stage_cap,
                                    cudaStream_t st) {
    if (ix.bits == 8) {
        switch (ix.M) {
            case 8: return launch_collect_t<8, 8, MODE>(ix, nq, a, stage_cap, st);
            case 16: return launch_collect_t<16, 8, MODE>(ix, nq, a, stage_cap, st);
            case 32: return launch_collect_t<32, 8, MODE>(ix, nq, a, stage_cap, st);
        }
    } else if (ix.bits == 4) {
        switch (ix.M) {
            case 32: return launch_collect_t<32, 4, MODE>(ix, nq, a, stage_cap, st);
            case 64: return launch_collect_t<64, 4, MODE>(ix, nq, a, stage_cap, st);
        }
    }
    return cudaErrorInvalidValue;
}

bool scan_collect_supported(const DevIndex& ix, int mode, int nprobe, int64_t kc, uint32_t stage_cap) {
    if (mode != 1 && mode != 2) return false;
    if (ix.resid) return false;            // the baseline collectors take plain PQ codes
    int lut_words = 0;
    if (ix.bits == 8 && (ix.M == 8 || ix.M == 16 || ix.M == 32)) lut_words = 256 * 64;
    else if (ix.bits == 4 && (ix.M == 32 || ix.M == 64)) lut_words = 16 * (ix.M <= 32 ? 64 : 128);
    else return false;
    size_t smem = (size_t)lut_words * 4 + (size_t)nprobe * 16;
    if (mode == 2) smem += ((size_t)kc + stage_cap) * 8;
    return smem + 8 * 1024 <= 227 * 1024;
}

cudaError_t launch_scan_collect(const DevIndex& ix, int64_t nq, const ScanArgs& a, int mode, uint32_t stage_cap,
                                cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    if (!scan_collect_supported(ix, mode, a.nprobe, a.kc, stage_cap)) return cudaErrorInvalidValue;
    return mode == 1 ? launch_collect_m<1>(ix, nq, a, stage_cap, st) : launch_collect_m<2>(ix, nq, a, stage_cap, st);
}

bool scan_supported(int M, int bits) {
    if (bits == 8) return M == 8 || M == 16 || M == 32 || M == 64 || M == 96 || M == 128;
    if (bits == 4) return M == 32 || M == 64 || M == 128;
    return false;
}

cudaError_t launch_scan_split(const DevIndex& ix, int64_t nq, const ScanArgs& a, int G, unsigned int* counters,
                              cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    if (ix.bits == 8) {
        switch (ix.M) {
            case 8: return launch_split_t<8, 8>(ix, nq, a, G, counters, st);
            case 16: return launch_split_t<16, 8>(ix, nq, a, G, counters, st);
            case 32: return launch_split_t<32, 8>(ix, nq, a, G, counters, st);
            case 64: return launch_split_t<64, 8>(ix, nq, a, G, counters, st);
            case 96: return launch_split_t<96, 8>(ix, nq, a, G, counters, st);
            case 128: return launch_split_t<128, 8>(ix, nq, a, G, counters, st);
        }
    } else if (ix.bits == 4) {
        switch (ix.M) {
            case 32: return launch_split_t<32, 4>(ix, nq, a, G, counters, st);
            case 64: return launch_split_t<64, 4>(ix, nq, a, G, counters, st);
            case 128: return launch_split_t<128, 4>(ix, nq, a, G, counters, st);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_scan(const DevIndex& ix, int64_t nq, const ScanArgs& a, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    if (ix.bits == 8) {
        switch (ix.M) {
            case 8: return launch_scan_t<8, 8>(ix, nq, a, st);
            case 16: return launch_scan_t<16, 8>(ix, nq, a, st);
            case 32: return launch_scan_t<32, 8>(ix, nq, a, st);
            case 64: return launch_scan_t<64, 8>(ix, nq, a, st);
            case 96: return launch_scan_t<96, 8>(ix, nq, a, st);
            case 128: return launch_scan_t<128, 8>(ix, nq, a, st);
        }
    } else if (ix.bits == 4) {
        switch (ix.M) {
            case 32: return launch_scan_t<32, 4>(ix, nq, a, st);
            case 64: return launch_scan_t<64, 4>(ix, nq, a, st);
            case 128: return launch_scan_t<128, 4>(ix, nq, a, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace bbc
