// The final collection of one query (the last step of Algorithm 1's
// Collect), by the whole CTA: shared by the standalone selection kernel
// (k_select.cu) and the scan kernel's tail (k_scan.cu), which runs it while
// the query's region is still in L2.
//
// The bucket counts of the appended objects give the exact threshold bucket
// tau* = first bucket whose running count reaches K_c (Update on the final
// buffer).  Every object whose bucket is below tau* is a candidate (buckets
// are ordered by distance range, so they all precede the K_c-th); the
// remaining s = K_c - below candidates are the s smallest (e, id) of bucket
// tau*, found by a radix select on the 64-bit key (e << 32 | id).  When fewer
// than K_c objects were scanned, all of them are candidates.
//
// The region holds (e, list position); ids[position] gives the vector id, which
// is looked up only for the K_c winners and the threshold-bucket objects.
//
// Why this is the exact top-K_c by (e, id): bucket ids are a monotone
// function of e, and an object is dropped during the scan only when its
// bucket exceeds the current tau, which never falls below tau*; so every
// object in buckets <= tau* was appended.
#pragma once

#include "bbc_internal.cuh"
#include "dev_util.cuh"

namespace bbc {

__device__ __forceinline__ uint32_t sel_bucket(uint32_t e, const bbc_collector_state& st, const uint8_t* map) {
    uint32_t b = 0;
    if (e > st.d_min) {
        b = (e - st.d_min) >> st.sh;
        b = b > 255u ? 255u : b;
    }
    return map[b];
}

// tkeys: tcap 64-bit keys of shared memory for the threshold bucket's objects.
static __device__ void select_query(const DevIndex& ix, const SelectArgs& a, int64_t qi, unsigned long long* tkeys,
                             uint32_t tcap) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t sc[2];
    __shared__ uint8_t map[256];
    __shared__ uint32_t s_out, s_t;
    __shared__ int s_tau;
    __shared__ long long s_below;
    __shared__ unsigned long long s_kmin, s_kmax;
    bbc_collector_state& st = a.state[qi];
    const int tid = threadIdx.x, bs = blockDim.x;
    const int m = st.m;
    const int64_t kc = a.qp.KC(qi);
    const int64_t cap = a.qp.rcap(qi);
    const int64_t n = st.pushed < cap ? st.pushed : cap;
    const uint2* region = a.region + a.qp.roff(qi);
    uint32_t* cand = a.cand + a.qp.coff(qi);
    // early re-rank: carry each candidate's exact distance from the scan (-1: none)
    float* cearly = a.cand_early ? a.cand_early + a.qp.coff(qi) : nullptr;
    const float* rdist = a.rdist ? a.rdist + a.qp.roff(qi) : nullptr;
    for (int i = tid; i < 256; i += bs) map[i] = st.map[i];
    if (warp_id() == 0) {
        // tau* and the count below it
        const unsigned ln = lane_id();
        uint32_t h[8], s = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int b = (int)ln * 8 + i;
            h[i] = b < m ? st.hist[b] : 0u;
            s += h[i];
        }
        const unsigned long long inc = warp_incl_scan64(s);
        const unsigned hit = __ballot_sync(0xFFFFFFFFu, inc >= (unsigned long long)kc);
        if (!hit) {
            if (ln == 0) { s_tau = m; s_below = (long long)n; }
        } else {
            const unsigned src = __ffs(hit) - 1;
            if (ln == src) {
                unsigned long long c = inc - s;
                for (int i = 0; i < 8; ++i) {
                    if (c + h[i] >= (unsigned long long)kc) { s_tau = (int)(ln * 8 + i); s_below = (long long)c; break; }
                    c += h[i];
                }
            }
        }
        if (ln == 0) { s_out = 0; s_t = 0; s_kmin = ~0ull; s_kmax = 0ull; }
    }
    __syncthreads();
    const int tau = s_tau;
    const long long below = s_below;
    const unsigned ln = lane_id();
    const unsigned lt_mask = (1u << ln) - 1u;
    if (tau >= m) {
        // fewer than K_c objects: all appended objects are candidates
        for (int64_t i = tid; i < n && i < kc; i += bs) {
            cand[i] = ix.ids[region[i].y];
            if (cearly) cearly[i] = rdist[i];
        }
        if (tid == 0) {
            a.cand_count[qi] = n < kc ? n : kc;
            st.tau = tau;
            st.below = n;
        }
        return;
    }
    const uint32_t nt = st.hist[tau];
    const bool in_smem = nt <= tcap;
    // pass 1: buckets < tau* go straight out; bucket tau* is staged.  Four
    // entries per thread per step, their id gathers issued together.
    // (the next step's entries are loaded while this step's ids are gathered)
    constexpr int SU = 4;
    uint2 vn[SU];
#pragma unroll
    for (int u = 0; u < SU; ++u) {
        const int64_t i = (int64_t)u * bs + tid;
        vn[u] = i < n ? region[i] : make_uint2(0, 0);
    }
    for (int64_t i0 = 0; i0 < n; i0 += (int64_t)SU * bs) {
        uint2 v[SU];
        uint32_t b[SU], idv[SU];
#pragma unroll
        for (int u = 0; u < SU; ++u) {
            v[u] = vn[u];
            const int64_t inext = i0 + (int64_t)(SU + u) * bs + tid;
            vn[u] = inext < n ? region[inext] : make_uint2(0, 0);
        }
#pragma unroll
        for (int u = 0; u < SU; ++u) {
            const int64_t i = i0 + (int64_t)u * bs + tid;
            b[u] = i < n ? sel_bucket(v[u].x, st, map) : 0xFFFFFFFFu;
        }
#pragma unroll
        for (int u = 0; u < SU; ++u) idv[u] = b[u] <= (uint32_t)tau ? ix.ids[v[u].y] : 0u;
#pragma unroll
        for (int u = 0; u < SU; ++u) {
            const bool take = b[u] < (uint32_t)tau;
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, take);
            if (bal) {
                uint32_t base = 0;
                if (ln == 0) base = atomicAdd(&s_out, (uint32_t)__popc(bal));
                base = __shfl_sync(0xFFFFFFFFu, base, 0);
                const uint32_t pos = base + __popc(bal & lt_mask);
                if (take && (int64_t)pos < kc) {
                    cand[pos] = idv[u];
                    if (cearly) cearly[pos] = rdist[i0 + (int64_t)u * bs + tid];
                }
            }
            if (in_smem && b[u] == (uint32_t)tau) {
                const uint32_t p = atomicAdd(&s_t, 1u);
                if (p < tcap) tkeys[p] = ((unsigned long long)v[u].x << 32) | idv[u];
            }
        }
    }
    __syncthreads();
    const uint32_t s = (uint32_t)(kc - below);
    unsigned long long kth;
    if (in_smem) {
        const uint32_t cnt = min(s_t, tcap);
        // the staged keys share their bits above the highest bit where the
        // smallest and largest differ: the radix select starts below them
        unsigned long long kmn = ~0ull, kmx = 0ull;
        for (uint32_t i = tid; i < cnt; i += bs) {
            kmn = min(kmn, tkeys[i]);
            kmx = max(kmx, tkeys[i]);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            kmn = min(kmn, (unsigned long long)__shfl_xor_sync(0xFFFFFFFFu, kmn, o));
            kmx = max(kmx, (unsigned long long)__shfl_xor_sync(0xFFFFFFFFu, kmx, o));
        }
        if (ln == 0 && kmn <= kmx) {
            atomicMin(&s_kmin, kmn);
            atomicMax(&s_kmax, kmx);
        }
        __syncthreads();
        const unsigned long long diff = s_kmin ^ s_kmax;
        if (diff == 0ull) {
            kth = s_kmin;                                      // one distinct key
        } else {
            const int top = ((63 - __clzll((long long)diff)) / 8) * 8;
            const unsigned long long low = top >= 56 ? ~0ull : ((1ull << (top + 8)) - 1ull);
            const unsigned long long high = s_kmin & ~low;
            kth = high | cta_select_u64(cnt, s - 1, [&](int64_t i) { return tkeys[i] & low; }, hist, sc, top);
        }
        for (uint32_t i0 = 0; i0 < cnt; i0 += bs) {
            const uint32_t i = i0 + tid;
            const bool take = i < cnt && tkeys[i] <= kth;
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, take);
            if (bal) {
                uint32_t base = 0;
                if (ln == 0) base = atomicAdd(&s_out, (uint32_t)__popc(bal));
                base = __shfl_sync(0xFFFFFFFFu, base, 0);
                const uint32_t pos = base + __popc(bal & lt_mask);
                if (take && (int64_t)pos < kc) {
                    cand[pos] = (uint32_t)(tkeys[i] & 0xFFFFFFFFu);
                    if (cearly) cearly[pos] = -1.f;             // the region slot is not kept here
                }
            }
        }
    } else {
        // large threshold bucket: select straight from the region (read-only passes)
        kth = cta_select_u64(n, s - 1, [&](int64_t i) {
            const uint2 v = region[i];
            return sel_bucket(v.x, st, map) == (uint32_t)tau ? (((unsigned long long)v.x << 32) | ix.ids[v.y]) : ~0ull;
        }, hist, sc, 56);
        for (int64_t i0 = 0; i0 < n; i0 += bs) {
            const int64_t i = i0 + tid;
            bool take = false;
            uint32_t id = 0;
            if (i < n) {
                const uint2 v = region[i];
                if (sel_bucket(v.x, st, map) == (uint32_t)tau) {
                    id = ix.ids[v.y];
                    take = (((unsigned long long)v.x << 32) | id) <= kth;
                }
            }
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, take);
            if (bal) {
                uint32_t base = 0;
                if (ln == 0) base = atomicAdd(&s_out, (uint32_t)__popc(bal));
                base = __shfl_sync(0xFFFFFFFFu, base, 0);
                const uint32_t pos = base + __popc(bal & lt_mask);
                if (take && (int64_t)pos < kc) {
                    cand[pos] = id;
                    if (cearly) cearly[pos] = rdist[i];
                }
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        if ((int64_t)s_out != kc) atomicOr(ix.status, kStatusSelectOverrun);
        a.cand_count[qi] = min((int64_t)s_out, kc);
        st.tau = tau;
        st.below = below;
    }
}

}  // namespace bbc
