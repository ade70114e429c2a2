// Device-side building blocks: order-preserving keys, CTA-wide radix select
// and bitonic sort in shared memory, warp scans.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bbc {

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned warp_id() { return threadIdx.x >> 5; }

// Order-preserving map float -> u32 (ascending floats give ascending keys).
// -0 is folded onto +0 first so that equal values get equal keys.
__device__ __forceinline__ uint32_t f32_key(float f) {
    f = f + 0.0f;
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_f32(uint32_t k) {
    uint32_t b = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
    return __uint_as_float(b);
}
__device__ __forceinline__ unsigned long long f64_key(double f) {
    f = f + 0.0;
    unsigned long long b = (unsigned long long)__double_as_longlong(f);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

// f64_key((double)x) for a float x built with integer instructions (double
// precision is slow on this GPU); subnormals, infinities and NaN take the
// double path.
__device__ __forceinline__ unsigned long long f64_key_f32(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t e = (b >> 23) & 0xFFu;
    const uint32_t m = b & 0x7FFFFFu;
    unsigned long long db;
    if (e == 0u && m == 0u) {
        db = 0ull;                                               // -0 orders as +0
    } else if (e == 0u || e == 0xFFu) {
        return f64_key((double)x);
    } else {
        db = ((unsigned long long)(b >> 31) << 63) | ((unsigned long long)(e + 896u) << 52) |
             ((unsigned long long)m << 29);
    }
    return (db & 0x8000000000000000ull) ? ~db : (db | 0x8000000000000000ull);
}

__device__ __forceinline__ double key_f64(unsigned long long k) {
    unsigned long long b = (k & 0x8000000000000000ull) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
    return __longlong_as_double((long long)b);
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane_id() >= (unsigned)o) v += t;
    }
    return v;
}

__device__ __forceinline__ unsigned long long warp_incl_scan64(unsigned long long v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long t = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane_id() >= (unsigned)o) v += t;
    }
    return v;
}

// Warp 0 helper: given hist[256] (u32) and a 0-based rank r, find the digit
// d with cum(<d) <= r < cum(<=d); returns (d, r - cum(<d)) to all lanes of
// warp 0.  Requires sum(hist) > r.
__device__ __forceinline__ void warp_find_digit(const uint32_t* hist, uint32_t r, uint32_t* digit,
                                                uint32_t* rem) {
    const unsigned ln = lane_id();
    uint32_t h[8];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) { h[i] = hist[ln * 8 + i]; s += h[i]; }
    uint32_t inc = warp_incl_scan(s);
    uint32_t exc = inc - s;
    unsigned hit = __ballot_sync(0xFFFFFFFFu, r < inc);
    unsigned src = __ffs(hit) - 1;
    if (ln == src) {
        uint32_t c = exc;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (r < c + h[i]) { *digit = ln * 8 + i; *rem = r - c; break; }
            c += h[i];
        }
    }
}

// CTA-wide selection: the r-th smallest (0-based) of n u32 keys produced by
// get(i), examining 8-bit digits from bit `top` downwards (keys must be
// < 2^(top+8)).  hist: 256 u32 in shared memory; sc: 2 u32 in shared memory.
// Every thread of the block must call it.
template <typename Get>
__device__ uint32_t cta_select_u32(int64_t n, uint32_t r, Get get, uint32_t* hist, uint32_t* sc,
                                   int top = 24) {
    uint32_t prefix = 0, mask = 0;
    for (int sh = top; sh >= 0; sh -= 8) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        // four loads in flight per thread before the shared atomics
        const int64_t bs = blockDim.x;
        for (int64_t i = threadIdx.x; i < n; i += 4 * bs) {
            uint32_t k[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) k[u] = i + u * bs < n ? get(i + u * bs) : 0u;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (i + u * bs < n && (k[u] & mask) == prefix) atomicAdd(&hist[(k[u] >> sh) & 255u], 1u);
        }
        __syncthreads();
        if (warp_id() == 0) warp_find_digit(hist, r, &sc[0], &sc[1]);
        __syncthreads();
        prefix |= sc[0] << sh;
        mask |= 255u << sh;
        r = sc[1];
        __syncthreads();
    }
    return prefix;
}

// Same for 64-bit keys.
template <typename Get>
__device__ unsigned long long cta_select_u64(int64_t n, uint32_t r, Get get, uint32_t* hist,
                                             uint32_t* sc, int top = 56) {
    unsigned long long prefix = 0, mask = 0;
    for (int sh = top; sh >= 0; sh -= 8) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            unsigned long long k = get(i);
            if ((k & mask) == prefix) atomicAdd(&hist[(unsigned)(k >> sh) & 255u], 1u);
        }
        __syncthreads();
        if (warp_id() == 0) warp_find_digit(hist, r, &sc[0], &sc[1]);
        __syncthreads();
        prefix |= (unsigned long long)sc[0] << sh;
        mask |= 255ull << sh;
        r = sc[1];
        __syncthreads();
    }
    return prefix;
}

// Ascending bitonic sort of n (a power of two) 64-bit keys in shared memory.
__device__ inline void cta_bitonic_u64(unsigned long long* a, int n) {
    for (int k = 2; k <= n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                int p = i ^ j;
                if (p > i) {
                    unsigned long long x = a[i], y = a[p];
                    bool up = (i & k) == 0;
                    if ((x > y) == up) { a[i] = y; a[p] = x; }
                }
            }
            __syncthreads();
        }
    }
}

// Ascending bitonic sort of (key, val) pairs ordered by (key, val).
__device__ inline void cta_bitonic_kv(unsigned long long* key, uint32_t* val, int n) {
    for (int k = 2; k <= n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                int p = i ^ j;
                if (p > i) {
                    unsigned long long x = key[i], y = key[p];
                    uint32_t u = val[i], v = val[p];
                    bool gt = x > y || (x == y && u > v);
                    bool up = (i & k) == 0;
                    if (gt == up) { key[i] = y; key[p] = x; val[i] = v; val[p] = u; }
                }
            }
            __syncthreads();
        }
    }
}

__host__ __device__ inline int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

}  // namespace bbc
