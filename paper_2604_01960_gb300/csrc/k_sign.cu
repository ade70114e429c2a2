// S9b: the bounded re-rank with a 1-bit sign quantizer (Section 3.4; Obs. 1,
// Alg. 2, Alg. 3).  The paper cites RaBitQ for the bounds without stating
// them; the bounds here are hard (deterministic):
//
//   object o in list l: u = o - c_l, r = P u (P the stored rotation), codes
//   s_i = [r_i > 0] as +-1, alpha = mean |r_i| (stored FP32), e = ||r - alpha s||
//   (rounded up), ||u||^2;
//   query per list: q' = P q - P c_l (FP64, then FP32), lo = min q', Delta =
//   (max q' - lo) / 15, u_i = nearest level in [0, 15], q~ = lo + Delta u,
//   eta = ||q' - q~||;  <q~, s> = lo (2 pc - d) + Delta (2 sum_i u_i b_i - sum_i u_i)
//   with sum_i u_i b_i from four AND + POPC bit planes (exact integers);
//   <P t, r> in alpha <q~, s> +- (|alpha| rounding of <q~, s> + scale (|alpha| eta sqrt(d)
//   + ||q'|| e) + ||q' - P t|| ||r||),  t = q - c_l;
//   ||q - o||^2 = ||t||^2 + ||u||^2 - 2 <t, u>, |<t, u> - <P t, P u>| <= eps ||t|| ||u||
//   with eps = ||P^T P - I||_F; a 2^-20 relative allowance covers the FP32
//   evaluation.  scale = 1 gives hard bounds; both Cauchy-Schwarz terms are
//   worst cases that a random rotation makes about sqrt(d) too wide, so
//   scale = eps0 / sqrt(d - 1) gives intervals in the spirit of RaBitQ's
//   probabilistic bound (not hard).
//
// Collection (a result buffer on the upper bound, Alg. 1 and Alg. 3): the
// histogram counts every scanned object by the bucket of its upper bound;
// tau (Update, >= k) therefore bounds the bucket of U_k, the k-th smallest
// upper bound, and an object is appended when the bucket of its lower bound
// is <= tau, which keeps every object of S = {lb <= U_k}.
//
// Re-rank in two rounds with exact returned distances: B = the k smallest
// (ub, slot) of S are re-ranked first; U' = the largest upper FP32 bound in
// B (>= Dist_k); then S' = {o in S \ B : lb <= U'}; the final k come from
// B u S' in exact order (FP32 with its bound, FP64 at ties).
#include "bbc_internal.cuh"
#include "dev_util.cuh"

namespace bbc {

namespace {

constexpr int RT_TM = 64, RT_TN = 64, RT_TK = 16, RT_THREADS = 256;
constexpr int SG_THREADS = 512;
constexpr int SG_MAXW = 64;                  // d <= 2048

// ---------------------------------------------------------------------------
// FP64 tiled product with the rotation: out[i][r] = sum_j P[r][j] a_i[j].
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(RT_THREADS) rotate_f64_kernel(const float* __restrict__ A,
                                                                const int64_t* __restrict__ rows,
                                                                const int32_t* __restrict__ lists,
                                                                const float* __restrict__ cent,
                                                                const float* __restrict__ P, int64_t n, int d,
                                                                double* __restrict__ out) {
    __shared__ double As[RT_TK][RT_TM];
    __shared__ double Ps[RT_TK][RT_TN];
    const int tid = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.y * RT_TM;
    const int r0 = blockIdx.x * RT_TN;
    const int ty = tid / 16, tx = tid % 16;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < d; k0 += RT_TK) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = tid + u * RT_THREADS;
            const int rr = e / RT_TK, kk = e % RT_TK;
            const int64_t i = i0 + rr;
            double v = 0.0;
            if (i < n && k0 + kk < d) {
                const int64_t row = rows ? rows[i] : i;
                if (row >= 0) {
                    v = (double)A[row * d + k0 + kk];
                    if (lists) v -= (double)cent[(int64_t)lists[i] * d + k0 + kk];
                }
            }
            As[kk][rr] = v;
            const int c = r0 + rr;
            Ps[kk][rr] = (c < d && k0 + kk < d) ? (double)P[(int64_t)c * d + k0 + kk] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < RT_TK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int x = 0; x < 4; ++x) { a[x] = As[kk][ty * 4 + x]; b[x] = Ps[kk][tx * 4 + x]; }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        const int64_t i = i0 + ty * 4 + x;
        if (i >= n) continue;
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int c = r0 + tx * 4 + y;
            if (c < d) out[i * d + c] = acc[x][y];
        }
    }
}

// ---------------------------------------------------------------------------
// Codes and factors of one slot per warp from its rotated residual.
// ---------------------------------------------------------------------------
__global__ void sign_factors_kernel(const double* __restrict__ R, int64_t s0, int64_t n, int d,
                                    const int64_t* __restrict__ rows, const int32_t* __restrict__ lists,
                                    const float* __restrict__ vec, const float* __restrict__ cent,
                                    uint32_t* __restrict__ codes, float4* __restrict__ fac) {
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    const int64_t slot = s0 + i;
    const unsigned ln = lane_id();
    const int W = d / 32;
    const int64_t blk = slot / 32;
    const int t = (int)(slot % 32);
    const int64_t row = rows[slot];
    if (row < 0) {                                        // padding slot
        for (int w = ln; w < W; w += 32) codes[(blk * W + w) * 32 + t] = 0u;
        if (ln == 0) fac[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const double* r = R + i * d;
    double sabs = 0.0, un2 = 0.0, rn2 = 0.0;
    int pc = 0;
    const float* o = vec + row * d;
    const float* c = cent + (int64_t)lists[slot] * d;
    for (int w = 0; w < W; ++w) {
        const double v = r[w * 32 + ln];
        const unsigned bits = __ballot_sync(0xFFFFFFFFu, v > 0.0);
        if (ln == 0) codes[(blk * W + w) * 32 + t] = bits;
        pc += __popc(bits);
        sabs += fabs(v);
        rn2 += v * v;
        const double uu = (double)o[w * 32 + ln] - (double)c[w * 32 + ln];
        un2 += uu * uu;
    }
    for (int s = 16; s; s >>= 1) {
        sabs += __shfl_xor_sync(0xFFFFFFFFu, sabs, s);
        un2 += __shfl_xor_sync(0xFFFFFFFFu, un2, s);
        rn2 += __shfl_xor_sync(0xFFFFFFFFu, rn2, s);
    }
    const float alpha = (float)(sabs / d);                // the stored alpha defines e below
    double e2 = 0.0;
    for (int w = 0; w < W; ++w) {
        const double v = r[w * 32 + ln];
        const double df = v - (v > 0.0 ? (double)alpha : -(double)alpha);
        e2 += df * df;
    }
    for (int s = 16; s; s >>= 1) e2 += __shfl_xor_sync(0xFFFFFFFFu, e2, s);
    if (ln == 0) {
        // e covers the FP64 evaluation of r = P u (about d^1.5 2^-53 ||u||)
        const float e = __double2float_ru((sqrt(e2) + 1e-10 * sqrt(un2)) * (1.0 + 1e-12));
        fac[slot] = make_float4(alpha, e, (float)un2, (float)pc);
    }
    (void)rn2;
}

// ---------------------------------------------------------------------------
// The bounds.
// ---------------------------------------------------------------------------
struct ListSetup {
    float lo, delta, tn2, tn, eta_sd, qn, dterm;
    int usum;
};

// Per-list query preparation (all threads of the CTA): q' in sq, the four bit
// planes, and the list's scalars.  qnorm = ||q||.
__device__ void sign_list_setup(const DevIndex& ix, const double* __restrict__ qrot, const float* __restrict__ q,
                                float qnorm, int l, float* sq, uint32_t (*planes)[SG_MAXW], ListSetup* ls,
                                double* redd, float* redf, int* redi) {
    const int d = ix.d, W = d / 32;
    const int tid = threadIdx.x, nw = blockDim.x >> 5;
    const double* cr = ix.crot + (int64_t)l * d;
    const float* c = ix.centroids + (int64_t)l * d;
    double tn2 = 0.0, qn2 = 0.0;
    float lo = INFINITY, hi = -INFINITY;
    for (int i = tid; i < d; i += blockDim.x) {
        const float f = (float)(qrot[i] - cr[i]);
        sq[i] = f;
        qn2 += (double)f * (double)f;
        const double t = (double)q[i] - (double)c[i];
        tn2 += t * t;
        lo = fminf(lo, f);
        hi = fmaxf(hi, f);
    }
    for (int s = 16; s; s >>= 1) {
        tn2 += __shfl_xor_sync(0xFFFFFFFFu, tn2, s);
        qn2 += __shfl_xor_sync(0xFFFFFFFFu, qn2, s);
        lo = fminf(lo, __shfl_xor_sync(0xFFFFFFFFu, lo, s));
        hi = fmaxf(hi, __shfl_xor_sync(0xFFFFFFFFu, hi, s));
    }
    if (lane_id() == 0) {
        redd[warp_id() * 3 + 0] = tn2;
        redd[warp_id() * 3 + 1] = qn2;
        redf[warp_id() * 2 + 0] = lo;
        redf[warp_id() * 2 + 1] = hi;
    }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, b = 0.0;
        float l0 = INFINITY, h0 = -INFINITY;
        for (int w = 0; w < nw; ++w) {
            a += redd[w * 3 + 0];
            b += redd[w * 3 + 1];
            l0 = fminf(l0, redf[w * 2 + 0]);
            h0 = fmaxf(h0, redf[w * 2 + 1]);
        }
        ls->lo = l0;
        ls->delta = (h0 - l0) / 15.f;
        ls->tn2 = (float)a;
        ls->tn = __double2float_ru(sqrt(a) * (1.0 + 1e-12));
        ls->qn = __double2float_ru(sqrt(b) * (1.0 + 1e-12));
        // ||q' - P t||: FP32 rounding of q' plus the FP64 products (about d^1.5 2^-53 (||q|| + ||c||))
        ls->dterm = 2.384185791015625e-7f * ls->qn + 1e-10f * (qnorm + sqrtf(ix.cnorm[l]));
    }
    __syncthreads();
    const float lo0 = ls->lo, dl = ls->delta;
    double eta2 = 0.0;
    int usum = 0;
    for (int w = warp_id(); w < W; w += nw) {
        const int i = w * 32 + lane_id();
        const float f = sq[i];
        int u = 0;
        if (dl > 0.f) {
            const float v = rintf((f - lo0) / dl);
            u = v < 0.f ? 0 : (v > 15.f ? 15 : (int)v);
        }
        const double df = (double)f - ((double)lo0 + (double)dl * (double)u);
        eta2 += df * df;
        usum += u;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const unsigned bits = __ballot_sync(0xFFFFFFFFu, (u >> j) & 1);
            if (lane_id() == 0) planes[j][w] = bits;
        }
    }
    for (int s = 16; s; s >>= 1) {
        eta2 += __shfl_xor_sync(0xFFFFFFFFu, eta2, s);
        usum += __shfl_xor_sync(0xFFFFFFFFu, usum, s);
    }
    if (lane_id() == 0) { redd[warp_id() * 3 + 2] = eta2; redi[warp_id()] = usum; }
    __syncthreads();
    if (tid == 0) {
        double e = 0.0;
        int us = 0;
        for (int w = 0; w < nw; ++w) { e += redd[w * 3 + 2]; us += redi[w]; }
        ls->eta_sd = __double2float_ru(sqrt(e * (double)d) * (1.0 + 1e-12));
        ls->usum = us;
    }
    __syncthreads();
}

// Bounds of the object in slot (codes in the block layout), with the planes
// and scalars of its list.
__device__ __forceinline__ void sign_bound(const DevIndex& ix, int64_t slot, const uint32_t (*planes)[SG_MAXW],
                                           const ListSetup& ls, float scale, float eps, float& lb, float& ub) {
    const int W = ix.d >> 5;
    const int64_t blk = slot >> 5;
    const int t = (int)(slot & 31);
    const uint32_t* cw = ix.sgn + blk * W * 32 + t;
    int s2 = 0;
#pragma unroll 6
    for (int w = 0; w < W; ++w) {
        const uint32_t c = __ldg(cw + w * 32);
        s2 += __popc(planes[0][w] & c) + 2 * __popc(planes[1][w] & c) + 4 * __popc(planes[2][w] & c) +
              8 * __popc(planes[3][w] & c);
    }
    const float4 f = __ldg(ix.sfac + slot);
    const float S1 = 2.f * f.w - (float)ix.d;
    const float S2 = (float)(2 * s2 - ls.usum);
    const float x1 = ls.lo * S1, x2 = ls.delta * S2;
    const float X = x1 + x2;
    const float eX = 2.384185791015625e-7f * (fabsf(x1) + fabsf(x2));       // 2^-22 (|x1| + |x2|)
    const float alpha = f.x, e = f.y, un2 = f.z;
    const float un = sqrtf(un2) * (1.f + 2.384185791015625e-7f);
    const float est = alpha * X;
    const float H = fabsf(alpha) * eX + scale * (fabsf(alpha) * ls.eta_sd + ls.qn * e) + ls.dterm * un * (1.f + eps);
    const float base = ls.tn2 + un2;
    const float rotE = 2.f * eps * ls.tn * un;
    const float slack = 9.5367431640625e-7f * (base + 2.f * fabsf(est) + 2.f * H + rotE);   // 2^-20
    lb = fmaxf(base - 2.f * (est + H) - rotE - slack, 0.f);
    ub = base - 2.f * (est - H) + rotE + slack;
}

__device__ __forceinline__ uint32_t sg_bucket(uint32_t key, uint32_t dmin, int sh, const uint8_t* map) {
    uint32_t b = key < dmin ? 0u : (key - dmin) >> sh;
    return map[b < 255u ? b : 255u];
}

__device__ __forceinline__ uint32_t sg_append(bool take, uint32_t* counter) {
    const unsigned m = __ballot_sync(0xFFFFFFFFu, take);
    const unsigned ln = lane_id();
    const int leader = m ? __ffs(m) - 1 : 0;
    uint32_t base = 0;
    if (m && (int)ln == leader) base = atomicAdd(counter, (uint32_t)__popc(m));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    return base + __popc(m & ((1u << ln) - 1u));
}

// ---------------------------------------------------------------------------
// Scan + result buffer on the upper bounds (one CTA per query).  DEBUG: write
// the bounds of every scanned object in probe order instead.
// ---------------------------------------------------------------------------
template <bool DEBUG>
__global__ void __launch_bounds__(SG_THREADS) sign_scan_kernel(DevIndex ix, SignArgs a) {
    extern __shared__ float sq[];                          // d floats
    __shared__ uint32_t planes[4][SG_MAXW];
    __shared__ ListSetup ls;
    __shared__ double redd[(SG_THREADS / 32) * 3];
    __shared__ float redf[(SG_THREADS / 32) * 2];
    __shared__ int redi[SG_THREADS / 32];
    __shared__ uint32_t hist[256];
    __shared__ uint32_t sc[2];
    __shared__ uint8_t smap[256];
    __shared__ uint32_t s_cnt, s_tau, s_dmin, s_over;
    __shared__ int s_sh, s_ns;
    __shared__ int64_t s_sq;
    __shared__ float s_qnorm;
    const int64_t qi = blockIdx.x;
    const int d = ix.d;
    const int P = a.qp.P(qi);
    const int kq = a.qp.K(qi);
    const int m = a.m;
    const int32_t* lists = a.lists + a.qp.poff(qi);
    uint4* region = a.region + a.qp.roff(qi);
    const int64_t cap = a.qp.rcap(qi);
    const double* qrot = a.qrot + qi * d;
    const float* q = a.q + qi * d;
    const float eps = (float)(ix.eps_p * (1.0 + 1e-6)) + 1e-12f;
    const int tid = threadIdx.x, nw = blockDim.x >> 5;
    if (tid == 0) {
        double qq = 0.0;
        for (int i = 0; i < d; ++i) qq += (double)q[i] * (double)q[i];
        s_qnorm = __double2float_ru(sqrt(qq) * (1.0 + 1e-12));
        // sample plan: at least min(sample_min, P) lists, extended to min(k, S_q) objects
        int64_t sqn = 0;
        for (int j = 0; j < P; ++j) sqn += ix.list_len[lists[j]];
        s_sq = sqn;
        const int64_t want = sqn < kq ? sqn : kq;
        const int smin = a.sample_min < P ? a.sample_min : P;
        int ns = 0;
        int64_t acc = 0;
        while (ns < P && (ns < smin || acc < want)) acc += ix.list_len[lists[ns++]];
        s_ns = ns;
        s_cnt = 0;
        s_over = 0;
        s_tau = (uint32_t)m;
    }
    __syncthreads();
    const float qnorm = s_qnorm;
    if (DEBUG) {
        int64_t base = 0;
        for (int j = 0; j < P; ++j) {
            const int l = lists[j];
            sign_list_setup(ix, qrot, q, qnorm, l, sq, planes, &ls, redd, redf, redi);
            const int len = ix.list_len[l];
            const int64_t b0 = ix.list_blk[l];
            for (int p = tid; p < len; p += blockDim.x) {
                float lb, ub;
                sign_bound(ix, b0 * 32 + p, planes, ls, a.scale, eps, lb, ub);
                if (base + p < cap) {
                    a.dbg_lb[a.qp.roff(qi) + base + p] = lb;
                    a.dbg_ub[a.qp.roff(qi) + base + p] = ub;
                }
            }
            base += len;
        }
        if (tid == 0) {
            a.scanned[qi] = s_sq;
            if (s_sq > cap) atomicOr(ix.status, kStatusRegionOverrun);
        }
        return;
    }
    // ---- sample: upper-bound keys of the first lists ----
    const int ns = s_ns;
    for (int j = 0; j < ns; ++j) {
        const int l = lists[j];
        sign_list_setup(ix, qrot, q, qnorm, l, sq, planes, &ls, redd, redf, redi);
        const int len = ix.list_len[l];
        const int64_t b0 = ix.list_blk[l];
        const int nb = (len + 31) >> 5;
        for (int b = warp_id(); b < nb; b += nw) {
            const int p = b * 32 + (int)lane_id();
            const bool valid = p < len;
            float lb = 0.f, ub = 0.f;
            if (valid) sign_bound(ix, b0 * 32 + p, planes, ls, a.scale, eps, lb, ub);
            const uint32_t pos = sg_append(valid, &s_cnt);
            if (valid && pos < cap) region[pos] = make_uint4(0u, f32_key(ub), 0u, 0u);
        }
        __syncthreads();
    }
    // ---- codebook: d_min, d_max = t-th smallest sampled key, equal-depth map ----
    const int64_t nsamp = min((int64_t)s_cnt, cap);
    if (nsamp > 0) {
        const int64_t t = nsamp < kq ? nsamp : kq;
        const uint32_t dmax = cta_select_u32(nsamp, (uint32_t)(t - 1), [&](int64_t i) { return region[i].y; },
                                             hist, sc, 24);
        uint32_t mn = 0xFFFFFFFFu;
        for (int64_t i = tid; i < nsamp; i += blockDim.x) mn = min(mn, region[i].y);
        mn = __reduce_min_sync(0xFFFFFFFFu, mn);
        if (tid == 0) s_dmin = 0xFFFFFFFFu;
        __syncthreads();
        if (lane_id() == 0) atomicMin(&s_dmin, mn);
        for (int i = tid; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        if (tid == 0) {
            int sh = 0;
            while (((dmax - s_dmin) >> sh) > 255u) ++sh;
            s_sh = sh;
        }
        __syncthreads();
        const uint32_t dmin = s_dmin;
        const int sh = s_sh;
        for (int64_t i = tid; i < nsamp; i += blockDim.x) {
            const uint32_t k = region[i].y;
            if (k <= dmax) atomicAdd(&hist[min((k - dmin) >> sh, 255u)], 1u);
        }
        __syncthreads();
        if (tid == 0) {                                     // equal-width bins -> equal-depth buckets
            uint64_t T = 0;
            for (int b = 0; b < 256; ++b) T += hist[b];
            uint64_t cum = 0;
            for (int b = 0; b < 256; ++b) {
                const uint64_t v = T ? (uint64_t)m * cum / T : 0;
                smap[b] = (uint8_t)(v < (uint64_t)(m - 1) ? v : (uint64_t)(m - 1));
                cum += hist[b];
            }
        }
        __syncthreads();
    } else {
        if (tid == 0) { s_dmin = 0; s_sh = 0; }
        for (int i = tid; i < 256; i += blockDim.x) smap[i] = 0;
        __syncthreads();
    }
    for (int i = tid; i < 256; i += blockDim.x) hist[i] = 0;
    if (tid == 0) { s_cnt = 0; s_tau = (uint32_t)m; }
    __syncthreads();
    const uint32_t dmin = s_dmin;
    const int sh = s_sh;
    // ---- main pass: histogram on the upper bound, push on the lower bound ----
    for (int j = 0; j < P; ++j) {
        const int l = lists[j];
        sign_list_setup(ix, qrot, q, qnorm, l, sq, planes, &ls, redd, redf, redi);
        const int len = ix.list_len[l];
        const int64_t b0 = ix.list_blk[l];
        const int nb = (len + 31) >> 5;
        const uint32_t tau = s_tau;
        for (int b = warp_id(); b < nb; b += nw) {
            const int p = b * 32 + (int)lane_id();
            const bool valid = p < len;
            float lb = 0.f, ub = 0.f;
            if (valid) sign_bound(ix, b0 * 32 + p, planes, ls, a.scale, eps, lb, ub);
            const uint32_t ubk = f32_key(ub), lbk = f32_key(lb);
            if (valid) atomicAdd(&hist[sg_bucket(ubk, dmin, sh, smap)], 1u);
            const bool push = valid && sg_bucket(lbk, dmin, sh, smap) <= tau;
            const uint32_t pos = sg_append(push, &s_cnt);
            if (push) {
                if (pos < cap) region[pos] = make_uint4(lbk, ubk, (uint32_t)(b0 * 32 + p), 0u);
                else s_over = 1;
            }
        }
        __syncthreads();
        if (tid == 0) {                                     // Update: first bucket reaching k
            uint32_t run = 0, t = (uint32_t)m;
            for (int i = 0; i < m; ++i) {
                run += hist[i];
                if (run >= (uint32_t)kq) { t = (uint32_t)i; break; }
            }
            s_tau = min(s_tau, t);
        }
        __syncthreads();
    }
    if (tid == 0) {
        a.pushed[qi] = min((int64_t)s_cnt, cap);
        a.scanned[qi] = s_sq;
        if (s_over) atomicOr(ix.status, kStatusRegionOverrun);
    }
}

// ---------------------------------------------------------------------------
// First round: U_k, S, the k smallest (ub, slot) of S (B) and the rest of S.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(SG_THREADS) sign_select_kernel(DevIndex ix, SignSelectArgs a) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t sc[2];
    __shared__ uint32_t s_b, s_r;
    const int64_t qi = blockIdx.x;
    const int64_t n = a.pushed[qi];
    const int64_t kq = a.qp.K(qi);
    const int64_t off = a.qp.coff(qi);
    const uint4* reg = a.region + a.qp.roff(qi);
    if (threadIdx.x == 0) { s_b = 0; s_r = 0; }
    __syncthreads();
    const bool all = a.scanned[qi] <= kq;                   // every scanned object is a result
    uint32_t uk = 0xFFFFFFFFu;
    unsigned long long kth = ~0ull;
    if (!all && n > 0) {
        const uint32_t r = (uint32_t)(min(n, kq) - 1);
        uk = cta_select_u32(n, r, [&](int64_t i) { return reg[i].y; }, hist, sc, 24);
        kth = cta_select_u64(n, r, [&](int64_t i) { return ((unsigned long long)reg[i].y << 32) | reg[i].z; },
                             hist, sc, 56);
    }
    const int64_t n_pad = (n + 31) / 32 * 32;
    for (int64_t i = threadIdx.x; i < n_pad; i += blockDim.x) {
        bool inb = false, inr = false;
        uint4 e = make_uint4(0, 0, 0, 0);
        if (i < n) {
            e = reg[i];
            inb = all || (((unsigned long long)e.y << 32) | e.z) <= kth;
            inr = !inb && e.x <= uk;
        }
        const uint32_t sb = sg_append(inb, &s_b);
        if (inb) a.clist[off + sb] = ix.ids[e.z];
        const uint32_t sr = sg_append(inr, &s_r);
        if (inr) { a.rest_key[off + sr] = e.x; a.rest_id[off + sr] = ix.ids[e.z]; }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a.n_b[qi] = s_b;
        a.n_c[qi] = s_b;
        a.n_rest[qi] = s_r;
        atomicAdd(&a.totals[0], (unsigned long long)a.scanned[qi]);
        atomicAdd(&a.totals[1], (unsigned long long)(s_b + s_r));
    }
}

// Second round: U' = the largest FP32 upper bound in B; S' = rest with lb <= U'.
__global__ void __launch_bounds__(SG_THREADS) sign_filter_kernel(DevIndex ix, SignSelectArgs a) {
    __shared__ uint32_t s_u, s_c;
    const int64_t qi = blockIdx.x;
    const int64_t nb = a.n_b[qi];
    const int64_t nr = a.n_rest[qi];
    const int64_t off = a.qp.coff(qi);
    if (threadIdx.x == 0) { s_u = 0u; s_c = 0u; }
    __syncthreads();
    uint32_t mx = 0u;
    for (int64_t i = threadIdx.x; i < nb; i += blockDim.x) mx = max(mx, f32_key(__fadd_ru(a.cd[off + i], a.cr[off + i])));
    mx = __reduce_max_sync(0xFFFFFFFFu, mx);
    if (lane_id() == 0) atomicMax(&s_u, mx);
    __syncthreads();
    const uint32_t up = s_u;
    const int64_t n_pad = (nr + 31) / 32 * 32;
    for (int64_t i = threadIdx.x; i < n_pad; i += blockDim.x) {
        const bool take = i < nr && a.rest_key[off + i] <= up;
        const uint32_t s = sg_append(take, &s_c);
        if (take) a.clist[off + nb + s] = a.rest_id[off + i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a.n_c[qi] = nb + s_c;
        atomicAdd(&a.totals[2], (unsigned long long)(nb + s_c));
        atomicAdd(&a.totals[3], 1ull);
    }
}

}  // namespace

cudaError_t launch_rotate_f64(const float* A, const int64_t* rows, const int32_t* lists, const float* centroids,
                              const float* P, int64_t n, int d, double* out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    dim3 grid((unsigned)((d + RT_TN - 1) / RT_TN), (unsigned)((n + RT_TM - 1) / RT_TM));
    rotate_f64_kernel<<<grid, RT_THREADS, 0, st>>>(A, rows, lists, centroids, P, n, d, out);
    return cudaGetLastError();
}

cudaError_t launch_sign_factors(const double* R, int64_t s0, int64_t n, int d, const int64_t* rows,
                                     const int32_t* lists, const float* vec, const float* cent, uint32_t* codes,
                                     float4* fac, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int wpb = 8;
    sign_factors_kernel<<<(unsigned)((n + wpb - 1) / wpb), 32 * wpb, 0, st>>>(R, s0, n, d, rows, lists, vec, cent,
                                                                            codes, fac);
    return cudaGetLastError();
}

cudaError_t launch_sign_scan(const DevIndex& ix, int64_t nq, const SignArgs& a, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    if (ix.d % 32 || ix.d > 32 * SG_MAXW) return cudaErrorInvalidValue;
    const size_t smem = (size_t)ix.d * sizeof(float);
    if (a.dbg_lb) sign_scan_kernel<true><<<(unsigned)nq, SG_THREADS, smem, st>>>(ix, a);
    else sign_scan_kernel<false><<<(unsigned)nq, SG_THREADS, smem, st>>>(ix, a);
    return cudaGetLastError();
}

cudaError_t launch_sign_select(const DevIndex& ix, int64_t nq, const SignSelectArgs& a, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    sign_select_kernel<<<(unsigned)nq, SG_THREADS, 0, st>>>(ix, a);
    return cudaGetLastError();
}

cudaError_t launch_sign_filter(const DevIndex& ix, int64_t nq, const SignSelectArgs& a, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    sign_filter_kernel<<<(unsigned)nq, SG_THREADS, 0, st>>>(ix, a);
    return cudaGetLastError();
}

}  // namespace bbc
