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
// Estimator mode (est = 1): RaBitQ's estimator and its probabilistic bound.
//   <o_bar, o_r> = alpha sqrt(d) / ||r|| with ||r||^2 = e^2 + d alpha^2 (r -
//   alpha s is orthogonal to s); the estimate of <q', r> is kappa <q~, s>,
//   kappa = ||r||^2 / (d alpha), within
//     eps0 / sqrt(d - 1) ||q'|| ||r|| e / (alpha sqrt(d))   (the estimator's bound)
//     + kappa eps0 eta                                      (the 4-bit query, same confidence)
//   with high probability over the random rotation; the rest as above.
//
// Collection (a result buffer on the upper bound, Alg. 1 and Alg. 3): the
// histogram counts every scanned object by the bucket of its upper bound;
// tau (Update, >= k) therefore bounds the bucket of U_k, the k-th smallest
// upper bound, and an object is appended when the bucket of its lower bound
// is <= tau, which keeps every object of S = {lb <= U_k}.
//
// Re-rank in two rounds with exact returned distances: B = the ceil(f k)
// members of S with the smallest interval centre (lb + ub) / 2 (slot breaking
// ties) are re-ranked first; U' = the k-th smallest FP32 upper bound of their
// distances (>= Dist_k: any k objects have a k-th smallest >= Dist_k); then
// S' = {o in S \ B : lb <= U'}; the final k come from B u S' in exact order
// (FP32 with its bound, FP64 at ties).  Centres put the likeliest members
// first, so U' lands near Dist_k and S' stays small.
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
// Query preparation per (query, probed list), one warp each: q' = P q - P c_l
// (FP64 difference rounded to FP32), its 4-bit levels as four bit planes, and
// the list's scalars, written as one record of R = 4W + 8 words:
//   [plane j word w] (j-major), lo, Delta, ||t||^2, ||t|| (up), eta sqrt(d)
//   (up), ||q'|| (up), dterm, sum u.
// Sums are FP32; each carries its rounding: a sum of squares of n terms
// evaluated with chains of at most c roundings is within 2 c 2^-24 of the
// exact value (relative), c = W + 8 here.
// ---------------------------------------------------------------------------
struct ListSetup {
    float lo, delta, tn2, tn, eta_sd, qn, dterm;
    int usum;
    float eta;          // eta itself (rounded up), for the estimator mode
};

__host__ __device__ inline int sign_rec_words(int d) { return 4 * (d / 32) + 8; }

__global__ void sign_prep_kernel(DevIndex ix, SignArgs a, uint32_t* __restrict__ rec) {
    const int64_t qi = blockIdx.y;
    const int j = blockIdx.x * (blockDim.x >> 5) + (int)(threadIdx.x >> 5);
    const int P = a.qp.P(qi);
    if (j >= P) return;
    const int d = ix.d, W = d / 32;
    const unsigned ln = lane_id();
    const int l = a.lists[a.qp.poff(qi) + j];
    const double* qr = a.qrot + qi * d;
    const double* cr = ix.crot + (int64_t)l * d;
    const float* q = a.q + qi * d;
    const float* c = ix.centroids + (int64_t)l * d;
    float qf[SG_MAXW];
    float lo = INFINITY, hi = -INFINITY, qn2 = 0.f, tn2 = 0.f, qq2 = 0.f;
#pragma unroll 4
    for (int w = 0; w < W; ++w) {
        const int i = w * 32 + (int)ln;
        const float f = (float)(qr[i] - cr[i]);
        qf[w] = f;
        lo = fminf(lo, f);
        hi = fmaxf(hi, f);
        qn2 = fmaf(f, f, qn2);
        const float t = q[i] - c[i];
        tn2 = fmaf(t, t, tn2);
        qq2 = fmaf(q[i], q[i], qq2);
    }
    for (int o = 16; o; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xFFFFFFFFu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xFFFFFFFFu, hi, o));
        qn2 += __shfl_xor_sync(0xFFFFFFFFu, qn2, o);
        tn2 += __shfl_xor_sync(0xFFFFFFFFu, tn2, o);
        qq2 += __shfl_xor_sync(0xFFFFFFFFu, qq2, o);
    }
    const float g = 2.f * (float)(W + 8) * 5.9604644775390625e-8f;
    const float delta = (hi - lo) / 15.f;
    const float inv = delta > 0.f ? 1.f / delta : 0.f;
    uint32_t* out = rec + (a.qp.poff(qi) + j) * (int64_t)sign_rec_words(d);
    float e2 = 0.f;
    int usum = 0;
#pragma unroll 4
    for (int w = 0; w < W; ++w) {
        int u = 0;
        if (delta > 0.f) {
            const float v = rintf((qf[w] - lo) * inv);
            u = v < 0.f ? 0 : (v > 15.f ? 15 : (int)v);
        }
        const float df = qf[w] - fmaf(delta, (float)u, lo);
        e2 = fmaf(df, df, e2);
        usum += u;
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const unsigned bits = __ballot_sync(0xFFFFFFFFu, (u >> jj) & 1);
            if (ln == (unsigned)(w & 31)) out[jj * W + w] = bits;
        }
    }
    for (int o = 16; o; o >>= 1) {
        e2 += __shfl_xor_sync(0xFFFFFFFFu, e2, o);
        usum += __shfl_xor_sync(0xFFFFFFFFu, usum, o);
    }
    if (ln == 0) {
        const float up = 1.f + 2.384185791015625e-7f;                    // 1 + 2^-22 for the square roots
        const float qn = sqrtf(qn2 * (1.f + g)) * up;
        // eta = ||q' - (lo + Delta u)||: each difference carries two roundings
        const float eta = sqrtf(e2 * (1.f + g)) * (1.f + 2.5e-7f) + 2.5e-7f * qn;
        float* fo = reinterpret_cast<float*>(out + 4 * W);
        fo[0] = lo;
        fo[1] = delta;
        fo[2] = tn2;
        fo[3] = sqrtf(tn2 * (1.f + g)) * up;
        fo[4] = eta * sqrtf((float)d) * up;
        fo[5] = qn;
        // ||q' - P t||: FP32 rounding of q' plus the FP64 products (about d^1.5 2^-53 (||q|| + ||c||))
        fo[6] = 2.384185791015625e-7f * qn + 1e-10f * (sqrtf(qq2) * up + sqrtf(ix.cnorm[l]) * up);
        reinterpret_cast<int*>(out)[4 * W + 7] = usum;
    }
}

// Bounds of the object in slot (codes in the block layout) against the
// prepared list (planes in this warp's shared memory, scalars in registers).
__device__ __forceinline__ void sign_bound(const DevIndex& ix, int64_t slot, const uint32_t* planes,
                                           const ListSetup& ls, float scale, float eps, float g_t, float& lb,
                                           float& ub, int est_mode = 0, float eps0 = 0.f, float tail = 0.f) {
    const int W = ix.d >> 5;
    const int64_t blk = slot >> 5;
    const int t = (int)(slot & 31);
    const uint32_t* cw = ix.sgn + blk * W * 32 + t;
    int s2 = 0;
#pragma unroll 6
    for (int w = 0; w < W; ++w) {
        const uint32_t c = __ldg(cw + w * 32);
        s2 += __popc(planes[w] & c) + 2 * __popc(planes[W + w] & c) + 4 * __popc(planes[2 * W + w] & c) +
              8 * __popc(planes[3 * W + w] & c);
    }
    const float4 f = __ldg(ix.sfac + slot);
    const float S1 = 2.f * f.w - (float)ix.d;
    const float S2 = (float)(2 * s2 - ls.usum);
    const float x1 = ls.lo * S1, x2 = ls.delta * S2;
    const float X = x1 + x2;
    const float eX = 2.384185791015625e-7f * (fabsf(x1) + fabsf(x2));       // 2^-22 (|x1| + |x2|)
    const float alpha = f.x, e = f.y, un2 = f.z;
    const float un = sqrtf(un2) * (1.f + 2.384185791015625e-7f);
    float est, H;
    if (est_mode && alpha > 0.f) {
        const float dd = (float)ix.d;
        const float rn2 = fmaf(e, e, dd * alpha * alpha);                   // ||r||^2
        const float kap = rn2 / (dd * alpha);
        const float rn = sqrtf(rn2) * (1.f + 2.384185791015625e-7f);
        const float spread = e / (alpha * sqrtf(dd));                         // sqrt((1 - ip^2) / ip^2)
        est = kap * X;
        H = kap * eX + tail * ls.qn * rn * spread + kap * eps0 * ls.eta + ls.dterm * un * (1.f + eps);
    } else {
        est = alpha * X;
        H = fabsf(alpha) * eX + scale * (fabsf(alpha) * ls.eta_sd + ls.qn * e) + ls.dterm * un * (1.f + eps);
    }
    const float base = ls.tn2 + un2;
    const float rotE = 2.f * eps * ls.tn * un;
    // 2^-20 relative for the FP32 evaluation here, g_t for the FP32 sum ||t||^2
    const float slack = 9.5367431640625e-7f * (base + 2.f * fabsf(est) + 2.f * H + rotE) + g_t * ls.tn2;
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

// This warp takes list j: planes into its shared slot, scalars into registers.
__device__ __forceinline__ ListSetup sign_load_list(const uint32_t* __restrict__ rec, int R, int W, uint32_t* planes) {
    for (int w = (int)lane_id(); w < 4 * W; w += 32) planes[w] = rec[w];
    const float* fo = reinterpret_cast<const float*>(rec + 4 * W);
    ListSetup ls;
    ls.lo = fo[0]; ls.delta = fo[1]; ls.tn2 = fo[2]; ls.tn = fo[3]; ls.eta_sd = fo[4]; ls.qn = fo[5]; ls.dterm = fo[6];
    ls.usum = reinterpret_cast<const int*>(rec)[4 * W + 7];
    ls.eta = ls.eta_sd / sqrtf((float)(32 * W)) * (1.f + 4.76837158203125e-7f);
    __syncwarp();
    (void)R;
    return ls;
}

// Largest key whose bucket is <= t (buckets are monotone in the bin).
__device__ __forceinline__ uint32_t sg_key_tau(const uint8_t* map, uint32_t dmin, int sh, uint32_t t) {
    const unsigned ln = lane_id();
    uint32_t c = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) c += map[ln * 8 + i] <= t ? 1u : 0u;
    c = __reduce_add_sync(0xFFFFFFFFu, c);
    if (c >= 256u) return 0xFFFFFFFFu;
    const unsigned long long v = (unsigned long long)dmin + ((unsigned long long)c << sh) - 1ull;
    return v > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)v;
}

// ---------------------------------------------------------------------------
// Scan + result buffer on the upper bounds (one CTA per query, one warp per
// list at a time).  DEBUG: write the bounds of every scanned object in probe
// order instead.
// ---------------------------------------------------------------------------
template <bool DEBUG>
__global__ void __launch_bounds__(SG_THREADS) sign_scan_kernel(DevIndex ix, SignArgs a, const uint32_t* rec) {
    extern __shared__ uint32_t spl[];                      // [warps][4W] planes, then [P + 1] prefixes (DEBUG)
    __shared__ uint32_t hist[256];
    __shared__ uint32_t sc[2];
    __shared__ uint8_t smap[256];
    __shared__ uint32_t s_cnt, s_tau, s_ktau, s_dmin, s_over;
    __shared__ int s_sh, s_ns;
    __shared__ int64_t s_sq;
    const int64_t qi = blockIdx.x;
    const int d = ix.d, W = d / 32, R = sign_rec_words(d);
    const int P = a.qp.P(qi);
    const int kq = a.qp.K(qi);
    const int m = a.m;
    const int32_t* lists = a.lists + a.qp.poff(qi);
    const uint32_t* qrec = rec + a.qp.poff(qi) * (int64_t)R;
    uint4* region = a.region + a.qp.roff(qi);
    const int64_t cap = a.qp.rcap(qi);
    const float eps = (float)(ix.eps_p * (1.0 + 1e-6)) + 1e-12f;
    const float g_t = 2.f * (float)(W + 8) * 5.9604644775390625e-8f;
    const float tail = a.eps0 / sqrtf((float)(d > 1 ? d - 1 : 1));
    const int tid = threadIdx.x, nw = blockDim.x >> 5;
    uint32_t* planes = spl + warp_id() * 4 * W;
    if (tid == 0) {
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
        s_ktau = 0xFFFFFFFFu;
        if (DEBUG) {
            int64_t* pre = reinterpret_cast<int64_t*>(spl + nw * 4 * W + (nw * 4 * W) % 2);
            int64_t b = 0;
            for (int j = 0; j < P; ++j) { pre[j] = b; b += ix.list_len[lists[j]]; }
        }
    }
    __syncthreads();
    if (DEBUG) {
        const int64_t* pre = reinterpret_cast<const int64_t*>(spl + nw * 4 * W + (nw * 4 * W) % 2);
        for (int j = warp_id(); j < P; j += nw) {
            const int l = lists[j];
            const ListSetup ls = sign_load_list(qrec + (int64_t)j * R, R, W, planes);
            const int len = ix.list_len[l];
            const int64_t b0 = ix.list_blk[l];
            for (int p = (int)lane_id(); p < len; p += 32) {
                float lb, ub;
                sign_bound(ix, b0 * 32 + p, planes, ls, a.scale, eps, g_t, lb, ub, a.est, a.eps0, tail);
                if (pre[j] + p < cap) {
                    a.dbg_lb[a.qp.roff(qi) + pre[j] + p] = lb;
                    a.dbg_ub[a.qp.roff(qi) + pre[j] + p] = ub;
                }
            }
            __syncwarp();
        }
        if (tid == 0) {
            a.scanned[qi] = s_sq;
            if (s_sq > cap) atomicOr(ix.status, kStatusRegionOverrun);
        }
        return;
    }
    // ---- sample: upper-bound keys of the first lists ----
    const int ns = s_ns;
    for (int j = warp_id(); j < ns; j += nw) {
        const int l = lists[j];
        const ListSetup ls = sign_load_list(qrec + (int64_t)j * R, R, W, planes);
        const int len = ix.list_len[l];
        const int64_t b0 = ix.list_blk[l];
        for (int b = 0; b < len; b += 32) {
            const int p = b + (int)lane_id();
            const bool valid = p < len;
            float lb = 0.f, ub = 0.f;
            if (valid) sign_bound(ix, b0 * 32 + p, planes, ls, a.scale, eps, g_t, lb, ub, a.est, a.eps0, tail);
            const uint32_t pos = sg_append(valid, &s_cnt);
            if (valid && pos < cap) region[pos] = make_uint4(0u, f32_key(ub), 0u, 0u);
        }
        __syncwarp();
    }
    __syncthreads();
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
    if (tid == 0) { s_cnt = 0; s_tau = (uint32_t)m; s_ktau = 0xFFFFFFFFu; }
    __syncthreads();
    const uint32_t dmin = s_dmin;
    const int sh = s_sh;
    // ---- main pass: histogram on the upper bound, push on the lower bound ----
    for (int j = warp_id(); j < P; j += nw) {
        const int l = lists[j];
        const ListSetup ls = sign_load_list(qrec + (int64_t)j * R, R, W, planes);
        const int len = ix.list_len[l];
        const int64_t b0 = ix.list_blk[l];
        const uint32_t ktau = *(volatile uint32_t*)&s_ktau;
        for (int b = 0; b < len; b += 32) {
            const int p = b + (int)lane_id();
            const bool valid = p < len;
            float lb = 0.f, ub = 0.f;
            if (valid) sign_bound(ix, b0 * 32 + p, planes, ls, a.scale, eps, g_t, lb, ub, a.est, a.eps0, tail);
            const uint32_t ubk = f32_key(ub), lbk = f32_key(lb);
            if (valid) atomicAdd(&hist[sg_bucket(ubk, dmin, sh, smap)], 1u);
            const bool push = valid && lbk <= ktau;         // bucket(lb) <= tau
            const uint32_t pos = sg_append(push, &s_cnt);
            if (push) {
                if (pos < cap) region[pos] = make_uint4(lbk, ubk, (uint32_t)(b0 * 32 + p), 0u);
                else s_over = 1;
            }
        }
        // Update from the shared counts (this warp), then the push threshold
        uint32_t h8[8], s = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int bk = (int)lane_id() * 8 + i;
            h8[i] = bk < m ? *(volatile uint32_t*)&hist[bk] : 0u;
            s += h8[i];
        }
        const uint32_t inc = warp_incl_scan(s);
        const unsigned hit = __ballot_sync(0xFFFFFFFFu, inc >= (uint32_t)kq);
        uint32_t t = (uint32_t)m;
        if (hit) {
            const unsigned src = __ffs(hit) - 1;
            uint32_t bk = 0;
            if (lane_id() == src) {
                uint32_t cum = inc - s;
                for (int i = 0; i < 8; ++i) {
                    cum += h8[i];
                    if (cum >= (uint32_t)kq) { bk = lane_id() * 8 + i; break; }
                }
            }
            t = __shfl_sync(0xFFFFFFFFu, bk, src);
        }
        const uint32_t kt = sg_key_tau(smap, dmin, sh, t);
        if (lane_id() == 0) { atomicMin(&s_tau, t); atomicMin(&s_ktau, kt); }
        __syncwarp();
    }
    __syncthreads();
    if (tid == 0) {
        a.pushed[qi] = min((int64_t)s_cnt, cap);
        a.scanned[qi] = s_sq;
        if (s_over) atomicOr(ix.status, kStatusRegionOverrun);
    }
}

// ---------------------------------------------------------------------------
// First round: U_k, S, the k smallest (ub, slot) of S (B) and the rest of S.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t sg_centre_key(const uint4& e) {
    return f32_key(0.5f * (key_f32(e.x) + key_f32(e.y)));
}

__global__ void __launch_bounds__(SG_THREADS) sign_select_kernel(DevIndex ix, SignSelectArgs a) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t sc[2];
    __shared__ uint32_t s_b, s_r, s_lt, s_eq, s_ns;
    const int64_t qi = blockIdx.x;
    const int64_t n = a.pushed[qi];
    const int64_t kq = a.qp.K(qi);
    const int64_t off = a.qp.coff(qi);
    const uint4* reg = a.region + a.qp.roff(qi);
    if (threadIdx.x == 0) { s_b = 0; s_r = 0; s_lt = 0; s_eq = 0; s_ns = 0; }
    __syncthreads();
    const bool all = a.scanned[qi] <= kq;                   // every scanned object is a result
    uint32_t uk = 0xFFFFFFFFu, ck = 0xFFFFFFFFu, slot_cut = 0xFFFFFFFFu;
    if (!all && n > 0) {
        // U_k, then S = {lb <= U_k} and its first round B: the ceil(f k)
        // smallest (centre, slot) of S
        const uint32_t r = (uint32_t)(min(n, kq) - 1);
        uk = cta_select_u32(n, r, [&](int64_t i) { return reg[i].y; }, hist, sc, 24);
        uint32_t ns = 0;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) ns += reg[i].x <= uk ? 1u : 0u;
        ns = __reduce_add_sync(0xFFFFFFFFu, ns);
        if (lane_id() == 0) atomicAdd(&s_ns, ns);
        __syncthreads();
        const int64_t want_b = min((int64_t)s_ns, (int64_t)ceilf(a.first * (float)kq));
        if (want_b < (int64_t)s_ns) {
            auto cen = [&](int64_t i) { const uint4 e = reg[i]; return e.x <= uk ? sg_centre_key(e) : 0xFFFFFFFFu; };
            ck = cta_select_u32(n, (uint32_t)(want_b - 1), cen, hist, sc, 24);
            uint32_t lt = 0, eq = 0;
            for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
                const uint32_t c = cen(i);
                lt += c < ck ? 1u : 0u;
                eq += c == ck ? 1u : 0u;
            }
            lt = __reduce_add_sync(0xFFFFFFFFu, lt);
            eq = __reduce_add_sync(0xFFFFFFFFu, eq);
            if (lane_id() == 0) { atomicAdd(&s_lt, lt); atomicAdd(&s_eq, eq); }
            __syncthreads();
            const uint32_t want = (uint32_t)want_b - s_lt;        // >= 1: members taken at the cut centre
            if (want < s_eq)
                slot_cut = cta_select_u32(n, want - 1, [&](int64_t i) { return cen(i) == ck ? reg[i].z : 0xFFFFFFFFu; },
                                          hist, sc, 24);
        }
    }
    const int64_t n_pad = (n + 31) / 32 * 32;
    for (int64_t i = threadIdx.x; i < n_pad; i += blockDim.x) {
        bool inb = false, inr = false;
        uint4 e = make_uint4(0, 0, 0, 0);
        if (i < n) {
            e = reg[i];
            const bool ins = all || e.x <= uk;
            const uint32_t c = ins ? sg_centre_key(e) : 0xFFFFFFFFu;
            inb = all || (ins && (c < ck || (c == ck && e.z <= slot_cut)));
            inr = !inb && ins;
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

// Second round: U' = the k-th smallest FP32 upper bound of the distances in
// B (the largest when B holds at most k); S' = rest with lb <= U'.
__global__ void __launch_bounds__(SG_THREADS) sign_filter_kernel(DevIndex ix, SignSelectArgs a) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t sc[2];
    __shared__ uint32_t s_c;
    const int64_t qi = blockIdx.x;
    const int64_t nb = a.n_b[qi];
    const int64_t nr = a.n_rest[qi];
    const int64_t kq = a.qp.K(qi);
    const int64_t off = a.qp.coff(qi);
    if (threadIdx.x == 0) s_c = 0u;
    __syncthreads();
    uint32_t up = 0u;
    if (nb > 0) {
        const uint32_t r = (uint32_t)(min(nb, kq) - 1);
        up = cta_select_u32(nb, r, [&](int64_t i) { return f32_key(__fadd_ru(a.cd[off + i], a.cr[off + i])); },
                            hist, sc, 24);
    }
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

size_t sign_prep_bytes(const DevIndex& ix, int64_t sum_probe) {
    return (size_t)sum_probe * (size_t)sign_rec_words(ix.d) * 4;
}

cudaError_t launch_sign_scan(const DevIndex& ix, int64_t nq, const SignArgs& a, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    if (ix.d % 32 || ix.d > 32 * SG_MAXW || !a.prep) return cudaErrorInvalidValue;
    const int wpb = 8;
    dim3 pg((unsigned)((a.nprobe + wpb - 1) / wpb), (unsigned)nq);
    sign_prep_kernel<<<pg, 32 * wpb, 0, st>>>(ix, a, a.prep);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nw = SG_THREADS / 32;
    size_t smem = (size_t)nw * 4 * (ix.d / 32) * 4 + 8;
    if (a.dbg_lb) smem += (size_t)(a.nprobe + 1) * 8;
    e = smem_attr_once((const void*)sign_scan_kernel<true>, 64 * 1024);
    if (e == cudaSuccess) e = smem_attr_once((const void*)sign_scan_kernel<false>, 64 * 1024);
    if (e != cudaSuccess) return e;
    if (smem > 64 * 1024) return cudaErrorInvalidValue;
    if (a.dbg_lb) sign_scan_kernel<true><<<(unsigned)nq, SG_THREADS, smem, st>>>(ix, a, a.prep);
    else sign_scan_kernel<false><<<(unsigned)nq, SG_THREADS, smem, st>>>(ix, a, a.prep);
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
