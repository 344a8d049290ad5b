// stage_dev.cuh -- block- and warp-level bodies of the per-stage steps, shared
// by the single-fit kernels (prep.cu) and the batched kernels (batched.cu) so
// that both run exactly the same arithmetic:
//   center_prep_block  FP32 / transposed copies of the FP64 centers, ||c||^2
//   stage_init_dev     fixed-point scales and loop state of one stage
//   finalize_block     new centers = cluster means (Lloyd's method, Section 4.1),
//                      largest movement (stop test, Sections 5-6), J (Eq. 3)
//   recheck_warps      FP64 re-evaluation of near-tie points (ties -> lowest index)
#pragma once

#include <cfloat>
#include <climits>

#include "common.cuh"

namespace km2 {

__device__ __forceinline__ double warp_sum_f64(double v)
{
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// FP32 copies and ||c_j||^2 of every center; st->cmax2 = max_j ||c_j||^2 rounded
// up.  Whole block; warps stride over centers; fixed reduction order.
// red: blockDim.x doubles of shared memory.
static __device__ void center_prep_block(Centers c, StageState* st, double* red)
{
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double mx = 0.0;
    for (int j = warp; j < c.k; j += nw) {
        double nn = 0.0;
        for (int t = lane; t < c.d; t += 32) {
            double v = c.c64[(long long)j * c.d + t];
            nn = fma(v, v, nn);
            c.c32[(long long)j * c.d + t] = (float)v;
            c.c32t[(long long)t * c.kpad + j] = (float)v;
        }
        nn = warp_sum_f64(nn);
        if (lane == 0) c.cnorm[j] = (float)nn;
        mx = fmax(mx, nn);
    }
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int s = blockDim.x >> 1; s; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) st->cmax2 = __double2float_ru(red[0]);
    __syncthreads();
}

// One thread.  Loop state of a new stage and its fixed-point scales from
// st->maxabs_bits (max |x| of the stage's points).
static __device__ void stage_init_dev(StageState* st, int d, double tol, int max_iter)
{
    unsigned int b = st->maxabs_bits;
    st->mode = kModeFull;
    st->iter = 0;
    st->done = 0;
    st->converged = 0;
    st->max_iter = max_iter;
    st->tol = tol;
    st->recheck_count = 0;
    st->rechecked_total = 0;
    st->undecided16_total = 0;
    for (int w = 0; w < 4; ++w) st->q[w] = 0ull;
    st->J = 0.0;
    st->shift = 0.0;
    st->empty = 0;
    st->error = 0;
    if (b >= 0x7f800000u) {
        st->error = kErrNonFinite;
        st->done = 1;
        return;
    }
    float mx = __uint_as_float(b);
    int E = -126;
    if (mx > 0.0f) frexpf(mx, &E);          // mx < 2^E
    if (E > 50) {
        st->error = kErrRange;
        st->done = 1;
        return;
    }
    (void)d;
    int F = min(120, max(-100, 46 - E));
    st->F = F;
    st->scaleF = ldexpf(1.0f, F);
    st->inv_scaleF = ldexp(1.0, -F);
}

// ---------------------------------------------------------------- exact J
// Error-free transformations (Knuth's TwoSum, Dekker's FastTwoSum, and the
// FMA two-product) for the center-displacement term of J.
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e)
{
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(double a, double b, double& s, double& e)
{
    s = a + b;
    e = b - (s - a);
}

// N c - s 2^-F for a center coordinate c (FP64), a cluster size N and the
// exact integer sum s of the cluster's fixed-point coordinates: N times the
// center's displacement from the cluster mean.  c N is split exactly into the
// double-word p + e (FMA two-product) and s 2^-F exactly into a1 + a2 (the
// 32-bit halves of s, scaled by powers of two), renormalised by TwoSum into
// the double-word b1 + b2; the two double-words are then added with the
// accurate double-word sum (two TwoSums, two renormalisations), whose relative
// error is below 3 * 2^-106 of the result however close c is to the mean.
__device__ __forceinline__ double displacement(double c, double N, __int128 s, double inv)
{
    const __int128 sh = s >> 32;                       // |sh| < 2^50: exact in FP64
    const double a1 = (double)(long long)sh * (inv * 4294967296.0);
    const double a2 = (double)(unsigned long long)(s - (sh << 32)) * inv;
    double b1, b2;
    two_sum(a1, a2, b1, b2);
    const double p = c * N;
    const double e = fma(c, N, -p);
    double s1, s2, t1, t2;
    two_sum(p, -b1, s1, s2);
    two_sum(e, -b2, t1, t2);
    s2 += t1;
    fast_two_sum(s1, s2, s1, s2);
    s2 += t2;
    fast_two_sum(s1, s2, s1, s2);
    return s1;
}

// 256-bit two's complement integers for the integer part of J.
struct U256 {
    unsigned long long w[4];
};

// a += v * 2^(64 limb), carries propagated to the top limb.
__device__ __forceinline__ void u256_add_at(U256& a, unsigned __int128 v, int limb)
{
    unsigned long long carry = 0;
    for (int i = limb; i < 4; ++i) {
        const unsigned long long add = (i == limb) ? (unsigned long long)v
                                     : (i == limb + 1) ? (unsigned long long)(v >> 64) : 0ull;
        const unsigned __int128 t = (unsigned __int128)a.w[i] + add + carry;
        a.w[i] = (unsigned long long)t;
        carry = (unsigned long long)(t >> 64);
    }
}

__device__ __forceinline__ void u256_neg(U256& a)
{
    unsigned long long carry = 1;
    for (int i = 0; i < 4; ++i) {
        const unsigned __int128 t = (unsigned __int128)(~a.w[i]) + carry;
        a.w[i] = (unsigned long long)t;
        carry = (unsigned long long)(t >> 64);
    }
}

// The signed value of a, rounded to FP64 (the top 128 significant bits are
// converted in one rounding; the rest is below 2^-64 of it).
__device__ __forceinline__ double u256_to_double(U256 a)
{
    const bool neg = (long long)a.w[3] < 0;
    if (neg) u256_neg(a);
    int top = 3;
    while (top > 0 && a.w[top] == 0) --top;
    double r;
    if (top == 0) {
        r = (double)a.w[0];
    } else {
        const unsigned __int128 hi = ((unsigned __int128)a.w[top] << 64) | a.w[top - 1];
        r = ldexp((double)hi, 64 * (top - 1));
        if (top >= 2) r += ldexp((double)a.w[top - 2], 64 * (top - 2));
    }
    return neg ? -r : r;
}

// One warp: the new center j (its cluster mean; an empty cluster keeps its
// center) with its FP32 copies and ||c_j||^2, and center j's terms of the
// movement, of J and of the empty count in clus (kClusSlots k doubles):
//   clus[j]          ||c_j' - c_j||^2
//   clus[k + j]      N_j ||c_j - mu_j||^2 - frac(T_j / N_j) 2^-2F
//   clus[2k + j]     ||c_j'||^2
//   clus[3k + j]     1 if the cluster is empty
//   clus[4k + 3j..]  floor(T_j / N_j) as three 64-bit limbs
// where s_jt = the exact integer sum of the cluster's fixed-point coordinates,
// mu_j = s_j 2^-F / N_j its mean and T_j = ||s_j||^2, so that over all clusters
// J = (sum s^2 - sum_j T_j / N_j) 2^-2F + sum_j N_j ||c_j - mu_j||^2
//   = sum_j sum_{i in j} ||x_i - c_j||^2   (Eq. 3, on the fixed-point values).
// Iteration it's records of center j go to tr.centers / tr.counts when those are set.
static __device__ __forceinline__ void finalize_center_warp(const Accum& acc, const Centers& c,
                                                            double inv, int j, double* clus,
                                                            const TrajDev& tr, int it)
{
    const int k = c.k, d = c.d;
    const int lane = threadIdx.x & 31;
    const long long N = (long long)acc.cnt[j];
    const double Nd = (double)N;
    double diff2 = 0.0, dev2 = 0.0, nn = 0.0;
    // T_j = t_hi 2^64 + t_lo, partial per lane (no carries needed: t_lo gains
    // < 2^65 per coordinate, t_hi < 2^101)
    unsigned __int128 t_lo = 0, t_hi = 0;
    for (int t = lane; t < d; t += 32) {
        long long e = (long long)j * d + t;
        const unsigned long long lo = acc.s_lo[e], hi = acc.s_hi[e];
        const __int128 v = (__int128)(long long)hi * (__int128)4294967296LL + (__int128)lo;
        double S = (double)v * inv;
        // carry the low word's upper half into the high word (same value):
        // every pass adds at most 2 n < 2^32 low parts below 2^32 each, so
        // the low word cannot wrap however many delta passes follow
        acc.s_lo[e] = lo & 0xffffffffull;
        acc.s_hi[e] = hi + (lo >> 32);
        double cv = c.c64[e];
        double cn = N > 0 ? S / Nd : cv;
        double df = cn - cv;
        diff2 = fma(df, df, diff2);
        nn = fma(cn, cn, nn);
        if (N > 0) {
            const unsigned __int128 a = (unsigned __int128)(v < 0 ? -v : v);   // < 2^82
            const unsigned long long al = (unsigned long long)a & 0xffffffffull;
            const unsigned __int128 ah = a >> 32;
            const unsigned __int128 m = 2 * ah * al;
            t_hi += ah * ah + (m >> 32);
            t_lo += ((m & 0xffffffffull) << 32) + (unsigned __int128)al * al;
            const double r = displacement(cv, Nd, v, inv);
            dev2 = fma(r, r, dev2);
        }
        c.c64[e] = cn;
        c.c32[e] = (float)cn;
        c.c32t[(long long)t * c.kpad + j] = (float)cn;
        if (tr.centers) tr.centers[(long long)it * k * d + e] = cn;
    }
    diff2 = warp_sum_f64(diff2);
    dev2 = warp_sum_f64(dev2);
    nn = warp_sum_f64(nn);
    t_lo = warp_sum_u128(t_lo);
    t_hi = warp_sum_u128(t_hi);
    if (lane == 0) {
        unsigned long long* qw = reinterpret_cast<unsigned long long*>(clus + 4 * k) + 3ll * j;
        double v = 0.0;
        unsigned __int128 q_hi = 0;
        unsigned long long q_lo = 0;
        if (N > 0) {
            // floor(T / N) and T mod N by long division (N < 2^63)
            t_hi += t_lo >> 64;
            const unsigned long long un = (unsigned long long)N;
            q_hi = t_hi / un;
            const unsigned __int128 x = ((t_hi % un) << 64) | (unsigned long long)t_lo;
            q_lo = (unsigned long long)(x / un);
            const unsigned long long rem = (unsigned long long)(x % un);
            v = dev2 / Nd - ((double)rem / Nd) * (inv * inv);
        }
        qw[0] = q_lo;
        qw[1] = (unsigned long long)q_hi;
        qw[2] = (unsigned long long)(q_hi >> 64);
        clus[j] = diff2;
        clus[k + j] = v;
        clus[2 * k + j] = nn;
        clus[3 * k + j] = (N == 0) ? 1.0 : 0.0;
        c.cnorm[j] = (float)nn;
        if (tr.counts) tr.counts[(long long)it * k + j] = N;
    }
}

struct FinalizeSmem {
    double r_shift[1024];
    double r_J[1024];
    double r_nn[1024];
    int r_empty[1024];
    unsigned __int128 r_q[32][3];
};

// Whole block (blockDim.x <= 1024, a power of two), after every center's
// finalize_center_warp: movement, J and loop control from clus, in a fixed
// order (thread 0 updates st).  The integer part of J, sum s^2 - sum_j
// floor(T_j / N_j), is exact (256-bit); it is rounded to FP64 once and added
// to the sum of the per-center remainders.  Ends with the block synchronised.
static __device__ void finalize_reduce_block(int k, StageState* st, const TrajDev& tr,
                                             const double* clus, FinalizeSmem& sm)
{
    double* traj_J = tr.J;
    double* traj_shift = tr.shift;
    const unsigned long long* qw = reinterpret_cast<const unsigned long long*>(clus + 4 * k);
    double sh = 0.0, jj = 0.0, mx = 0.0;
    int em = 0;
    unsigned __int128 a0 = 0, a1 = 0, a2 = 0;    // sums of the limbs of floor(T_j / N_j)
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        sh = fmax(sh, clus[j]);
        jj += clus[k + j];
        mx = fmax(mx, clus[2 * k + j]);
        em += (int)clus[3 * k + j];
        a0 += qw[3ll * j];
        a1 += qw[3ll * j + 1];
        a2 += qw[3ll * j + 2];
    }
    a0 = warp_sum_u128(a0);
    a1 = warp_sum_u128(a1);
    a2 = warp_sum_u128(a2);
    if ((threadIdx.x & 31) == 0) {
        sm.r_q[threadIdx.x >> 5][0] = a0;
        sm.r_q[threadIdx.x >> 5][1] = a1;
        sm.r_q[threadIdx.x >> 5][2] = a2;
    }
    sm.r_shift[threadIdx.x] = sh;
    sm.r_J[threadIdx.x] = jj;
    sm.r_nn[threadIdx.x] = mx;
    sm.r_empty[threadIdx.x] = em;
    __syncthreads();
    for (int s = blockDim.x >> 1; s; s >>= 1) {
        if ((int)threadIdx.x < s) {
            sm.r_shift[threadIdx.x] = fmax(sm.r_shift[threadIdx.x], sm.r_shift[threadIdx.x + s]);
            sm.r_J[threadIdx.x] += sm.r_J[threadIdx.x + s];
            sm.r_nn[threadIdx.x] = fmax(sm.r_nn[threadIdx.x], sm.r_nn[threadIdx.x + s]);
            sm.r_empty[threadIdx.x] += sm.r_empty[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // D = sum s^2 - sum_j floor(T_j / N_j)  (>= 0: Cauchy-Schwarz per cluster)
        U256 D = {{0ull, 0ull, 0ull, 0ull}};
        U256 Tq = {{0ull, 0ull, 0ull, 0ull}};
        u256_add_at(D, (unsigned __int128)st->q[0], 0);
        u256_add_at(D, (unsigned __int128)st->q[1] << 32, 0);
        u256_add_at(D, (unsigned __int128)st->q[2], 1);
        u256_add_at(D, (unsigned __int128)st->q[3] << 32, 1);
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            u256_add_at(Tq, sm.r_q[w][0], 0);
            u256_add_at(Tq, sm.r_q[w][1], 1);
            u256_add_at(Tq, sm.r_q[w][2], 2);
        }
        u256_neg(Tq);
        for (int i = 0; i < 4; ++i) u256_add_at(D, (unsigned __int128)Tq.w[i], i);
        const double inv = st->inv_scaleF;
        double J = u256_to_double(D) * (inv * inv) + sm.r_J[0];
        if (J < 0.0) J = 0.0;   // only rounding of an exactly zero objective can go below
        double shift = sqrt(sm.r_shift[0]);
        int it = st->iter;
        if (traj_J) traj_J[it] = J;
        if (traj_shift) traj_shift[it] = shift;
        st->J = J;
        st->shift = shift;
        st->empty = sm.r_empty[0];
        st->cmax2 = __double2float_ru(sm.r_nn[0]);
        st->iter = it + 1;
        int conv = shift <= st->tol;
        st->converged = conv;
        st->done = conv || (it + 1 >= st->max_iter);
        st->mode = kModeDelta;
        st->rechecked_total += st->recheck_count;
        st->recheck_count = 0;
    }
    __syncthreads();
}

// Whole block (blockDim.x <= 1024, a power of two).  New centers, movement,
// J; loop control for the next iteration (thread 0 updates st).  clus: 4 k
// doubles of scratch.  Ends with the block synchronised.
static __device__ void finalize_block(Accum acc, Centers c, StageState* st, TrajDev tr,
                                      double* clus, FinalizeSmem& sm)
{
    const double inv = st->inv_scaleF;
    const int it = st->iter;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = warp; j < c.k; j += nw) finalize_center_warp(acc, c, inv, j, clus, tr, it);
    __syncthreads();
    finalize_reduce_block(c.k, st, tr, clus, sm);
}

// FP32 D_j = ||c_j||^2 - 2 x.c_j of one point against centers j0 + 32 i
// (i < 4): the CUDA-core FMA chain whose error tie_kappa bounds, t ascending.
// c32t (dims x kpad, coalesced across the warp's lanes) holds the same FP32
// values as the row-major copy; fmaf(-2 x_t, c_t, a) equals fmaf(x_t, -2 c_t, a)
// (scaling by -2 is exact).  Padding centers read zeros.
static __device__ __forceinline__ void recheck_d4(const float* __restrict__ x, int d,
                                                  const Centers& c, int j0, float a[4])
{
    const int kpad = c.kpad;
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = c.cnorm[j0 + 32 * i];
    const float* ct = c.c32t + j0;
    for (int t = 0; t < d; ++t) {
        const float xm2 = -2.0f * __ldg(x + t);
        const float* row = ct + (long long)t * kpad;
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = fmaf(xm2, row[32 * i], a[i]);
    }
}

// One warp: re-decide point i.  Pass 1: FP32 D_j for every center on the CUDA
// cores (recheck_d4) and their minimum b1.  Pass 2: every center with
// D_j <= b1 + tie_kappa (2 C2 + X2) + tie_abs -- a set that provably holds the FP64
// argmin -- is evaluated exactly in the oracle's form (sum_t fma(x_t - c_t,
// x_t - c_t, acc), t ascending) and the smallest wins, lowest index on ties.
// The point's new label and the sums follow (delta mode: from its old label).
// cache: per-warp shared memory of cache_cap floats for the pass-1 values
// (pass 2 recomputes them when kpad > cache_cap or cache is null).
static __device__ __forceinline__ void recheck_point(const float* __restrict__ X, int d,
                                                     const Centers& c, int* __restrict__ labels,
                                                     int i, StageState* st, const Accum& acc,
                                                     float* cache, int cache_cap)
{
    const int mode = st->mode;
    const float scaleF = st->scaleF;
    const float c2x2 = 2.0f * st->cmax2;
    const float kap = tie_kappa(d);
    const int k = c.k;
    const bool cached = cache != nullptr && c.kpad <= cache_cap;
    const int lane = threadIdx.x & 31;
    const float* x = X + (long long)i * d;
    // the old label's load (a random row of the labels) overlaps the passes
    const int old = (mode == kModeDelta) ? labels[i] : -1;
    float x2 = 0.0f;
    for (int t = lane; t < d; t += 32) { float v = __ldg(x + t); x2 = fmaf(v, v, x2); }
    for (int o = 16; o; o >>= 1) x2 += __shfl_xor_sync(0xffffffffu, x2, o);
    float b1 = INFINITY;
    for (int j0 = lane; j0 < k; j0 += 128) {
        float a[4];
        recheck_d4(x, d, c, j0, a);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (j0 + 32 * q < k) b1 = fminf(b1, a[q]);
            if (cached) cache[j0 + 32 * q] = a[q];
        }
    }
    for (int o = 16; o; o >>= 1) b1 = fminf(b1, __shfl_xor_sync(0xffffffffu, b1, o));
    const float lim = b1 + kap * (c2x2 + x2) * 1.0009765625f + tie_abs(d + 1);
    double best = DBL_MAX;
    int bj = INT_MAX;
    for (int j0 = lane; j0 < k; j0 += 128) {
        float a[4];
        if (cached) {
#pragma unroll
            for (int q = 0; q < 4; ++q) a[q] = cache[j0 + 32 * q];
        } else {
            recheck_d4(x, d, c, j0, a);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = j0 + 32 * q;
            if (j < k && a[q] <= lim) {
                const double* cj64 = c.c64 + (long long)j * d;
                double a2 = 0.0;
                for (int t = 0; t < d; ++t) {
                    double e = (double)__ldg(x + t) - cj64[t];
                    a2 = fma(e, e, a2);
                }
                if (a2 < best || (a2 == best && j < bj)) { best = a2; bj = j; }
            }
        }
    }
    // lowest (distance, index) over the lanes; the FP64 sums of squares are
    // non-negative, so their bit patterns order as the values do and the
    // comparison stays off the (narrow) FP64 pipe
    unsigned long long bb = (unsigned long long)__double_as_longlong(best);
    for (int o = 16; o; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, bb, o);
        const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
        if (ob < bb || (ob == bb && oj < bj)) { bb = ob; bj = oj; }
    }
    __syncwarp();   // every lane has read the old label before lane 0 rewrites it
    if (bj != old && label_ok(bj, k, st) && old_label_ok(old, k, st)) {
        for (int t = lane; t < d; t += 32) {
            long long v = to_fixed(__ldg(x + t), scaleF);
            split_add(acc.s_lo + (long long)bj * d + t, acc.s_hi + (long long)bj * d + t, v);
            if (old >= 0)
                split_add(acc.s_lo + (long long)old * d + t, acc.s_hi + (long long)old * d + t, -v);
        }
        if (lane == 0) {
            atomicAdd(acc.cnt + bj, 1ull);
            if (old >= 0) atomicAdd(acc.cnt + old, ~0ull);
            labels[i] = bj;
        }
    }
}

// One warp per listed point (recheck_point); warps w0, w0 + wstride, ... of
// the caller each take the listed points.
static __device__ void recheck_warps(const float* __restrict__ X, int d, Centers c,
                                     int* __restrict__ labels, const int* __restrict__ list,
                                     StageState* st, Accum acc, long long gw, long long nw,
                                     float* cache, int cache_cap)
{
    const int count = st->recheck_count;
    for (long long w = gw; w < count; w += nw)
        recheck_point(X, d, c, labels, list[w], st, acc, cache, cache_cap);
}


}  // namespace km2
