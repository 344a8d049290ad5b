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
    st->q_lo = 0;
    st->q_hi = 0;
    st->J = 0.0;
    st->shift = 0.0;
    st->Qtot = 0.0;
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
    int lg = 0;
    while ((1 << lg) < d) ++lg;
    int F = min(120, max(-100, 46 - E));
    int G = min(120, max(-100, 62 - 2 * E - 16 - lg));
    st->F = F;
    st->G = G;
    st->scaleF = ldexpf(1.0f, F);
    st->scaleG = ldexpf(1.0f, G);
    st->inv_scaleF = ldexp(1.0, -F);
    st->inv_scaleG = ldexp(1.0, -G);
}

// One warp: the new center j (its cluster mean; an empty cluster keeps its
// center) with its FP32 copies and ||c_j||^2, and center j's terms of the
// movement, of J and of the empty count in clus (4 k doubles).  Iteration it's
// records of center j go to tr.centers / tr.counts when those are set.
static __device__ __forceinline__ void finalize_center_warp(const Accum& acc, const Centers& c,
                                                            double inv, int j, double* clus,
                                                            const TrajDev& tr, int it)
{
    const int k = c.k, d = c.d;
    const int lane = threadIdx.x & 31;
    long long N = (long long)acc.cnt[j];
    double diff2 = 0.0, cS = 0.0, cc = 0.0, nn = 0.0;
    for (int t = lane; t < d; t += 32) {
        long long e = (long long)j * d + t;
        const unsigned long long lo = acc.s_lo[e], hi = acc.s_hi[e];
        double S = split_value(lo, hi, inv);
        // carry the low word's upper half into the high word (same value):
        // every pass adds at most 2 n < 2^32 low parts below 2^32 each, so
        // the low word cannot wrap however many delta passes follow
        acc.s_lo[e] = lo & 0xffffffffull;
        acc.s_hi[e] = hi + (lo >> 32);
        double cv = c.c64[e];
        double cn = N > 0 ? S / (double)N : cv;
        double df = cn - cv;
        diff2 = fma(df, df, diff2);
        cS = fma(cv, S, cS);
        cc = fma(cv, cv, cc);
        nn = fma(cn, cn, nn);
        c.c64[e] = cn;
        c.c32[e] = (float)cn;
        c.c32t[(long long)t * c.kpad + j] = (float)cn;
        if (tr.centers) tr.centers[(long long)it * k * d + e] = cn;
    }
    diff2 = warp_sum_f64(diff2);
    cS = warp_sum_f64(cS);
    cc = warp_sum_f64(cc);
    nn = warp_sum_f64(nn);
    if (lane == 0) {
        clus[j] = diff2;
        clus[k + j] = 2.0 * cS - (double)N * cc;
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
    double Qtot;
};

// Whole block (blockDim.x <= 1024, a power of two), after every center's
// finalize_center_warp: movement, J and loop control from clus, in a fixed
// order (thread 0 updates st).  Ends with the block synchronised.
static __device__ void finalize_reduce_block(int k, StageState* st, const TrajDev& tr,
                                             const double* clus, FinalizeSmem& sm)
{
    double* traj_J = tr.J;
    double* traj_shift = tr.shift;
    if (threadIdx.x == 0) {
        double Q = st->Qtot;
        if (st->mode == kModeFull) {
            Q = split_value(st->q_lo, st->q_hi, st->inv_scaleG);
            st->Qtot = Q;
        }
        sm.Qtot = Q;
    }
    double sh = 0.0, jj = 0.0, mx = 0.0;
    int em = 0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        sh = fmax(sh, clus[j]);
        jj += clus[k + j];
        mx = fmax(mx, clus[2 * k + j]);
        em += (int)clus[3 * k + j];
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
        double J = sm.Qtot - sm.r_J[0];
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

// One warp per listed point.  Pass 1: FP32 D_j for every center on the CUDA
// cores (recheck_d4) and their minimum b1.  Pass 2: every center with
// D_j <= b1 + tie_kappa (2 C2 + X2) -- a set that provably holds the FP64
// argmin -- is evaluated exactly in the oracle's form (sum_t fma(x_t - c_t,
// x_t - c_t, acc), t ascending) and the smallest wins, lowest index on ties.
// cache: per-warp shared memory of cache_cap floats for the pass-1 values
// (pass 2 recomputes them when kpad > cache_cap or cache is null).
// Warps w0, w0 + wstride, ... of the caller each take the listed points.
static __device__ void recheck_warps(const float* __restrict__ X, int d, Centers c,
                                     int* __restrict__ labels, const int* __restrict__ list,
                                     StageState* st, Accum acc, long long gw, long long nw,
                                     float* cache, int cache_cap)
{
    const int count = st->recheck_count;
    const int mode = st->mode;
    const float scaleF = st->scaleF;
    const float c2x2 = 2.0f * st->cmax2;
    const float kap = tie_kappa(d);
    const int k = c.k;
    const bool cached = cache != nullptr && c.kpad <= cache_cap;
    int lane = threadIdx.x & 31;
    for (long long w = gw; w < count; w += nw) {
        int i = list[w];
        const float* x = X + (long long)i * d;
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
        const float lim = b1 + kap * (c2x2 + x2) * 1.0009765625f;
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
        for (int o = 16; o; o >>= 1) {
            double ob = __shfl_xor_sync(0xffffffffu, best, o);
            int oj = __shfl_xor_sync(0xffffffffu, bj, o);
            if (ob < best || (ob == best && oj < bj)) { best = ob; bj = oj; }
        }
        int old = (mode == kModeDelta) ? labels[i] : -1;
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
}


}  // namespace km2
