// assign_fp32.cu -- fused distance + nearest-center + cluster-sum kernels, FP32 on
// the CUDA cores (the hot loop of the Algorithm: the squared distance of each
// point to each center, the smallest one, and the point's new cluster; the sums
// feed the mean step of Lloyd's method, Section 4.1).
//
// The argmin needs only D_j = ||c_j||^2 - 2 x.c_j (||x||^2 is common to all
// centers).  Each kernel keeps the best and second-best D per point; when the
// gap between them is below the rounding-error bound (tie_kappa) the point is
// appended to a recheck list and decided in FP64 by recheck_kernel; otherwise
// the FP32 argmin is provably the FP64 argmin.
//
// Cluster sums are exact fixed-point integers (common.cuh).  In the first
// iteration of a stage (kModeFull) every point adds its coordinates; in later
// iterations (kModeDelta) only a point whose label changed moves its
// coordinates from the old cluster to the new one.  Integer sums make this
// incremental update exact, so later Lloyd iterations cost almost nothing
// beyond the distances.
//
// Two forms:
//  assign_small<D>     d <= 16.  Each thread owns P points (2 or 4) in registers and
//                      prefetches its next tile with cp.async; the k centers
//                      (pre-scaled by -2, with ||c||^2) sit in shared memory,
//                      interleaved in pairs and read as broadcast 128-bit
//                      loads; one packed FP32x2 FMA (fma.rn.f32x2, each half
//                      rounded like its own fmaf) advances both centers of a
//                      pair, halving the FMA instructions; the top-2 runs on
//                      packed keys (index in the low mantissa bits).  Per-CTA int64 partial sums in shared memory,
//                      flushed to the global split accumulators every 2^16 points.
//  assign_large        any d.  128 points x 128 centers register-blocked tiles
//                      (8 x 8 per thread) over 8-dimension slices staged in
//                      shared memory; per-thread top-2 merged across the 16
//                      threads of a half-warp with shuffles.  Sums go to the
//                      global accumulators directly.
#include <cfloat>
#include <cstdint>

#include "api_internal.h"

namespace km2 {

namespace {

constexpr int kThreads = 256;
constexpr int kSmallSmemCap = 200 * 1024;   // dynamic shared memory of assign_small, at most

__device__ __forceinline__ void top2_push(float v, int j, float& b1, float& b2, int& bi)
{
    if (v < b1) {
        b2 = b1;
        b1 = v;
        bi = j;
    } else {
        b2 = fminf(b2, v);
    }
}

// Merge another (best, second, index) triple; symmetric, lowest index on equal bests.
__device__ __forceinline__ void top2_merge(float& b1, float& b2, int& bi, float o1, float o2,
                                           int oi)
{
    if (o1 < b1 || (o1 == b1 && oi < bi)) {
        b2 = fminf(b1, o2);
        b1 = o1;
        bi = oi;
    } else {
        b2 = fminf(b2, o1);
    }
}

// Points per thread and resident CTAs per SM, measured on GB300 (n = 1e8,
// k = 32, d = 2 / 4 / 8; n = 5e7, k = 64, d = 16; best of P = 1..4 with 2-4
// CTAs per SM): 4 points at 2 CTAs up to d = 4, 2 points at 4 CTAs (62
// registers) for d = 5..8 (+7 % at d = 8), 4 points at 2 CTAs from d = 9 on
// (+8 % at d = 16 over 2 points).
template <int D>
struct SmallCfg {
    static constexpr int DS = (D + 3) & ~3;       // floats per center (-2c) in shared memory
    static constexpr int P = (D > 4 && D <= 8) ? 2 : 4;   // points per thread
    static constexpr int MINB = (D > 4 && D <= 8) ? 4 : 2;  // resident CTAs per SM
    static constexpr int V = (D % 4 == 0) ? 4 : ((D % 2 == 0) ? 2 : 1);   // copy width (floats)
    static constexpr int NV = D / V;              // copies per point
    static constexpr int TILE = kThreads * P;     // points per tile
    static constexpr int FLUSH_TILES = kFlushPoints / TILE;
};

// Packed key: the float v with its 5 low mantissa bits replaced by j (0..31).
// Compared as floats, keys order like the values up to 2^-18 |v|; which of two
// near-equal keys wins does not matter, since such points are rechecked.
__device__ __forceinline__ float pack_key(float v, unsigned j)
{
    return __uint_as_float((__float_as_uint(v) & ~31u) | j);
}

template <int D>
__device__ __forceinline__ void copy_point_async(float* sx, const float* src, int p, int tid)
{
    using C = SmallCfg<D>;
#pragma unroll
    for (int q = 0; q < C::NV; ++q) {
        float* dst = sx + ((size_t)(p * C::NV + q) * kThreads + tid) * C::V;
        if constexpr (C::V == 4) cp_async16(dst, src + 4 * q);
        else if constexpr (C::V == 2) cp_async8(dst, src + 2 * q);
        else cp_async4(dst, src + q);
    }
}

template <int D>
__device__ __forceinline__ void read_point(const float* sx, int p, int tid, float* x)
{
    using C = SmallCfg<D>;
#pragma unroll
    for (int q = 0; q < C::NV; ++q) {
        const float* src = sx + ((size_t)(p * C::NV + q) * kThreads + tid) * C::V;
        if constexpr (C::V == 4) {
            float4 v = *reinterpret_cast<const float4*>(src);
            x[4 * q] = v.x; x[4 * q + 1] = v.y; x[4 * q + 2] = v.z; x[4 * q + 3] = v.w;
        } else if constexpr (C::V == 2) {
            float2 v = *reinterpret_cast<const float2*>(src);
            x[2 * q] = v.x; x[2 * q + 1] = v.y;
        } else {
            x[q] = src[0];
        }
    }
}

// Points are owned by threads (tile point p * 256 + tid); each thread prefetches
// its own next-tile points (and old labels) with cp.async into its own shared
// slots while it computes the current tile, so no thread waits on another.
// Centers are walked in chunks of 32 and in pairs; the running top-2 of packed
// keys costs 2.5 min/max operations per distance (3-input min).
template <int D>
__global__ void __launch_bounds__(kThreads, SmallCfg<D>::MINB)
assign_small(const float* __restrict__ X, long long n, Centers c, int* __restrict__ labels,
             StageState* st, Accum acc, int* __restrict__ list, float kappa, float kpack,
             int use_sacc)
{
    using C = SmallCfg<D>;
    constexpr int DS = C::DS;
    constexpr int P = C::P;
    extern __shared__ __align__(16) float smem[];
    const int k = c.k;
    const int kc = (k + 31) & ~31;
    const int nchunks = kc >> 5;
    float* sc = smem;                                          // kc * DS: -2 c_j
    float* ss = sc + (size_t)kc * DS;                          // kc: ||c_j||^2
    float* sx = ss + kc;                                       // TILE * D (thread-major)
    int* sl = reinterpret_cast<int*>(sx + (size_t)C::TILE * D);  // TILE old labels
    long long* sacc = reinterpret_cast<long long*>(sl + C::TILE);  // k * D (if use_sacc)
    int* scnt = reinterpret_cast<int*>(sacc + (size_t)k * D);       // k (if use_sacc)

    if (st->error) return;
    const int mode = st->mode;
    const float scaleF = st->scaleF;
    const float thr_base = 2.0f * st->cmax2;
    const int tid = threadIdx.x;

    for (int e = tid; e < kc * DS; e += kThreads) {
        // center pairs interleaved: (pair, t, member)
        const int pr = e / (2 * DS), r = e - pr * 2 * DS;
        const int t = r >> 1, j = 2 * pr + (r & 1);
        sc[e] = (j < k && t < D) ? -2.0f * c.c32[(long long)j * D + t] : 0.0f;
    }
    for (int j = tid; j < kc; j += kThreads)
        ss[j] = (j < k) ? c.cnorm[j] : FLT_MAX;   // padding center: never the best
    if (use_sacc) {
        for (int e = tid; e < k * D; e += kThreads) sacc[e] = 0;
        for (int e = tid; e < k; e += kThreads) scnt[e] = 0;
    }
    __syncthreads();

    const long long ntiles = (n + C::TILE - 1) / C::TILE;
    auto prefetch = [&](long long tile, unsigned dep) {
        // `dep` is computed from this thread's reads of the slots about to be
        // refilled: consuming it here orders those reads before the copies.
        asm volatile("" ::"r"(dep) : "memory");
        const long long base = tile * C::TILE;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const long long i = base + (long long)p * kThreads + tid;
            if (i < n) {
                copy_point_async<D>(sx, X + i * D, p, tid);
                if (mode == kModeDelta) cp_async4(sl + p * kThreads + tid, labels + i);
            }
        }
        cp_async_commit();
    };
    if ((long long)blockIdx.x < ntiles) prefetch(blockIdx.x, 0u);

    int it = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const long long base = tile * C::TILE;
        cp_async_wait_all();
        float x[P][D];
        int oldl[P];
        float xn2[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const long long i = base + (long long)p * kThreads + tid;
            if (i < n) {
                read_point<D>(sx, p, tid, x[p]);
                oldl[p] = (mode == kModeDelta) ? sl[p * kThreads + tid] : -1;
            } else {
#pragma unroll
                for (int t = 0; t < D; ++t) x[p][t] = 0.0f;
                oldl[p] = -1;
            }
            float s2 = 0.0f;
#pragma unroll
            for (int t = 0; t < D; ++t) s2 = fmaf(x[p][t], x[p][t], s2);
            xn2[p] = s2;
        }
        const long long next = tile + gridDim.x;
        if (next < ntiles) {
            unsigned dep = __float_as_uint(xn2[0]);
#pragma unroll
            for (int p = 1; p < P; ++p) dep ^= __float_as_uint(xn2[p]);
            prefetch(next, dep);
        }

        float B1[P], B2[P];
        int BI[P];
#pragma unroll
        for (int p = 0; p < P; ++p) { B1[p] = INFINITY; B2[p] = INFINITY; BI[p] = 0; }
        for (int ch = 0; ch < nchunks; ++ch) {
            float b1[P], b2[P];
#pragma unroll
            for (int p = 0; p < P; ++p) { b1[p] = INFINITY; b2[p] = INFINITY; }
            const float* cbase = sc + (size_t)(ch << 5) * DS;
            const float* sbase = ss + (ch << 5);
            // one packed FMA evaluates dimension t for both centers of a
            // pair (each half rounds like its own fmaf)
#pragma unroll 4
            for (unsigned jj = 0; jj < 32; jj += 2) {
                float2 cp[DS];
                const float4* q = reinterpret_cast<const float4*>(cbase + jj * DS);
#pragma unroll
                for (int h = 0; h < DS / 2; ++h) {
                    const float4 v = q[h];
                    cp[2 * h] = make_float2(v.x, v.y);
                    cp[2 * h + 1] = make_float2(v.z, v.w);
                }
                const float2 st01 = *reinterpret_cast<const float2*>(sbase + jj);
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    float2 dd = st01;
#pragma unroll
                    for (int t = 0; t < D; ++t)
                        dd = __ffma2_rn(make_float2(x[p][t], x[p][t]), cp[t], dd);
                    const float k0 = pack_key(dd.x, jj), k1 = pack_key(dd.y, jj | 1u);
                    const float lo = fminf(k0, k1), hi = fmaxf(k0, k1);
                    b2[p] = fmin3(b2[p], hi, fmaxf(b1[p], lo));
                    b1[p] = fminf(b1[p], lo);
                }
            }
#pragma unroll
            for (int p = 0; p < P; ++p) {
                if (b1[p] < B1[p]) {
                    B2[p] = fminf(B1[p], b2[p]);
                    B1[p] = b1[p];
                    BI[p] = (ch << 5) | (int)(__float_as_uint(b1[p]) & 31u);
                } else {
                    B2[p] = fminf(B2[p], b1[p]);
                }
            }
        }
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const long long i = base + (long long)p * kThreads + tid;
            const bool valid = i < n;
            const float thr = kappa * (thr_base + xn2[p]) + tie_abs(D + 1) +
                              kpack * (fabsf(B1[p]) + fabsf(B2[p]));
            const bool flag = valid && (B2[p] - B1[p] <= thr);
            recheck_append(flag, (int)i, list, &st->recheck_count);
            if (valid && !flag && label_ok(BI[p], k, st) && old_label_ok(oldl[p], k, st)) {
                const int lab = BI[p];
                const int old = oldl[p];
                if (lab != old) {
#pragma unroll
                    for (int t = 0; t < D; ++t) {
                        const long long v = to_fixed(x[p][t], scaleF);
                        if (use_sacc) {
                            atomicAdd(reinterpret_cast<unsigned long long*>(sacc + lab * D + t),
                                      (unsigned long long)v);
                            if (old >= 0)
                                atomicAdd(reinterpret_cast<unsigned long long*>(sacc + old * D + t),
                                          (unsigned long long)(-v));
                        } else {
                            split_add(acc.s_lo + (long long)lab * D + t,
                                      acc.s_hi + (long long)lab * D + t, v);
                            if (old >= 0)
                                split_add(acc.s_lo + (long long)old * D + t,
                                          acc.s_hi + (long long)old * D + t, -v);
                        }
                    }
                    if (use_sacc) {
                        atomicAdd(scnt + lab, 1);
                        if (old >= 0) atomicAdd(scnt + old, -1);
                    } else {
                        atomicAdd(acc.cnt + lab, 1ull);
                        if (old >= 0) atomicAdd(acc.cnt + old, ~0ull);
                    }
                    labels[i] = lab;
                }
            }
        }
        // Static flush schedule: at most FLUSH_TILES tiles (2^16 points) per partial.
        const bool last = tile + gridDim.x >= ntiles;
        if ((it + 1) % C::FLUSH_TILES == 0 || last) {
            __syncthreads();
            if (use_sacc) {
                for (int e = tid; e < k * D; e += kThreads) {
                    const long long v = sacc[e];
                    if (v) {
                        split_add(acc.s_lo + e, acc.s_hi + e, v);
                        sacc[e] = 0;
                    }
                }
                for (int e = tid; e < k; e += kThreads) {
                    const int v = scnt[e];
                    if (v) {
                        atomicAdd(acc.cnt + e, (unsigned long long)(long long)v);
                        scnt[e] = 0;
                    }
                }
            }
            __syncthreads();
        }
    }
    cp_async_wait_all();
}

// ---------------------------------------------------------------- large d

constexpr int BM = 128, BN = 128, BK = 8;

__global__ void __launch_bounds__(kThreads)
assign_large(const float* __restrict__ X, long long n, int d, Centers c, int* __restrict__ labels,
             StageState* st, Accum acc, int* __restrict__ list, float kappa, int vec4)
{
    __shared__ __align__(16) float Xs[2][BK][BM];
    __shared__ __align__(16) float Cs[2][BK][BN];
    if (st->error) return;
    const int mode = st->mode;
    const float scaleF = st->scaleF;
    const float c2x2 = 2.0f * st->cmax2;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int kpad = c.kpad;
    const int nct = kpad / BN;
    const int nks = c.dpad / BK;
    const long long ntiles = (n + BM - 1) / BM;
    // loader roles
    const int xl_pt = tid >> 1, xl_d = (tid & 1) * 4;     // X: point, first of 4 dims
    const int cl_row = tid >> 5, cl_col = (tid & 31) * 4;  // C: dim row, first of 4 centers

    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long base = tile * BM;
        float b1[8], b2[8], xn2[8];
        int bi[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) { b1[r] = FLT_MAX; b2[r] = FLT_MAX; bi[r] = 0; xn2[r] = 0.f; }

        for (int ct = 0; ct < nct; ++ct) {
            float accm[8][8];
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int q = 0; q < 8; ++q) accm[r][q] = 0.0f;

            auto load_x = [&](int ks, float* xv) {
                const long long i = base + xl_pt;
                const int t0 = ks * BK + xl_d;
                if (i < n) {
                    const float* src = X + i * d + t0;
                    if (vec4 && t0 + 3 < d) {
                        float4 v = __ldg(reinterpret_cast<const float4*>(src));
                        xv[0] = v.x; xv[1] = v.y; xv[2] = v.z; xv[3] = v.w;
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q) xv[q] = (t0 + q < d) ? __ldg(src + q) : 0.0f;
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) xv[q] = 0.0f;
                }
            };
            auto load_c = [&](int ks) -> float4 {
                return __ldg(reinterpret_cast<const float4*>(
                    c.c32t + (long long)(ks * BK + cl_row) * kpad + ct * BN + cl_col));
            };
            float xv[4];
            load_x(0, xv);
            float4 cv4 = load_c(0);
#pragma unroll
            for (int q = 0; q < 4; ++q) Xs[0][xl_d + q][xl_pt] = xv[q];
            *reinterpret_cast<float4*>(&Cs[0][cl_row][cl_col]) = cv4;
            __syncthreads();
            for (int ks = 0; ks < nks; ++ks) {
                const int buf = ks & 1;
                if (ks + 1 < nks) {
                    load_x(ks + 1, xv);
                    cv4 = load_c(ks + 1);
                }
#pragma unroll
                for (int kk = 0; kk < BK; ++kk) {
                    float a[8], b[8];
                    float4 a0 = *reinterpret_cast<const float4*>(&Xs[buf][kk][ty * 4]);
                    float4 a1 = *reinterpret_cast<const float4*>(&Xs[buf][kk][64 + ty * 4]);
                    float4 b0 = *reinterpret_cast<const float4*>(&Cs[buf][kk][tx * 4]);
                    float4 b1v = *reinterpret_cast<const float4*>(&Cs[buf][kk][64 + tx * 4]);
                    a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
                    a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
                    b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
                    b[4] = b1v.x; b[5] = b1v.y; b[6] = b1v.z; b[7] = b1v.w;
#pragma unroll
                    for (int r = 0; r < 8; ++r)
#pragma unroll
                        for (int q = 0; q < 8; ++q) accm[r][q] = fmaf(a[r], b[q], accm[r][q]);
                    if (ct == 0) {
#pragma unroll
                        for (int r = 0; r < 8; ++r) xn2[r] = fmaf(a[r], a[r], xn2[r]);
                    }
                }
                if (ks + 1 < nks) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) Xs[buf ^ 1][xl_d + q][xl_pt] = xv[q];
                    *reinterpret_cast<float4*>(&Cs[buf ^ 1][cl_row][cl_col]) = cv4;
                }
                __syncthreads();
            }
            // epilogue of this center tile: D = ||c||^2 - 2 x.c, running top-2
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int col = ct * BN + (q < 4 ? tx * 4 + q : 64 + tx * 4 + (q - 4));
                const float cn = __ldg(c.cnorm + col);
#pragma unroll
                for (int r = 0; r < 8; ++r)
                    top2_push(fmaf(-2.0f, accm[r][q], cn), col, b1[r], b2[r], bi[r]);
            }
        }
        // merge the 16 column groups of each row (half-warp butterfly)
#pragma unroll
        for (int r = 0; r < 8; ++r) {
#pragma unroll
            for (int o = 1; o < 16; o <<= 1) {
                float o1 = __shfl_xor_sync(0xffffffffu, b1[r], o);
                float o2 = __shfl_xor_sync(0xffffffffu, b2[r], o);
                int oi = __shfl_xor_sync(0xffffffffu, bi[r], o);
                top2_merge(b1[r], b2[r], bi[r], o1, o2, oi);
            }
        }
        int olds[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const long long i = base + (r < 4 ? ty * 4 + r : 64 + ty * 4 + (r - 4));
            olds[r] = (mode == kModeDelta && i < n) ? labels[i] : -1;
        }
        __syncwarp();   // all lanes hold the old labels before lane tx == 0 rewrites them
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const long long i = base + (r < 4 ? ty * 4 + r : 64 + ty * 4 + (r - 4));
            const bool valid = i < n;
            const bool flag = valid && (b2[r] - b1[r] <= kappa * (c2x2 + xn2[r]) + tie_abs(d + 1));
            recheck_append(flag && tx == 0, (int)i, list, &st->recheck_count);
            if (!valid) continue;
            const float* xr = X + i * d;
            if (flag) continue;
            const int lab = bi[r];
            if (!label_ok(lab, c.k, st)) continue;
            const int old = olds[r];
            if (!old_label_ok(old, c.k, st) || lab == old) continue;
            for (int t = tx; t < d; t += 16) {
                long long v = to_fixed(__ldg(xr + t), scaleF);
                split_add(acc.s_lo + (long long)lab * d + t, acc.s_hi + (long long)lab * d + t, v);
                if (old >= 0)
                    split_add(acc.s_lo + (long long)old * d + t, acc.s_hi + (long long)old * d + t,
                              -v);
            }
            if (tx == 0) {
                atomicAdd(acc.cnt + lab, 1ull);
                if (old >= 0) atomicAdd(acc.cnt + old, ~0ull);
                labels[i] = lab;
            }
        }
    }
}

template <int D>
size_t small_smem(int k, bool with_acc)
{
    using C = SmallCfg<D>;
    size_t kc = (size_t)((k + 31) & ~31);
    size_t bytes = kc * (C::DS + 1) * sizeof(float) + (size_t)C::TILE * D * sizeof(float) +
                   (size_t)C::TILE * sizeof(int);
    if (with_acc) bytes += (size_t)k * D * sizeof(long long) + (size_t)k * sizeof(int);
    return bytes;
}

template <int D>
int launch_small(const float* X, long long n, const Centers& c, int* labels, StageState* st,
                 const Accum& acc, int* list, cudaStream_t s, int sm_count)
{
    const bool with_acc = small_smem<D>(c.k, true) <= (size_t)kSmallSmemCap;
    const size_t sm = small_smem<D>(c.k, with_acc);
    if (sm > (size_t)kSmallSmemCap) return KMEANS2_ERR_UNSUPPORTED;
    const void* kfn = (const void*)assign_small<D>;
    KM2_TRY(set_max_dynamic_smem(kfn, kSmallSmemCap));
    int per_sm = 0;
    KM2_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kThreads, sm));
    if (per_sm < 1) return KMEANS2_ERR_UNSUPPORTED;
    const long long tiles = (n + SmallCfg<D>::TILE - 1) / SmallCfg<D>::TILE;
    long long grid = (long long)sm_count * per_sm;
    if (grid > tiles) grid = tiles;
    if (grid < 1) grid = 1;
    ++g_launches;
    assign_small<D><<<(int)grid, kThreads, sm, s>>>(X, n, c, labels, st, acc, list, tie_kappa(D),
                                                    kPackSlack, with_acc ? 1 : 0);
    KM2_CUDA(cudaGetLastError());
    return KMEANS2_OK;
}

}  // namespace

// Shared memory of assign_small without per-CTA accumulators (the smallest form).
static size_t small_smem_min(int d, int k)
{
    size_t ds = (size_t)((d + 3) & ~3) + 1;
    size_t tile = (size_t)kThreads * ((d > 4 && d <= 8) ? 2 : 4);
    return (size_t)((k + 31) & ~31) * ds * 4 + tile * d * 4 + tile * 4;
}

int assign_fp32_supported(int d, int k)
{
    (void)d;
    (void)k;
    return 1;
}

int launch_assign_fp32(const float* X, long long n, int d, const Centers& c, int* labels,
                       StageState* st, const Accum& acc, int* list, cudaStream_t s, int sm_count)
{
    if (d <= 16 && small_smem_min(d, c.k) <= (size_t)kSmallSmemCap) {
        switch (d) {
#define KM2_CASE(DD) \
    case DD: return launch_small<DD>(X, n, c, labels, st, acc, list, s, sm_count);
            KM2_CASE(1) KM2_CASE(2) KM2_CASE(3) KM2_CASE(4) KM2_CASE(5) KM2_CASE(6) KM2_CASE(7)
            KM2_CASE(8) KM2_CASE(9) KM2_CASE(10) KM2_CASE(11) KM2_CASE(12) KM2_CASE(13)
            KM2_CASE(14) KM2_CASE(15) KM2_CASE(16)
#undef KM2_CASE
            default: break;
        }
    }
    int per_sm = 0;
    KM2_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, assign_large, kThreads, 0));
    if (per_sm < 1) per_sm = 1;
    long long tiles = (n + BM - 1) / BM;
    long long grid = (long long)sm_count * per_sm;
    if (grid > tiles) grid = tiles;
    int vec4 = (d % 4 == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0) ? 1 : 0;
    ++g_launches;
    assign_large<<<(int)grid, kThreads, 0, s>>>(X, n, d, c, labels, st, acc, list, tie_kappa(d),
                                                vec4);
    KM2_CUDA(cudaGetLastError());
    return KMEANS2_OK;
}

}  // namespace km2
