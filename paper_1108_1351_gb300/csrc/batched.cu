// batched.cu -- the batched form: many independent two-stage fits advancing
// together.  Every job keeps its own stage (fast, slow, done), iteration count
// and convergence flag in a device descriptor; one iteration of the whole
// batch is
//   batch_assign<DC>  one launch per dimension class over a list of work items
//                     (job, first 1024-point tile, tile count); items of jobs
//                     that are done, or beyond the current stage's points, are
//                     skipped
//   batch_recheck     FP64 re-decision of the near ties of every running job
//                     as one flat list (a scan of the jobs' flagged counts,
//                     then one warp per flagged point over the whole GPU)
//   batch_finalize    one CTA per job: means, movement, J, stop test, and the
//                     switch from the fast to the slow stage (Section 2)
//   batch_control     sets the graph's while condition: any job still running
// and the loop is captured once as a CUDA graph with a device-side WHILE node.
// The arithmetic of every step is the single-fit arithmetic (stage_dev.cuh,
// the same packed-key top-2, near-tie bound and exact sums).  A tile shape in
// which several lanes share a point adds that point's FP32 terms in another
// order, which the bound covers, so every decision, and with it each job's
// result, equals kmeans2_fit on that job alone.
//
// The tile shape (point slots per lane, lanes per point) and the tiles per
// work item are chosen per dimension class by an autotuner: on the first call
// for a class it times the real first pass of the batch and a delta pass
// after it for each shape and a few item sizes (resetting the sums between
// trials) and keeps the fastest for the rest of the process.  CTAs claim items from an atomic
// counter, largest jobs first, so the iterations in which only a few large
// jobs still run keep every SM busy.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "api_internal.h"
#include "stage_dev.cuh"

namespace km2 {

namespace {

constexpr int kThreads = 256;
constexpr int kTile = 1024;          // points per tile of a work item
constexpr int kMaxK = 256;
constexpr int kMaxD = 64;
constexpr int kMaxTilesPerItem = kFlushPoints / kTile;   // keeps per-item partials < 2^62

struct BatchInst {
    const float* X;          // n x d (caller's, device)
    float* Xs;               // m x d gathered subset
    int* lab_fast;           // m
    int* lab_slow;           // n
    int* list;               // n (recheck list)
    long long* subset;       // m
    long long* pos;          // k
    long long* seltmp;       // k
    double* clus;            // kClusSlots k
    Centers c;
    Accum acc;
    StageState st;
    long long n, m;
    unsigned long long seed;
    double tol_fast, tol_slow;
    int d, k, max_iter;
    int stage;               // 0 fast, 1 slow, 2 done
    unsigned int maxabs_x;   // max |x| over X (scale of the slow stage)
    int iters_fast, conv_fast, error;
    double shift_fast;
    long long rechecked;
};

struct WorkItem {
    int inst;
    int tile0;
    int ntile;
};

__device__ __forceinline__ unsigned int abs_bits(float v)
{
    return __float_as_uint(v) & 0x7fffffffu;
}

// ---------------------------------------------------------------- sampling

// Block-level exact radix select: ascending positions (relative to `off`) of
// the `want` smallest keys splitmix64_at(seed, off + i), i in [0, count).
__device__ void select_block(unsigned long long seed, unsigned long long off, long long count,
                             long long want, long long* out)
{
    __shared__ unsigned int hist[256];
    __shared__ unsigned long long prefix;
    __shared__ long long need;
    __shared__ long long scan[kThreads + 1];
    if (threadIdx.x == 0) { prefix = 0; need = want; }
    __syncthreads();
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 56 - 8 * pass;
        for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        const unsigned long long pf = prefix;
        for (long long i = threadIdx.x; i < count; i += blockDim.x) {
            const unsigned long long key = splitmix64_at(seed, off + (unsigned long long)i);
            const bool match = pass == 0 || (key >> (shift + 8)) == (pf >> (shift + 8));
            if (match) atomicAdd(&hist[(key >> shift) & 255ull], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long acc = 0, nd = need;
            for (int b = 0; b < 256; ++b) {
                if (nd <= acc + (long long)hist[b]) {
                    prefix = pf | ((unsigned long long)b << shift);
                    need = nd - acc;
                    break;
                }
                acc += hist[b];
            }
        }
        __syncthreads();
    }
    const unsigned long long T = prefix;     // the want-th smallest key (keys are distinct)
    const long long per = (count + blockDim.x - 1) / blockDim.x;
    const long long i0 = min(count, (long long)threadIdx.x * per), i1 = min(count, i0 + per);
    long long c = 0;
    for (long long i = i0; i < i1; ++i) c += splitmix64_at(seed, off + (unsigned long long)i) <= T;
    scan[threadIdx.x] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long a = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) { const long long v = scan[t]; scan[t] = a; a += v; }
    }
    __syncthreads();
    long long o = scan[threadIdx.x];
    for (long long i = i0; i < i1; ++i)
        if (splitmix64_at(seed, off + (unsigned long long)i) <= T) out[o++] = i;
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads) batch_sample_kernel(BatchInst* insts)
{
    BatchInst* I = insts + blockIdx.x;
    select_block(I->seed, 0ull, I->n, I->m, I->subset);
    select_block(I->seed, (unsigned long long)I->n, I->m, I->k, I->seltmp);
    // initial centers: the k selected positions in increasing key order
    for (int a = threadIdx.x; a < I->k; a += blockDim.x) {
        const unsigned long long ka = splitmix64_at(I->seed, (unsigned long long)(I->n + I->seltmp[a]));
        int rank = 0;
        for (int b = 0; b < I->k; ++b)
            rank += splitmix64_at(I->seed, (unsigned long long)(I->n + I->seltmp[b])) < ka;
        I->pos[rank] = I->seltmp[a];
    }
}

// Gather X_s, its max |x|, the initial centers, and max |x| over X.
__global__ void __launch_bounds__(kThreads) batch_gather_kernel(BatchInst* insts)
{
    __shared__ unsigned int mx_s, mx_x;
    BatchInst* I = insts + blockIdx.x;
    const int d = I->d;
    if (threadIdx.x == 0) { mx_s = 0; mx_x = 0; }
    __syncthreads();
    unsigned int a = 0;
    const long long total = I->m * d;
    for (long long e = threadIdx.x; e < total; e += blockDim.x) {
        const long long p = e / d;
        const int t = (int)(e - p * d);
        const float v = I->X[I->subset[p] * d + t];
        I->Xs[e] = v;
        a = max(a, abs_bits(v));
    }
    atomicMax(&mx_s, a);
    unsigned int b = 0;
    const long long all = I->n * d;
    for (long long e = threadIdx.x; e < all; e += blockDim.x) b = max(b, abs_bits(__ldg(I->X + e)));
    atomicMax(&mx_x, b);
    __syncthreads();
    for (long long e = threadIdx.x; e < (long long)I->k * d; e += blockDim.x) {
        const long long j = e / d;
        const int t = (int)(e - j * d);
        I->c.c64[e] = (double)I->Xs[I->pos[j] * d + t];
    }
    if (threadIdx.x == 0) {
        I->st.maxabs_bits = mx_s;
        I->maxabs_x = mx_x;
    }
}

// Fast-stage start: scales, loop state, center copies, zero sums.
__global__ void __launch_bounds__(kThreads) batch_prep_kernel(BatchInst* insts)
{
    __shared__ double red[kThreads];
    BatchInst* I = insts + blockIdx.x;
    if (threadIdx.x == 0) {
        stage_init_dev(&I->st, I->d, I->tol_fast, I->max_iter);
        I->stage = I->st.error ? 2 : 0;
        I->error = I->st.error;
        I->rechecked = 0;
        I->iters_fast = 0;
        I->conv_fast = 0;
        I->shift_fast = 0.0;
    }
    __syncthreads();
    center_prep_block(I->c, &I->st, red);
    const long long kd = (long long)I->k * I->d;
    for (long long e = threadIdx.x; e < kd; e += blockDim.x) { I->acc.s_lo[e] = 0; I->acc.s_hi[e] = 0; }
    for (int j = threadIdx.x; j < I->k; j += blockDim.x) I->acc.cnt[j] = 0;
}

// Back to the state of a stage's first pass (used between autotuning trials).
__global__ void __launch_bounds__(kThreads) batch_reset_kernel(BatchInst* insts)
{
    BatchInst* I = insts + blockIdx.x;
    const long long kd = (long long)I->k * I->d;
    for (long long e = threadIdx.x; e < kd; e += blockDim.x) { I->acc.s_lo[e] = 0; I->acc.s_hi[e] = 0; }
    for (int j = threadIdx.x; j < I->k; j += blockDim.x) I->acc.cnt[j] = 0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < 4; ++w) I->st.q[w] = 0ull;
        I->st.recheck_count = 0;
    }
}

// Sets every job's pass mode (autotuning trials: a delta pass after the full one).
__global__ void __launch_bounds__(kThreads) batch_mode_kernel(BatchInst* insts, int count, int mode)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < count) insts[j].st.mode = mode;
}

// ---------------------------------------------------------------- assign

// Tile shape of a dimension class.  G lanes share each point (a group is G
// adjacent lanes of a warp): lane q of a group holds coordinates 4 (c G + q) .. 4 (c G + q) + 3 (c = 0, 1, ...) of
// the group's P points, so every center value a lane reads from shared memory
// serves P FMAs while the lane keeps only P DC / G coordinates in registers.
// The G partial dot products of a point are added across the group with xor
// shuffles (P - P / G per center); afterwards each lane owns R = P / G points
// (their top-2, decision and label).  Slot s of lane q holds the group's
// point s ^ (q R), so every shuffle round adds the upper half of the slots
// into the lower half with the same code in every lane.  G = 1 is the plain
// form (P whole points per thread).  The autotuner picks (P, G) among the
// shapes the registers allow.
template <int DC, int PP, int GG>
struct BCfg {
    static constexpr int P = PP;                     // point slots per lane
    static constexpr int G = GG;                     // lanes per point
    static constexpr int R = P / G;                  // points each lane decides
    static constexpr int DG = DC / G;                // coordinates per lane and point
    static constexpr int GROUPS = kThreads / G;      // lane groups per CTA
    static constexpr int SUB = GROUPS * P;           // points per sub-tile
    static constexpr int NSUB = kTile / SUB;
    static constexpr bool SACC = DC <= 32;           // per-CTA partial sums
    static_assert(P % G == 0 && (G == 1 || DC % (4 * G) == 0), "G divides the point slots and the float4 chunks");
    static_assert(kTile % SUB == 0, "a tile holds whole sub-tiles");
};

// Coordinate held in element tt of a lane's point (lane q of a group of G).
template <int G>
__device__ __forceinline__ int lane_dim(int tt, int q)
{
    return G == 1 ? tt : 4 * ((tt >> 2) * G + q) + (tt & 3);
}

template <int DC>
constexpr size_t batch_smem()
{
    return (size_t)kMaxK * DC * 4 + (size_t)kMaxK * 4 +
           (DC <= 32 ? (size_t)kMaxK * DC * 8 + (size_t)kMaxK * 4 : 0);
}

__device__ __forceinline__ float pack_key(float v, unsigned j)
{
    return __uint_as_float((__float_as_uint(v) & ~31u) | j);
}

// Adds the G partial values of each point across the lane group (lanes
// q ^ m, m = G/2 .. 1): afterwards slots 0 .. R-1 hold whole sums.
template <int P, int G>
__device__ __forceinline__ void group_reduce(float (&a)[P])
{
    constexpr int R = P / G;
#pragma unroll
    for (int m = G / 2; m >= 1; m >>= 1) {
#pragma unroll
        for (int s = 0; s < m * R; ++s) a[s] += __shfl_xor_sync(0xffffffffu, a[s + m * R], m);
    }
}

template <int DC, int PP, int GG>
__global__ void __launch_bounds__(kThreads, 2)
batch_assign(BatchInst* insts, const WorkItem* items, int nitems, int* next_item)
{
    using C = BCfg<DC, PP, GG>;
    constexpr int P = C::P, G = C::G, R = C::R, DG = C::DG;
    extern __shared__ __align__(16) float smem[];
    float* sc = smem;                                         // kMaxK * DC: -2 c
    float* ss = sc + kMaxK * DC;                              // kMaxK: ||c||^2
    long long* sacc = reinterpret_cast<long long*>(ss + kMaxK);
    int* scnt = reinterpret_cast<int*>(sacc + kMaxK * DC);
    __shared__ unsigned long long sq[4];     // this item's sum of s^2 (wide_add4 words)
    __shared__ int s_item;
    const int tid = threadIdx.x;
    const int q = tid % G;                   // lane within its group
    const int gi = tid / G;                  // group
    // ||c||^2 enters each point's sum through lane 0 of its group
    const float own0 = q == 0 ? 1.0f : 0.0f;

    // items are claimed dynamically (largest jobs first), so the CTAs stay busy
    // when only a few jobs are still running
    for (;;) {
        if (tid == 0) s_item = atomicAdd(next_item, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();   // every thread has read it before thread 0 claims the next
        if (it >= nitems) break;
        const WorkItem w = items[it];
        BatchInst* I = insts + w.inst;
        const int stage = I->stage;
        if (stage >= 2) continue;
        const long long npts = stage == 0 ? I->m : I->n;
        const long long tiles = (npts + kTile - 1) / kTile;
        if (w.tile0 >= tiles) continue;
        const float* X = stage == 0 ? I->Xs : I->X;
        int* labels = stage == 0 ? I->lab_fast : I->lab_slow;
        StageState* st = &I->st;
        const int d = I->d, k = I->k;
        const int kc = (k + 31) & ~31;
        const int mode = st->mode;
        const float scaleF = st->scaleF;
        const float thr_base = 2.0f * st->cmax2;
        const float kappa = tie_kappa(d);

        __syncthreads();   // the previous item is done with shared memory
        for (int e = tid; e < kc * DC; e += kThreads) {
            const int j = e / DC, t = e - j * DC;
            sc[e] = (j < k && t < d) ? -2.0f * I->c.c32[(long long)j * d + t] : 0.0f;
        }
        for (int j = tid; j < kc; j += kThreads) ss[j] = j < k ? I->c.cnorm[j] : FLT_MAX;
        if (C::SACC) {
            for (int e = tid; e < k * DC; e += kThreads) sacc[e] = 0;
            for (int e = tid; e < k; e += kThreads) scnt[e] = 0;
        }
        if (tid < 4) sq[tid] = 0;
        __syncthreads();

        unsigned __int128 qloc = 0;     // full mode: exact sum of s^2 (J, Eq. 3)
        const long long t_end = min(tiles, (long long)w.tile0 + w.ntile);
        for (long long tile = w.tile0; tile < t_end; ++tile) {
            for (int sub = 0; sub < C::NSUB; ++sub) {
                const long long base = tile * kTile + (long long)sub * C::SUB;
                float x[P][DG];
#pragma unroll
                for (int s = 0; s < P; ++s) {
                    const long long i = base + (long long)(s ^ (q * R)) * C::GROUPS + gi;
                    if constexpr (DC % 4 == 0) {
                        if ((d & 3) == 0) {
                            // rows are 16-byte aligned: one 128-bit load per 4 coordinates
#pragma unroll
                            for (int cc = 0; cc < DG / 4; ++cc) {
                                const int t0 = lane_dim<G>(4 * cc, q);
                                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                                if (i < npts && t0 < d)
                                    v = __ldg(reinterpret_cast<const float4*>(X + i * d + t0));
                                x[s][4 * cc] = v.x; x[s][4 * cc + 1] = v.y;
                                x[s][4 * cc + 2] = v.z; x[s][4 * cc + 3] = v.w;
                            }
                            continue;
                        }
                    }
#pragma unroll
                    for (int tt = 0; tt < DG; ++tt) {
                        const int t = lane_dim<G>(tt, q);
                        x[s][tt] = (i < npts && t < d) ? __ldg(X + i * d + t) : 0.0f;
                    }
                }
                float B1[R], B2[R];
                int BI[R];
#pragma unroll
                for (int r = 0; r < R; ++r) { B1[r] = INFINITY; B2[r] = INFINITY; BI[r] = 0; }
                for (int ch = 0; ch < kc; ch += 32) {
                    float b1[R], b2[R];
#pragma unroll
                    for (int r = 0; r < R; ++r) { b1[r] = INFINITY; b2[r] = INFINITY; }
#pragma unroll 2
                    for (unsigned jj = 0; jj < 32; jj += 2) {
                        const float* c0 = sc + (ch + jj) * DC;
                        const float* c1 = c0 + DC;
                        const float s0 = ss[ch + jj] * own0, s1 = ss[ch + jj + 1] * own0;
                        float a0[P], a1[P];
#pragma unroll
                        for (int s = 0; s < P; ++s) { a0[s] = s0; a1[s] = s1; }
                        if constexpr (G == 1) {
#pragma unroll
                            for (int s = 0; s < P; ++s) {
#pragma unroll
                                for (int t = 0; t < DC; ++t) {
                                    a0[s] = fmaf(x[s][t], c0[t], a0[s]);
                                    a1[s] = fmaf(x[s][t], c1[t], a1[s]);
                                }
                            }
                        } else {
#pragma unroll
                            for (int cc = 0; cc < DG / 4; ++cc) {
                                const int t0 = lane_dim<G>(4 * cc, q);
                                const float4 u0 = *reinterpret_cast<const float4*>(c0 + t0);
                                const float4 u1 = *reinterpret_cast<const float4*>(c1 + t0);
#pragma unroll
                                for (int s = 0; s < P; ++s) {
                                    a0[s] = fmaf(x[s][4 * cc], u0.x, a0[s]);
                                    a1[s] = fmaf(x[s][4 * cc], u1.x, a1[s]);
                                    a0[s] = fmaf(x[s][4 * cc + 1], u0.y, a0[s]);
                                    a1[s] = fmaf(x[s][4 * cc + 1], u1.y, a1[s]);
                                    a0[s] = fmaf(x[s][4 * cc + 2], u0.z, a0[s]);
                                    a1[s] = fmaf(x[s][4 * cc + 2], u1.z, a1[s]);
                                    a0[s] = fmaf(x[s][4 * cc + 3], u0.w, a0[s]);
                                    a1[s] = fmaf(x[s][4 * cc + 3], u1.w, a1[s]);
                                }
                            }
                            group_reduce<P, G>(a0);
                            group_reduce<P, G>(a1);
                        }
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            const float k0 = pack_key(a0[r], jj), k1 = pack_key(a1[r], jj | 1u);
                            const float lo = fminf(k0, k1), hi = fmaxf(k0, k1);
                            b2[r] = fmin3(b2[r], hi, fmaxf(b1[r], lo));
                            b1[r] = fminf(b1[r], lo);
                        }
                    }
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if (b1[r] < B1[r]) {
                            B2[r] = fminf(B1[r], b2[r]);
                            B1[r] = b1[r];
                            BI[r] = ch | (int)(__float_as_uint(b1[r]) & 31u);
                        } else {
                            B2[r] = fminf(B2[r], b1[r]);
                        }
                    }
                }
                float xn2[P];
#pragma unroll
                for (int s = 0; s < P; ++s) {
                    float a = 0.f;
#pragma unroll
                    for (int tt = 0; tt < DG; ++tt) a = fmaf(x[s][tt], x[s][tt], a);
                    xn2[s] = a;
                }
                group_reduce<P, G>(xn2);
                if (mode == kModeFull) {
#pragma unroll
                    for (int s = 0; s < P; ++s) {
                        if (base + (long long)(s ^ (q * R)) * C::GROUPS + gi < npts) {
#pragma unroll
                            for (int tt = 0; tt < DG; ++tt)
                                if (lane_dim<G>(tt, q) < d) qloc += sq_fixed(x[s][tt], scaleF);
                        }
                    }
                }
                // decisions of the lane's own points: the new label where it
                // changed (else -1) and the old one
                int dec[R], olds[R];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const long long i = base + (long long)(r + q * R) * C::GROUPS + gi;
                    const bool valid = i < npts;
                    // a key adds up to d + G - 1 rounded products and sums
                    const float thr = kappa * (thr_base + xn2[r]) + tie_abs(d + G) +
                                      kPackSlack * (fabsf(B1[r]) + fabsf(B2[r]));
                    const bool flag = valid && (B2[r] - B1[r] <= thr);
                    recheck_append(flag, (int)i, I->list, &st->recheck_count);
                    dec[r] = -1;
                    olds[r] = -1;
                    if (valid && !flag) {
                        const int lab = BI[r];
                        const int old = (mode == kModeDelta) ? labels[i] : -1;
                        if (lab != old && label_ok(lab, I->c.k, st) &&
                            old_label_ok(old, I->c.k, st)) {
                            dec[r] = lab;
                            olds[r] = old;
                            labels[i] = lab;
                        }
                    }
                }
                // exact sums: every lane moves its coordinates of each of its
                // slots' points whose label changed (the decision comes from
                // the point's owner, lane q ^ (s / R), slot s % R)
#pragma unroll
                for (int s = 0; s < P; ++s) {
                    int lab = dec[s % R], old = olds[s % R];
                    if constexpr (G > 1) {
                        if (s / R != 0) {
                            lab = __shfl_xor_sync(0xffffffffu, lab, s / R);
                            old = __shfl_xor_sync(0xffffffffu, old, s / R);
                        }
                    }
                    if (lab < 0) continue;
#pragma unroll
                    for (int tt = 0; tt < DG; ++tt) {
                        const int t = lane_dim<G>(tt, q);
                        if (t >= d) break;
                        const long long v = to_fixed(x[s][tt], scaleF);
                        if (C::SACC) {
                            atomicAdd(reinterpret_cast<unsigned long long*>(sacc + lab * DC + t),
                                      (unsigned long long)v);
                            if (old >= 0)
                                atomicAdd(reinterpret_cast<unsigned long long*>(sacc + old * DC + t),
                                          (unsigned long long)(-v));
                        } else {
                            split_add(I->acc.s_lo + (long long)lab * d + t,
                                      I->acc.s_hi + (long long)lab * d + t, v);
                            if (old >= 0)
                                split_add(I->acc.s_lo + (long long)old * d + t,
                                          I->acc.s_hi + (long long)old * d + t, -v);
                        }
                    }
                    if (s < R) {   // the owner counts its point once
                        if (C::SACC) {
                            atomicAdd(scnt + lab, 1);
                            if (old >= 0) atomicAdd(scnt + old, -1);
                        } else {
                            atomicAdd(I->acc.cnt + lab, 1ull);
                            if (old >= 0) atomicAdd(I->acc.cnt + old, ~0ull);
                        }
                    }
                }
            }
        }
        if (mode == kModeFull) {
            qloc = warp_sum_u128(qloc);
            if ((tid & 31) == 0 && qloc) wide_add4(sq, qloc);
        }
        __syncthreads();
        if (C::SACC) {
            for (int e = tid; e < k * DC; e += kThreads) {
                const int j = e / DC, t = e - j * DC;
                const long long v = sacc[e];
                if (v && t < d)
                    split_add(I->acc.s_lo + (long long)j * d + t, I->acc.s_hi + (long long)j * d + t, v);
            }
            for (int j = tid; j < k; j += kThreads)
                if (scnt[j]) atomicAdd(I->acc.cnt + j, (unsigned long long)(long long)scnt[j]);
        }
        if (tid < 4 && sq[tid]) atomicAdd(&st->q[tid], sq[tid]);
    }
}

// ---------------------------------------------------------------- recheck, finalize, control

// The recheck of the whole batch as one flat list: prefix[j] = flagged points
// of the running jobs before job j, prefix[count] = all of them (one CTA,
// sequential over thread slices: jobs in order, so the list order is fixed).
__global__ void __launch_bounds__(1024) batch_recheck_scan_kernel(const BatchInst* insts, int count,
                                                                  long long* prefix)
{
    __shared__ long long part[1024];
    const int per = (count + (int)blockDim.x - 1) / (int)blockDim.x;
    const int j0 = min(count, (int)threadIdx.x * per), j1 = min(count, j0 + per);
    auto flagged = [&](int j) -> long long {
        const BatchInst& I = insts[j];
        return (I.stage < 2 && I.st.error == 0) ? (long long)I.st.recheck_count : 0ll;
    };
    long long sum = 0;
    for (int j = j0; j < j1; ++j) sum += flagged(j);
    part[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long acc = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) { const long long v = part[t]; part[t] = acc; acc += v; }
        prefix[count] = acc;
    }
    __syncthreads();
    long long acc = part[threadIdx.x];
    for (int j = j0; j < j1; ++j) {
        prefix[j] = acc;
        acc += flagged(j);
    }
}

// One warp per flagged point of the flat list (recheck_point): the work of
// all jobs is spread over the whole GPU, so a job with many near ties no
// longer holds one CTA for the rest of the iteration.
__global__ void __launch_bounds__(kThreads) batch_recheck_flat_kernel(BatchInst* insts, int count,
                                                                      const long long* prefix)
{
    __shared__ float cache[kThreads / 32][256];     // k <= 256 in the batched form
    const long long total = prefix[count];
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += nw) {
        // the job of entry w: the first j with prefix[j + 1] > w (warp-uniform)
        int lo = 0, hi = count - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (prefix[mid + 1] > w) hi = mid; else lo = mid + 1;
        }
        BatchInst* I = insts + lo;
        const float* X = I->stage == 0 ? I->Xs : I->X;
        int* labels = I->stage == 0 ? I->lab_fast : I->lab_slow;
        recheck_point(X, I->d, I->c, labels, I->list[w - prefix[lo]], &I->st, I->acc,
                      cache[threadIdx.x >> 5], 256);
    }
}

__global__ void __launch_bounds__(kThreads) batch_finalize_kernel(BatchInst* insts, int* active)
{
    __shared__ FinalizeSmem sm;
    __shared__ int switched;
    BatchInst* I = insts + blockIdx.x;
    const int stage = I->stage;
    if (stage >= 2) return;
    if (I->st.error) {
        if (threadIdx.x == 0) { I->stage = 2; I->error = I->st.error; }
        return;
    }
    finalize_block(I->acc, I->c, &I->st, TrajDev{nullptr, nullptr, nullptr, nullptr}, I->clus, sm);
    if (threadIdx.x == 0) {
        switched = 0;
        if (I->st.done) {
            I->rechecked += I->st.rechecked_total;
            if (stage == 0) {
                // slow stage on S_n from the fast stage's final centers (Section 2)
                I->iters_fast = I->st.iter;
                I->conv_fast = I->st.converged;
                I->shift_fast = I->st.shift;
                I->st.maxabs_bits = I->maxabs_x;
                stage_init_dev(&I->st, I->d, I->tol_slow, I->max_iter);
                if (I->st.error) {
                    I->stage = 2;
                    I->error = I->st.error;
                } else {
                    I->stage = 1;
                    switched = 1;
                }
            } else {
                I->stage = 2;
            }
        }
        if (I->stage < 2) atomicAdd(active, 1);
    }
    __syncthreads();
    if (switched) {
        const long long kd = (long long)I->k * I->d;
        for (long long e = threadIdx.x; e < kd; e += blockDim.x) { I->acc.s_lo[e] = 0; I->acc.s_hi[e] = 0; }
        for (int j = threadIdx.x; j < I->k; j += blockDim.x) I->acc.cnt[j] = 0;
    }
}

__global__ void batch_control_kernel(int* active, int* iter, int* next_item, int nclass, int cap,
                                     unsigned long long handle)
{
    const int a = *active;
    *active = 0;
    for (int c = 0; c < nclass; ++c) next_item[c] = 0;   // work lists of the next iteration
    const int it = ++*iter;
    cudaGraphSetConditional(handle, (a > 0 && it < cap) ? 1u : 0u);
}

// Host-driven form of batch_control_kernel (profiled runs): hands the number of
// jobs still running to the host instead of a graph condition.
__global__ void batch_step_kernel(int* active, int* iter, int* next_item, int nclass, int* out)
{
    const int a = *active;
    *active = 0;
    for (int c = 0; c < nclass; ++c) next_item[c] = 0;
    ++*iter;
    *out = a;
}

// ---------------------------------------------------------------- host

int dclass(int d)
{
    if (d <= 2) return 2;
    if (d <= 4) return 4;
    if (d <= 8) return 8;
    if (d <= 16) return 16;
    if (d <= 32) return 32;
    return 64;
}

template <int DC, int P, int G>
int launch_batch_assign(BatchInst* insts, const WorkItem* items, int nitems, int* next_item,
                        cudaStream_t s, int sm_count)
{
    const size_t sm = batch_smem<DC>();
    KM2_TRY(set_max_dynamic_smem((const void*)batch_assign<DC, P, G>, (int)sm));
    int per_sm = 0;
    KM2_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_assign<DC, P, G>,
                                                           kThreads, sm));
    if (per_sm < 1) per_sm = 1;
    long long grid = (long long)sm_count * per_sm;
    if (grid > nitems) grid = nitems;
    if (grid < 1) grid = 1;
    ++g_launches;
    batch_assign<DC, P, G><<<(int)grid, kThreads, sm, s>>>(insts, items, nitems, next_item);
    KM2_CUDA(cudaGetLastError());
    return KMEANS2_OK;
}

// Tile shape of the distance kernel: point slots per lane and lanes per point.
struct TileShape {
    int p = 0;
    int g = 0;
};

// Tile shapes the autotuner may pick for a dimension class: as many point
// slots as the registers hold (a lane keeps p DC / g floats); shared points
// (g > 1) for the wide classes, where one point per thread would spend a
// shared-memory read on every FMA.
std::vector<TileShape> tile_shapes(int dc)
{
    if (dc <= 16) return {{2, 1}, {4, 1}};
    if (dc <= 32) return {{1, 1}, {2, 1}, {4, 2}, {4, 4}};
    return {{1, 1}, {2, 2}, {4, 4}};
}

// Debug builds (KM2_DEBUG_CHECKS): KMEANS2_DEBUG_BATCH_POINTS = "p" or "pxg"
// forces one tile shape on every dimension class that offers it, without
// tuning, so that a test can run each kernel variant; p = 0 otherwise.
TileShape forced_tile_shape(int dc)
{
#ifdef KM2_DEBUG_CHECKS
    const char* v = std::getenv("KMEANS2_DEBUG_BATCH_POINTS");
    if (v && *v) {
        char* end = nullptr;
        TileShape f;
        f.p = (int)std::strtol(v, &end, 10);
        f.g = (end && *end == 'x') ? (int)std::strtol(end + 1, nullptr, 10) : 1;
        for (const TileShape& t : tile_shapes(dc))
            if (t.p == f.p && t.g == f.g) return f;
    }
#else
    (void)dc;
#endif
    return TileShape{};
}

int launch_class(int dc, TileShape sh, BatchInst* insts, const WorkItem* items, int nitems,
                 int* next_item, cudaStream_t s, int sm_count)
{
#define KM2_BA(DD, PP, GG)                                                                  \
    if (dc == DD && sh.p == PP && sh.g == GG)                                               \
        return launch_batch_assign<DD, PP, GG>(insts, items, nitems, next_item, s, sm_count);
    KM2_BA(2, 2, 1) KM2_BA(2, 4, 1) KM2_BA(4, 2, 1) KM2_BA(4, 4, 1) KM2_BA(8, 2, 1)
    KM2_BA(8, 4, 1) KM2_BA(16, 2, 1) KM2_BA(16, 4, 1) KM2_BA(32, 1, 1) KM2_BA(32, 2, 1)
    KM2_BA(32, 4, 2) KM2_BA(32, 4, 4) KM2_BA(64, 1, 1) KM2_BA(64, 2, 2) KM2_BA(64, 4, 4)
#undef KM2_BA
    set_last_error_text("batched form: no kernel for this tile shape");
    return KMEANS2_ERR_UNSUPPORTED;
}

std::mutex g_tune_mu;
// dimension class -> (tile shape, tiles per work item)
std::map<int, std::pair<TileShape, int>> g_tuned;

struct ClassItems {
    int dc = 0;
    TileShape shape;
    int tpi = 0;
    std::vector<WorkItem> host;
    WorkItem* dev = nullptr;
    int count = 0;
};

// Work items of a dimension class, largest jobs first (longest-processing-
// time order: the big jobs' items start early and the small ones fill in).
void build_items(ClassItems& ci, const std::vector<int>& members, const std::vector<long long>& n,
                 int tpi)
{
    ci.host.clear();
    std::vector<int> order(members);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
    for (int j : order) {
        const long long tiles = (n[j] + kTile - 1) / kTile;
        for (long long t = 0; t < tiles; t += tpi)
            ci.host.push_back(WorkItem{j, (int)t, tpi});
    }
    ci.count = (int)ci.host.size();
    ci.tpi = tpi;
}

}  // namespace

}  // namespace km2

using namespace km2;

extern "C" int kmeans2_batched_tile_shape(int32_t d, int32_t* points, int32_t* lanes,
                                          int32_t* tiles)
{
    if (d < 1 || d > kMaxD || !points || !lanes || !tiles) return KMEANS2_ERR_INVALID;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto f = g_tuned.find(dclass(d));
    if (f == g_tuned.end()) return KMEANS2_ERR_INVALID;
    *points = f->second.first.p;
    *lanes = f->second.first.g;
    *tiles = f->second.second;
    return KMEANS2_OK;
}

extern "C" int kmeans2_fit_batched(int32_t count, const kmeans2_job* jobs, kmeans2_result* results,
                                   const kmeans2_options* opt)
{
    auto t0 = std::chrono::steady_clock::now();
    if (count < 1 || !jobs) return KMEANS2_ERR_INVALID;
    kmeans2_options o;
    kmeans2_default_options(&o);
    if (opt) o = *opt;
    if (o.precision != KMEANS2_PRECISION_FP32 && o.precision != KMEANS2_PRECISION_AUTO) {
        set_last_error_text("the batched form runs the FP32 CUDA-core kernels only");
        return KMEANS2_ERR_UNSUPPORTED;
    }
    for (int j = 0; j < count; ++j) {
        const kmeans2_job& J = jobs[j];
        if (!J.X || !J.centers_out || !J.labels_out || J.n < 1 || J.n >= (1ll << 31) || J.d < 1 ||
            J.d > kMaxD || J.k < 1 || J.k > kMaxK || J.k > J.n ||
            !(J.subset_fraction > 0.0 && J.subset_fraction <= 1.0) || !(J.tol >= 0.0) ||
            J.max_iter < 1 || (reinterpret_cast<uintptr_t>(J.X) & 15) != 0) {
            char msg[160];
            std::snprintf(msg, sizeof(msg), "kmeans2_fit_batched: job %d is out of range", j);
            set_last_error_text(msg);
            return KMEANS2_ERR_INVALID;
        }
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, J.X) != cudaSuccess ||
            (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            set_last_error_text("kmeans2_fit_batched: X must be device memory");
            return KMEANS2_ERR_INVALID;
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(o.stream);
    int dev = 0;
    KM2_CUDA(cudaGetDevice(&dev));
    if (!s) s = private_stream(dev);
    const long long launches0 = g_launches;
    int rc = KMEANS2_OK;
    {
        DeviceScratch ws(s);
        // ---- per-job layout in one arena
        auto up = [](size_t b) { return (b + 255) / 256 * 256; };
        std::vector<BatchInst> hi(count);
        std::vector<size_t> offs(count);
        std::vector<long long> nvec(count);
        size_t total = 0;
        int max_iter_all = 1;
        for (int j = 0; j < count; ++j) {
            const kmeans2_job& J = jobs[j];
            const long long m = kmeans2_subset_size(J.n, J.k, J.subset_fraction);
            const int kpad = (J.k + 127) / 128 * 128, dpad = (J.d + 7) / 8 * 8;
            const size_t kd = (size_t)J.k * J.d;
            offs[j] = total;
            total += up(m * J.d * 4) + up(m * 4) + up(J.n * 4) + up(J.n * 4) + up(m * 8) +
                     3 * up((size_t)J.k * 8) + up((size_t)kClusSlots * J.k * 8) + up(kd * 8) + up(kd * 4) +
                     up((size_t)dpad * kpad * 4) + up((size_t)kpad * 4) + 2 * up(kd * 8) +
                     up((size_t)J.k * 8);
            nvec[j] = J.n;
            max_iter_all = std::max(max_iter_all, J.max_iter);
        }
        unsigned char* arena = nullptr;
        BatchInst* dinst = nullptr;
        int* counters = nullptr;
        KM2_TRY(ws.alloc((void**)&arena, total, s));
        KM2_TRY(ws.alloc((void**)&dinst, sizeof(BatchInst) * (size_t)count, s));
        // active, iteration, 6 item counters, active count handed to the host
        KM2_TRY(ws.alloc((void**)&counters, 9 * sizeof(int), s));
        long long* rprefix = nullptr;      // flat recheck list: per-job offsets, total
        KM2_TRY(ws.alloc((void**)&rprefix, sizeof(long long) * ((size_t)count + 1), s));
        for (int j = 0; j < count; ++j) {
            const kmeans2_job& J = jobs[j];
            BatchInst& I = hi[j];
            std::memset(&I, 0, sizeof(I));
            const long long m = kmeans2_subset_size(J.n, J.k, J.subset_fraction);
            const int kpad = (J.k + 127) / 128 * 128, dpad = (J.d + 7) / 8 * 8;
            const size_t kd = (size_t)J.k * J.d;
            unsigned char* p = arena + offs[j];
            auto take = [&](size_t b) { unsigned char* q = p; p += up(b); return q; };
            I.X = J.X;
            I.Xs = (float*)take(m * J.d * 4);
            I.lab_fast = (int*)take(m * 4);
            I.lab_slow = (int*)take(J.n * 4);
            I.list = (int*)take(J.n * 4);
            I.subset = (long long*)take(m * 8);
            I.pos = (long long*)take((size_t)J.k * 8);
            I.seltmp = (long long*)take((size_t)J.k * 8);
            take((size_t)J.k * 8);
            I.clus = (double*)take((size_t)kClusSlots * J.k * 8);
            I.c.c64 = (double*)take(kd * 8);
            I.c.c32 = (float*)take(kd * 4);
            I.c.c32t = (float*)take((size_t)dpad * kpad * 4);
            I.c.cnorm = (float*)take((size_t)kpad * 4);
            I.c.k = J.k;
            I.c.d = J.d;
            I.c.kpad = kpad;
            I.c.dpad = dpad;
            I.acc.s_lo = (unsigned long long*)take(kd * 8);
            I.acc.s_hi = (unsigned long long*)take(kd * 8);
            I.acc.cnt = (unsigned long long*)take((size_t)J.k * 8);
            I.n = J.n;
            I.m = m;
            I.seed = J.seed;
            I.tol_slow = J.tol;
            I.tol_fast = o.tol_fast > 0.0 ? o.tol_fast : J.tol;
            I.d = J.d;
            I.k = J.k;
            I.max_iter = J.max_iter;
        }
        KM2_CUDA(cudaMemcpyAsync(dinst, hi.data(), sizeof(BatchInst) * (size_t)count,
                                 cudaMemcpyHostToDevice, s));
        KM2_CUDA(cudaMemsetAsync(counters, 0, 9 * sizeof(int), s));
        g_launches += 3;
        batch_sample_kernel<<<count, kThreads, 0, s>>>(dinst);
        batch_gather_kernel<<<count, kThreads, 0, s>>>(dinst);
        batch_prep_kernel<<<count, kThreads, 0, s>>>(dinst);
        KM2_CUDA(cudaGetLastError());

        // ---- work items per dimension class, item size from the autotuner
        std::map<int, std::vector<int>> members;
        for (int j = 0; j < count; ++j) members[dclass(jobs[j].d)].push_back(j);
        std::vector<ClassItems> classes;
        for (auto& kv : members) {
            ClassItems ci;
            ci.dc = kv.first;
            int tpi = 0;
            TileShape shape = forced_tile_shape(ci.dc);
            if (shape.p > 0) {
                tpi = 2;
            } else {
                std::lock_guard<std::mutex> lock(g_tune_mu);
                auto f = g_tuned.find(ci.dc);
                if (f != g_tuned.end()) { shape = f->second.first; tpi = f->second.second; }
            }
            if (tpi == 0) {
                // time the real first pass and a delta pass after it for each
                // tile shape and item size (tiles per work item), resetting the
                // sums between trials: small items keep every SM busy once only a
                // few jobs still run, more point slots per lane reuse each center
                // load more often
                const int cand[4] = {1, 2, 4, 8};
                static_assert(8 <= kMaxTilesPerItem, "item partial sums must stay below 2^62");
                float best_ms = 0.f;
                bool first = true;
                cudaEvent_t e0, e1, e2, e3;
                KM2_CUDA(cudaEventCreate(&e0));
                KM2_CUDA(cudaEventCreate(&e1));
                KM2_CUDA(cudaEventCreate(&e2));
                KM2_CUDA(cudaEventCreate(&e3));
                for (const TileShape& sh : tile_shapes(ci.dc)) {
                    for (int c = 0; c < 4; ++c) {
                        ClassItems trial;
                        build_items(trial, kv.second, nvec, cand[c]);
                        KM2_TRY(ws.alloc((void**)&trial.dev, sizeof(WorkItem) * (size_t)trial.count, s));
                        KM2_CUDA(cudaMemcpyAsync(trial.dev, trial.host.data(),
                                                 sizeof(WorkItem) * (size_t)trial.count,
                                                 cudaMemcpyHostToDevice, s));
                        // the full first pass, then a delta pass over the labels it
                        // wrote (same centers: no label moves), which is what the
                        // later iterations of a fit cost
                        KM2_CUDA(cudaMemsetAsync(counters + 2, 0, sizeof(int), s));
                        KM2_CUDA(cudaEventRecord(e0, s));
                        KM2_TRY(launch_class(ci.dc, sh, dinst, trial.dev, trial.count, counters + 2,
                                             s, ws.sm_count));
                        KM2_CUDA(cudaEventRecord(e1, s));
                        g_launches += 2;
                        batch_reset_kernel<<<count, kThreads, 0, s>>>(dinst);
                        batch_mode_kernel<<<(count + kThreads - 1) / kThreads, kThreads, 0, s>>>(
                            dinst, count, kModeDelta);
                        KM2_CUDA(cudaMemsetAsync(counters + 2, 0, sizeof(int), s));
                        KM2_CUDA(cudaEventRecord(e2, s));
                        KM2_TRY(launch_class(ci.dc, sh, dinst, trial.dev, trial.count, counters + 2,
                                             s, ws.sm_count));
                        KM2_CUDA(cudaEventRecord(e3, s));
                        g_launches += 2;
                        batch_reset_kernel<<<count, kThreads, 0, s>>>(dinst);
                        batch_mode_kernel<<<(count + kThreads - 1) / kThreads, kThreads, 0, s>>>(
                            dinst, count, kModeFull);
                        KM2_CUDA(cudaEventSynchronize(e3));
                        float ms = 0.f, ms2 = 0.f;
                        KM2_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                        KM2_CUDA(cudaEventElapsedTime(&ms2, e2, e3));
                        ms += ms2;
                        if (first || ms < best_ms) { best_ms = ms; tpi = cand[c]; shape = sh; first = false; }
                    }
                }
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                cudaEventDestroy(e2);
                cudaEventDestroy(e3);
                std::lock_guard<std::mutex> lock(g_tune_mu);
                g_tuned[ci.dc] = std::make_pair(shape, tpi);
            }
            ci.shape = shape;
            build_items(ci, kv.second, nvec, tpi);
            KM2_TRY(ws.alloc((void**)&ci.dev, sizeof(WorkItem) * (size_t)ci.count, s));
            KM2_CUDA(cudaMemcpyAsync(ci.dev, ci.host.data(), sizeof(WorkItem) * (size_t)ci.count,
                                     cudaMemcpyHostToDevice, s));
            classes.push_back(std::move(ci));
        }

        KM2_CUDA(cudaMemsetAsync(counters + 2, 0, 6 * sizeof(int), s));
        // one side stream per dimension class: the classes' distance kernels run
        // side by side (parallel branches of the graph body)
        std::vector<cudaStream_t> side(classes.size(), nullptr);
        std::vector<cudaEvent_t> joins(classes.size(), nullptr);
        cudaEvent_t fork = nullptr;
        KM2_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        for (size_t c = 0; c < classes.size(); ++c) {
            KM2_CUDA(cudaStreamCreateWithFlags(&side[c], cudaStreamNonBlocking));
            KM2_CUDA(cudaEventCreateWithFlags(&joins[c], cudaEventDisableTiming));
        }
        auto destroy_side = [&]() {
            for (size_t c = 0; c < classes.size(); ++c) {
                if (side[c]) cudaStreamDestroy(side[c]);
                if (joins[c]) cudaEventDestroy(joins[c]);
            }
            cudaEventDestroy(fork);
        };
        auto launch_classes = [&]() -> int {
            if (cudaEventRecord(fork, s) != cudaSuccess) return KMEANS2_ERR_CUDA;
            for (size_t c = 0; c < classes.size(); ++c) {
                if (cudaStreamWaitEvent(side[c], fork, 0) != cudaSuccess) return KMEANS2_ERR_CUDA;
                const int r = launch_class(classes[c].dc, classes[c].shape, dinst, classes[c].dev,
                                           classes[c].count,
                                           counters + 2 + c, side[c], ws.sm_count);
                if (r != KMEANS2_OK) return r;
                if (cudaEventRecord(joins[c], side[c]) != cudaSuccess) return KMEANS2_ERR_CUDA;
                if (cudaStreamWaitEvent(s, joins[c], 0) != cudaSuccess) return KMEANS2_ERR_CUDA;
            }
            return KMEANS2_OK;
        };
        const int cap = 2 * max_iter_all + 2;
        if (o.profile) {
            // ---- profiled: host-driven loop, CUDA events around each iteration's
            // distance kernels (every kernel is then visible to profilers)
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            for (int it = 0; it < cap && rc == KMEANS2_OK; ++it) {
                cudaEventRecord(e0, s);
                rc = launch_classes();
                if (rc != KMEANS2_OK) break;
                cudaEventRecord(e1, s);
                g_launches += 2;
                batch_recheck_scan_kernel<<<1, 1024, 0, s>>>(dinst, count, rprefix);
                batch_recheck_flat_kernel<<<ws.sm_count * 4, kThreads, 0, s>>>(dinst, count, rprefix);
                ++g_launches;
                batch_finalize_kernel<<<count, kThreads, 0, s>>>(dinst, counters);
                ++g_launches;
                batch_step_kernel<<<1, 1, 0, s>>>(counters, counters + 1, counters + 2,
                                                  (int)classes.size(), counters + 8);
                int active = 0;
                cudaError_t e = cudaMemcpyAsync(&active, counters + 8, sizeof(int),
                                                cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) { set_last_error("batched loop", e); rc = KMEANS2_ERR_CUDA; break; }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                o.profile->assign_launches += (long long)classes.size();
                o.profile->assign_ms += ms;
                if (active == 0) break;
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
        }
        // ---- the iteration loop as one graph with a device-side while condition
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        if (!o.profile) KM2_CUDA(cudaGraphCreate(&graph, 0));
        do {
            if (o.profile) break;
            cudaGraphConditionalHandle handle;
            cudaError_t e = cudaGraphConditionalHandleCreate(&handle, graph, 1u, cudaGraphCondAssignDefault);
            if (e != cudaSuccess) { set_last_error("cudaGraphConditionalHandleCreate", e); rc = KMEANS2_ERR_CUDA; break; }
            alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
            std::memset(raw, 0, sizeof(raw));
            cudaGraphNodeParams* gp = reinterpret_cast<cudaGraphNodeParams*>(raw);
            gp->type = cudaGraphNodeTypeConditional;
            gp->conditional.handle = handle;
            gp->conditional.type = cudaGraphCondTypeWhile;
            gp->conditional.size = 1;
            cudaGraphNode_t node;
            e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, gp);
            if (e != cudaSuccess) { set_last_error("cudaGraphAddNode", e); rc = KMEANS2_ERR_CUDA; break; }
            cudaGraph_t body = gp->conditional.phGraph_out[0];
            e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) { set_last_error("cudaStreamBeginCaptureToGraph", e); rc = KMEANS2_ERR_CUDA; break; }
            rc = launch_classes();
            if (rc == KMEANS2_OK) {
                batch_recheck_scan_kernel<<<1, 1024, 0, s>>>(dinst, count, rprefix);
                batch_recheck_flat_kernel<<<ws.sm_count * 4, kThreads, 0, s>>>(dinst, count, rprefix);
                batch_finalize_kernel<<<count, kThreads, 0, s>>>(dinst, counters);
                batch_control_kernel<<<1, 1, 0, s>>>(counters, counters + 1, counters + 2,
                                                     (int)classes.size(), cap,
                                                     (unsigned long long)handle);
            }
            cudaGraph_t captured = nullptr;
            e = cudaStreamEndCapture(s, &captured);
            if (rc != KMEANS2_OK) break;
            if (e != cudaSuccess) { set_last_error("cudaStreamEndCapture", e); rc = KMEANS2_ERR_CUDA; break; }
            e = cudaGraphInstantiate(&exec, graph, 0);
            if (e != cudaSuccess) { set_last_error("cudaGraphInstantiate", e); rc = KMEANS2_ERR_CUDA; break; }
            e = cudaGraphLaunch(exec, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) { set_last_error("batched graph", e); rc = KMEANS2_ERR_CUDA; break; }
        } while (0);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamSynchronize(s);
        destroy_side();
        if (rc == KMEANS2_OK && !o.profile) {
            int iters = 0;
            KM2_CUDA(cudaMemcpyAsync(&iters, counters + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
            KM2_CUDA(cudaStreamSynchronize(s));
            g_launches += (long long)iters * ((long long)classes.size() + 4);
        }
        if (rc == KMEANS2_OK) {
            // ---- results
            KM2_CUDA(cudaMemcpyAsync(hi.data(), dinst, sizeof(BatchInst) * (size_t)count,
                                     cudaMemcpyDeviceToHost, s));
            KM2_CUDA(cudaStreamSynchronize(s));
            for (int j = 0; j < count && rc == KMEANS2_OK; ++j) {
                const kmeans2_job& J = jobs[j];
                const BatchInst& I = hi[j];
                KM2_CUDA(cudaMemcpyAsync(J.centers_out, I.c.c64, sizeof(double) * (size_t)J.k * J.d,
                                         cudaMemcpyDefault, s));
                KM2_CUDA(cudaMemcpyAsync(J.labels_out, I.lab_slow, sizeof(int) * (size_t)J.n,
                                         cudaMemcpyDefault, s));
            }
            KM2_CUDA(cudaStreamSynchronize(s));
            const double secs =
                std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            bool nonfinite = false;
            for (int j = 0; j < count; ++j) {
                const BatchInst& I = hi[j];
                if (I.error) nonfinite = true;
                if (!results) continue;
                kmeans2_result& r = results[j];
                std::memset(&r, 0, sizeof(r));
                r.J = I.st.J;
                r.iters_fast = I.iters_fast;
                r.iters_slow = I.error ? 0 : I.st.iter;
                r.converged_fast = I.conv_fast;
                r.converged_slow = I.error ? 0 : I.st.converged;
                r.empty_clusters = I.st.empty;
                r.precision_used = KMEANS2_PRECISION_FP32;
                r.subset_size = I.m;
                r.rechecked_points = I.rechecked;
                r.distance_evals = (int64_t)r.iters_fast * I.m * I.k + (int64_t)r.iters_slow * I.n * I.k;
                if (o.profile) {
                    const double pts = (double)r.iters_fast * I.m + (double)r.iters_slow * I.n;
                    o.profile->assign_flops += 2.0 * pts * I.k * I.d;
                    o.profile->assign_bytes += 4.0 * pts * I.d;
                }
                r.shift_fast = I.shift_fast;
                r.shift_slow = I.st.shift;
                r.seconds = secs;
            }
            if (nonfinite) {
                set_last_error_text("kmeans2_fit_batched: some job holds NaN or infinity");
                rc = KMEANS2_ERR_NONFINITE;
            }
        }
    }
    cudaStreamSynchronize(s);
    if (o.profile) o.profile->kernel_launches += g_launches - launches0;
    return rc;
}
