// common.cuh -- definitions shared by the kernels of libkmeans2 (not by the oracle).
//
// Exact cluster sums.  Each FP32 coordinate x enters the sums as the integer
// s = round(x * 2^F).  The per-stage exponent F = 46 - E, with max|x| < 2^E, keeps
// one value below 2^46 in magnitude, so an int64 partial over at most
// kFlushPoints = 2^16 points cannot overflow.  Global sums are kept as two
// 64-bit words: `lo` accumulates the low 32 bits of every contribution
// (unsigned) and `hi` the arithmetic high part, so that the exact sum is
// (int128)hi * 2^32 + lo for any number of contributions below 2^31.  Integer
// addition is associative, so the sums, the centers and J do not depend on the
// order in which threads add: every mode is deterministic.
//
// The objective J (Eq. 3) is formed from the same integers: sum_i s_i^2 over a
// stage's coordinates (st->q, exact), the sums S_j and the counts N_j, so that
// J = W + M with W = sum ||x||^2 - sum_j ||S_j||^2 / N_j (exact integer
// arithmetic) and M = sum_j N_j ||c_j - S_j / N_j||^2 (each difference formed
// without cancellation): no term is a difference of large nearly equal sums.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace km2 {

constexpr int kFlushPoints = 1 << 16;   // max points folded into one int64 partial
constexpr int kModeFull = 0;            // first iteration of a stage: sums from scratch
constexpr int kModeDelta = 1;           // later iterations: only points whose label changed

// Per-stage device state, one instance per stage run, read by every kernel of
// the loop.  Written only by the single-thread / single-CTA kernels
// (stage_init, finalize) except for the atomically updated counters.
struct StageState {
    // fixed-point scale (stage_init)
    int F;                        // exponent of the coordinate fixed point
    float scaleF;                 // 2^F
    double inv_scaleF;            // 2^-F
    unsigned int maxabs_bits;     // max |x| as float bits (atomicMax; NaN/inf sort above)
    int error;                    // nonzero: stage aborted (see kErr*)
    // loop control
    int mode;                     // kModeFull / kModeDelta
    int iter;                     // iterations completed
    int done;                     // converged or iter == max_iter
    int converged;
    int max_iter;
    int empty;                    // empty clusters after the last update
    double tol;
    // per iteration
    float cmax2;                  // >= max_j ||c_j||^2, rounded up to FP32
    int recheck_count;            // entries in the recheck list this iteration
    long long rechecked_total;
    double J;                     // objective of the last assignment
    double shift;                 // last max center movement
    // sum of s^2 over every coordinate of the stage's points (s = round(x 2^F)),
    // exact: the value is sum_w q[w] 2^(32 w) (qsum pass, wide_add4)
    unsigned long long q[4];
    // single-pass FP16 form: rows its bound left undecided, summed over the stage
    long long undecided16_total;
};

// Per-center scratch of finalize, in doubles per center (finalize_center_warp).
constexpr int kClusSlots = 7;

constexpr int kErrNonFinite = 1;
constexpr int kErrRange = 2;       // max|x| >= 2^50
constexpr int kErrTimeout = 3;     // a bounded device-side wait gave up
constexpr int kErrBounds = 4;      // a debug-build index check failed (KM2_DEBUG_CHECKS)

// Debug builds (-DKM2_DEBUG_CHECKS) check every decided label, and every old
// label read back in delta mode (-1 = none), against [0, k) before it
// addresses the cluster sums; a failure records kErrBounds and the point is
// skipped (no trap).  Release builds compile the checks away.
__device__ __forceinline__ bool label_ok(int lab, int k, StageState* st)
{
#ifdef KM2_DEBUG_CHECKS
    if ((unsigned)lab >= (unsigned)k) {
        atomicExch(&st->error, kErrBounds);
        return false;
    }
#else
    (void)lab; (void)k; (void)st;
#endif
    return true;
}
__device__ __forceinline__ bool old_label_ok(int old, int k, StageState* st)
{
    return old == -1 || label_ok(old, k, st);
}

// Accumulator arrays of one stage (device, zeroed by the host before a full pass).
struct Accum {
    unsigned long long* s_lo;     // k*d
    unsigned long long* s_hi;     // k*d
    unsigned long long* cnt;      // k (two's complement int64)
};

// Optional per-iteration records of a stage (device arrays, null = off).
struct TrajDev {
    double* J;                 // max_iter
    double* shift;             // max_iter
    double* centers;           // max_iter * k * d: the updated centers
    long long* counts;         // max_iter * k: the cluster sizes of the assignment
};

// Center copies derived from the FP64 master by center_prep / finalize.
struct Centers {
    double* c64;                  // k*d   FP64 master (row-major)
    float* c32;                   // k*d   FP32 copy (row-major)
    float* c32t;                  // dpad*kpad FP32 copy, transposed (dims x centers)
    float* cnorm;                 // kpad  FP32 of ||c_j||^2; +inf for padding
    int k, d, kpad, dpad;
};

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) as a counter-based generator:
// output number pos of the stream seeded with `seed`.
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed,
                                                             unsigned long long pos)
{
    unsigned long long z = seed + (pos + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ long long to_fixed(float x, float scale)
{
    return __float2ll_rn(x * scale);
}

// Add an int64 contribution to a split (lo, hi) global accumulator.
__device__ __forceinline__ void split_add(unsigned long long* lo, unsigned long long* hi,
                                          long long v)
{
    unsigned long long l = (unsigned long long)v & 0xffffffffull;
    long long h = v >> 32;
    if (l) atomicAdd(lo, l);
    if (h) atomicAdd(hi, (unsigned long long)h);
}

// Exact value of a split accumulator, times 2^-F, as FP64.
__device__ __forceinline__ double split_value(unsigned long long lo, unsigned long long hi,
                                              double inv_scale)
{
    __int128 v = (__int128)(long long)hi * (__int128)4294967296LL + (__int128)lo;
    return (double)v * inv_scale;
}

// s^2 of one coordinate's fixed-point integer s = to_fixed(x, scale), exactly
// (|s| < 2^46, so s^2 < 2^92).
__device__ __forceinline__ unsigned __int128 sq_fixed(float x, float scale)
{
    const long long v = to_fixed(x, scale);
    const unsigned long long a = (unsigned long long)(v < 0 ? -v : v);
    return (unsigned __int128)a * a;
}

// Adds v (< 2^128) to a wide accumulator w[0..3] whose value is
// sum_i w[i] 2^(32 i): piece i of v (32 bits) goes to w[i].  Each word gains
// less than 2^32 per call, so fewer than 2^31 calls cannot wrap it.
__device__ __forceinline__ void wide_add4(unsigned long long* w, unsigned __int128 v)
{
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const unsigned long long piece = (unsigned long long)(v >> (32 * i)) & 0xffffffffull;
        if (piece) atomicAdd(w + i, piece);
    }
}

__device__ __forceinline__ unsigned __int128 warp_sum_u128(unsigned __int128 v)
{
    for (int o = 16; o; o >>= 1) {
        const unsigned long long lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)v, o);
        const unsigned long long hi = __shfl_xor_sync(0xffffffffu, (unsigned long long)(v >> 64), o);
        v += ((unsigned __int128)hi << 64) | lo;
    }
    return v;
}

// 3-input minimum (sm_100+ PTX form).
__device__ __forceinline__ float fmin3(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// Asynchronous global->shared copies of one thread's own data (Ampere-style
// cp.async; completion is waited for by the same thread with cp_async_wait_all).
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(sdst)), "l"(gsrc)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(sdst)), "l"(gsrc)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(sdst)), "l"(gsrc)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Append point i to the recheck list (warp-aggregated; all lanes must call).
__device__ __forceinline__ void recheck_append(bool flag, int i, int* list, int* count)
{
    unsigned mask = __ballot_sync(0xffffffffu, flag);
    if (mask == 0) return;
    int lane = threadIdx.x & 31;
    int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (flag) list[base + __popc(mask & lanemask_lt())] = i;
}

// Near-tie threshold on the FP32 gap between the best and second-best
// expanded distances ||c||^2 - 2 x.c (derivation in the design notes):
// |D_fp32 - D_exact| <= (d+1) u (||c||^2 + 2 ||x|| ||c||) <= (d+1) u (2 C2 + X2)
// per distance, u = 2^-24, C2 = max_j ||c_j||^2, X2 = ||x||^2.  Two distances,
// the FP32 rounding of the gap and of X2, and the oracle's own FP64 rounding
// are covered by kappa = 2 (d + 3) 2^-24 * 1.0625.
__host__ __device__ inline float tie_kappa(int d)
{
    return 2.0f * (float)(d + 3) * 5.9604644775390625e-8f * 1.0625f;
}

// Absolute floor of the near-tie bound.  The relative bounds above hold for
// FP32 values in the normal range; below 2^-126 a result keeps an absolute
// error of up to 2^-126 (IEEE subnormal rounding on the CUDA cores, possible
// flushing to zero inside the tensor cores), and a packed key adds at most 31
// subnormal steps.  With nt products per key, each rounded and accumulated,
// two keys lose at most (4 nt + 16) 2^-126 more: for data of ordinary size
// this is far below the relative term; for tiny data (max|x| below about
// 2^-50) it takes over and flags more points, which the FP64 recheck decides.
__host__ __device__ inline float tie_abs(int nt)
{
    return (float)(4 * nt + 16) * 1.1754943508222875e-38f;
}

// The small-d kernel compares packed keys: D_j with the center's index within
// its chunk of 32 written into the 5 low mantissa bits, compared as floats.  A
// key differs from D_j by less than 2^-18 |D_j|, so the two keys of a point
// add at most 2^-18 (|key_1| + |key_2|) (1 + 2^-17) to the gap error; the
// threshold adds kPackSlack (|key_1| + |key_2|) to the FMA bound.
constexpr float kPackSlack = 3.814697265625e-6f * 1.0625f;   // 2^-18 * 1.0625

}  // namespace km2
