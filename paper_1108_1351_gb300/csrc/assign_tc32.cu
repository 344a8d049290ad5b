// assign_tc32.cu -- fused distance + nearest-center + exact-sum kernel with the
// cross term x.c on the 5th-generation tensor cores (tcgen05, kind::tf32),
// for FP32 data with d in {4, 8, 16, 32} and k <= 256.
//
// TF32 keeps 10 mantissa bits, so each FP32 operand is split exactly into a
// high part (its TF32 truncation) and the FP32 remainder: x = xh + xl,
// m = -2c = mh + ml.  Three MMAs per K-step accumulate xh.mh + xh.ml + xl.mh
// (the dropped xl.ml is below 2^-20 |x||m|), and one more K-step adds
// ||c||^2 = nh + nl against a constant [1, 1, 0, ...] A tile, so the
// accumulator holds D_j = ||c_j||^2 - 2 x.c_j for all centers of a 128-point
// tile.  The CUDA cores only split the points and run the epilogue: packed-key
// top-2, the near-tie flag (a bound that covers the split, the tensor core's
// FP32 accumulation and the key packing), labels and the exact fixed-point
// cluster sums.  A row inside the (looser) 3xTF32 bound is first re-decided on
// the CUDA cores with the FP32 FMA chain of the CUDA-core kernels and their
// tighter bound; only rows inside that bound go to the FP64 recheck list.
//
// Warp-specialised pipeline, one CTA per SM, 14 warps.  The unit of every
// hand-off is a group of T 128-point tiles (T = 4, 2 or 1 as k grows), so
// each barrier round trip is paid once per T tiles and each epilogue thread
// works on T independent rows:
//   warp 0      loader: T bulk TMA copies per unit (raw X rows, and the old
//               labels in delta mode) into an RS-stage ring; the rows stay
//               until the unit's epilogue is done (the sums read them back);
//   warps 1-4   producers: thread r splits row r of each tile into the hi / lo
//               A tiles of an SA-stage ring (K-major core-matrix layout);
//   warp 5      MMA issuer: per tile 3 KD + 1 MMAs (M 128, N npad, K 8) into
//               column block t of a TMEM accumulator, one commit per unit;
//   warps 6-13  two epilogue groups taking alternate units, each with NB (1 or
//               2) accumulators of T x npad columns: thread r owns row r of the
//               unit's T tiles; flagged points are queued per warp in shared
//               memory and partial sums kept per warp (when they fit).
// The B operand (every center's -2c hi / lo per K-step and ||c||^2 hi / lo) is
// built once per launch and stays in shared memory.  Roles are coupled only by
// mbarriers; every wait is bounded, and on a timeout the CTA records an error,
// lets its own copies and MMAs finish (bounded), frees TMEM and exits.
#include <cfloat>
#include <cstdint>

#include "api_internal.h"
#include "tc_common.cuh"

namespace km2 {

namespace {

constexpr int kWarps = 14;
constexpr int kThreads = 32 * kWarps;
constexpr int kEpiWarps = 8;
constexpr int kRows = 128;                 // points per tile (UMMA M)
constexpr int kStepBytes = kRows * 32;     // one K-step (8 TF32) of a 128-row A tile
constexpr int kMaxRS = 12, kMaxSA = 4;
constexpr int kSmemBudget = 210 * 1024;
constexpr int kWaitTries = 1 << 22;
constexpr int kRecheckQ = 256;             // flagged points staged per epilogue warp

__device__ __forceinline__ float tf32_hi(float v)
{
    return __uint_as_float(__float_as_uint(v) & 0xffffe000u);
}

__device__ __forceinline__ float pack_key(float v, unsigned j)
{
    return __uint_as_float((__float_as_uint(v) & ~31u) | j);
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(mbar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(mbar))
                 : "memory");
}

__device__ __forceinline__ void bulk_load(void* sdst, const void* gsrc, uint32_t bytes,
                                          uint64_t* mbar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            (uint32_t)__cvta_generic_to_shared(sdst)),
        "l"(gsrc), "r"(bytes), "r"((uint32_t)__cvta_generic_to_shared(mbar))
        : "memory");
}

// Bounded wait that also gives up once another role has aborted.
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                         StageState* st, int tries = kWaitTries)
{
    const uint32_t addr = (uint32_t)__cvta_generic_to_shared(bar);
    for (int i = 0; i < tries; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(addr), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((i & 63) == 63 && *abort_flag) return false;
    }
    *abort_flag = 1;
    atomicExch(&st->error, kErrTimeout);
    return false;
}

// Packed-key top-2 of 32 accumulator columns (center indices j0 .. j0 + 31)
// folded into the running (B1, B2, BI) of a row.
__device__ __forceinline__ void top2_cols(const uint32_t* r, int j0, float& B1, float& B2, int& BI)
{
    float q1[4], q2[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) { q1[q] = INFINITY; q2[q] = INFINITY; }
#pragma unroll
    for (int j = 0; j < 32; j += 8) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int jj = j + 2 * q;
            const float k0 = pack_key(__uint_as_float(r[jj]), (unsigned)jj);
            const float k1 = pack_key(__uint_as_float(r[jj + 1]), (unsigned)jj + 1u);
            const float lo = fminf(k0, k1), hi = fmaxf(k0, k1);
            q2[q] = fmin3(q2[q], hi, fmaxf(q1[q], lo));
            q1[q] = fminf(q1[q], lo);
        }
    }
    const float m01 = fmin3(q2[0], q2[1], fmaxf(q1[0], q1[1]));
    const float l01 = fminf(q1[0], q1[1]);
    const float m23 = fmin3(q2[2], q2[3], fmaxf(q1[2], q1[3]));
    const float l23 = fminf(q1[2], q1[3]);
    const float b2 = fmin3(m01, m23, fmaxf(l01, l23));
    const float b1 = fminf(l01, l23);
    if (b1 < B1) {
        B2 = fminf(B1, b2);
        B1 = b1;
        BI = j0 + (int)(__float_as_uint(b1) & 31u);
    } else {
        B2 = fminf(B2, b1);
    }
}

template <int D>
struct TcCfg {
    static constexpr int KD = (D + 7) / 8;                     // data K-steps
    static constexpr uint32_t ABYTES = 2u * KD * kStepBytes;   // hi + lo A tiles of one tile
};

struct TcLayout {
    int T;                   // tiles per unit
    int rs, sa, nb;          // raw ring, A ring (units), accumulators per epilogue group
    int sacc;                // per-warp shared-memory partial sums
    int lab_bulk;            // old labels arrive with the raw rows (delta mode, aligned labels)
    uint32_t a_off, ones_off, b_off, raw_off, lab_off, rq_off, acc_off, acc_bytes, total;
};

__host__ __device__ inline uint32_t align_up(uint32_t v, uint32_t a) { return (v + a - 1) / a * a; }

__host__ __device__ inline TcLayout tc_layout(int D, int T, int npad, int k, int rs, int sa, int sacc)
{
    const int KD = (D + 7) / 8;
    TcLayout L;
    L.T = T;
    L.rs = rs;
    L.sa = sa;
    L.nb = 4 * T * npad <= 512 ? 2 : 1;
    L.sacc = sacc;
    L.lab_bulk = 0;
    uint32_t o = 0;
    L.a_off = o;
    o += (uint32_t)sa * (uint32_t)T * 2u * KD * kStepBytes;
    L.ones_off = o;
    o += kStepBytes;
    L.b_off = o;
    o += (uint32_t)(2 * KD + 1) * (uint32_t)npad * 32u;
    o = align_up(o, 128);
    L.raw_off = o;
    o += (uint32_t)rs * (uint32_t)T * kRows * (uint32_t)D * 4u;
    o = align_up(o, 16);
    L.lab_off = o;                                 // old labels of each raw stage
    o += (uint32_t)rs * (uint32_t)T * kRows * 4u;
    L.rq_off = o;                                  // recheck queues of the epilogue warps
    o += (uint32_t)kEpiWarps * kRecheckQ * 4u;
    o = align_up(o, 16);
    L.acc_off = o;
    L.acc_bytes = align_up((uint32_t)k * (uint32_t)D * 8u + (uint32_t)k * 4u, 16);
    if (sacc) o += (uint32_t)kEpiWarps * L.acc_bytes;
    L.total = align_up(o, 16);
    return L;
}

struct TcBars {
    uint64_t raw_full[kMaxRS], raw_empty[kMaxRS];
    uint64_t a_full[kMaxSA], a_empty[kMaxSA];
    uint64_t acc_full[4], acc_empty[4];
    uint64_t drain;
};

// The row's FP32 distances to every center by the CUDA-core FMA chain
// (||c||^2 + sum_t fma(x_t, -2 c_t), t ascending), whose rounding tie_kappa
// bounds, and their top-2 (lowest index on equal values).  For rows the
// 3xTF32 bound cannot decide.
template <int D>
__device__ __forceinline__ void fp32_top2(const float* x, const Centers& c, float& b1, float& b2,
                                          int& bi)
{
    b1 = INFINITY;
    b2 = INFINITY;
    bi = 0;
    for (int j = 0; j < c.k; ++j) {
        float a = __ldg(c.cnorm + j);
        const float* cj = c.c32 + (long long)j * D;
#pragma unroll
        for (int t = 0; t < D; ++t) a = fmaf(x[t], -2.0f * __ldg(cj + t), a);
        if (a < b1) {
            b2 = b1;
            b1 = a;
            bi = j;
        } else {
            b2 = fminf(b2, a);
        }
    }
}

template <int D, int T>
__global__ void __launch_bounds__(kThreads, 1)
assign_tc32(const float* __restrict__ X, long long n, Centers c, int* __restrict__ labels,
            StageState* st, Accum acc, int* __restrict__ list, float kappa, float kpack,
            float kappa32, int npad, uint32_t tmem_cols, TcLayout L, int ctries)
{
    using C = TcCfg<D>;
    constexpr int KD = C::KD;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ TcBars bars;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    if (st->error) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int k = c.k;
    const int RS = L.rs, SA = L.sa, NB = L.nb;
    unsigned char* sA = smem + L.a_off;
    unsigned char* sOnes = smem + L.ones_off;
    unsigned char* sB = smem + L.b_off;
    float* raw = reinterpret_cast<float*>(smem + L.raw_off);
    int* lab_ring = reinterpret_cast<int*>(smem + L.lab_off);
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    const int mode = st->mode;
    const bool lab_bulk = L.lab_bulk != 0 && mode == kModeDelta;
    volatile int* abort_v = &abort_flag;
    constexpr uint32_t kRawUnit = (uint32_t)T * kRows * D;        // floats per raw stage
    constexpr uint32_t kAUnit = (uint32_t)T * C::ABYTES;          // bytes per A stage

    // ---- B operand: -2c split in TF32 hi / lo per K-step, then ||c||^2 hi / lo
    const int bitems = npad * (2 * KD + 1) * 2;        // (row, tile, 16-byte chunk)
    for (int e = tid; e < bitems; e += kThreads) {
        const int j = e % npad;
        const int rest = e / npad;
        const int kc = rest & 1;
        const int tile = rest >> 1;                    // 0..2KD-1: (s, part); 2KD: norm
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        if (tile < 2 * KD) {
            const int s = tile >> 1, part = tile & 1;
            if (j < k) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int t = 8 * s + 4 * kc + q;
                    const float m = t < D ? -2.0f * c.c32[(long long)j * D + t] : 0.0f;
                    const float h = tf32_hi(m);
                    v[q] = part == 0 ? h : m - h;
                }
            }
        } else if (kc == 0) {
            // a padding center gets the largest finite TF32 norm: never the best
            const float nrm = j < k ? c.cnorm[j] : 3.3895313892515355e38f;
            const float h = tf32_hi(nrm);
            v[0] = h;
            v[1] = nrm - h;
        }
        *reinterpret_cast<float4*>(sB + (size_t)tile * npad * 32 + tc::tile_offset(j, kc)) =
            make_float4(v[0], v[1], v[2], v[3]);
    }
    // constant A tile [1, 1, 0, ...] for the norm K-step
    if (tid < kRows) {
        *reinterpret_cast<float4*>(sOnes + tc::tile_offset(tid, 0)) = make_float4(1.f, 1.f, 0.f, 0.f);
        *reinterpret_cast<float4*>(sOnes + tc::tile_offset(tid, 1)) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (L.sacc) {
        long long* s0 = reinterpret_cast<long long*>(smem + L.acc_off);
        const int words = (int)((uint32_t)kEpiWarps * L.acc_bytes / 8u);
        for (int e = tid; e < words; e += kThreads) s0[e] = 0;
    }
    if (warp == 5) tc::tmem_alloc(&tmem_base, tmem_cols);
    if (tid == 0) {
        for (int s = 0; s < kMaxRS; ++s) {
            tc::mbar_init(&bars.raw_full[s], 1);
            tc::mbar_init(&bars.raw_empty[s], 4);      // the 4 warps of the consuming group
        }
        for (int s = 0; s < kMaxSA; ++s) {
            tc::mbar_init(&bars.a_full[s], 4);         // the 4 producer warps
            tc::mbar_init(&bars.a_empty[s], 1);
        }
        for (int b = 0; b < 4; ++b) {
            tc::mbar_init(&bars.acc_full[b], 1);
            tc::mbar_init(&bars.acc_empty[b], 4);
        }
        tc::mbar_init(&bars.drain, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;

    // local tile i of this CTA is global tile blockIdx.x + i * gridDim.x;
    // unit u holds local tiles u T .. u T + T - 1 (the last unit may hold fewer)
    const long long ntiles = (n + kRows - 1) / kRows;
    const long long cnt = (long long)blockIdx.x < ntiles
                              ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const long long units = (cnt + T - 1) / T;
    auto tile_of = [&](long long u, int t) { return blockIdx.x + (u * T + t) * gridDim.x; };
    auto tiles_in = [&](long long u) { return (int)(cnt - u * T < T ? cnt - u * T : T); };

    if (warp == 0) {
        // ---------------- loader: raw rows (and old labels) of unit u -> raw stage u % RS
        if (lane == 0) {
            long long issued = 0;
            for (long long u = 0; u < units; ++u) {
                const int rs = (int)(u % RS);
                if (!wait_bar(&bars.raw_empty[rs], (uint32_t)(((u / RS) & 1) ^ 1), abort_v, st))
                    break;
                const int nt = tiles_in(u);
                uint32_t total = 0;
                for (int t = 0; t < nt; ++t) {
                    const long long tile = tile_of(u, t);
                    const long long rows = n - tile * kRows < kRows ? n - tile * kRows : kRows;
                    total += (uint32_t)rows * (uint32_t)D * 4u;               // D * 4: multiple of 16
                    if (lab_bulk) total += (uint32_t)(rows & ~3ll) * 4u;     // 16-byte multiple
                }
                mbar_expect_tx(&bars.raw_full[rs], total);
                for (int t = 0; t < nt; ++t) {
                    const long long tile = tile_of(u, t);
                    const long long rows = n - tile * kRows < kRows ? n - tile * kRows : kRows;
                    bulk_load(raw + (size_t)rs * kRawUnit + (size_t)t * kRows * D, X + tile * kRows * D,
                              (uint32_t)rows * (uint32_t)D * 4u, &bars.raw_full[rs]);
                    const uint32_t lbytes = lab_bulk ? (uint32_t)(rows & ~3ll) * 4u : 0u;
                    if (lbytes)
                        bulk_load(lab_ring + ((size_t)rs * T + t) * kRows, labels + tile * kRows,
                                  lbytes, &bars.raw_full[rs]);
                }
                issued = u + 1;
            }
            // let this CTA's own copies land before it can exit
            for (long long u = issued > RS ? issued - RS : 0; u < issued; ++u)
                tc::mbar_wait(&bars.raw_full[u % RS], (uint32_t)((u / RS) & 1), kWaitTries);
        }
    } else if (warp <= 4) {
        // ---------------- producers: thread r splits row r of each tile of unit u
        const int r = tid - 32;
        for (long long u = 0; u < units; ++u) {
            const int rs = (int)(u % RS), sa = (int)(u % SA);
            bool ok = wait_bar(&bars.raw_full[rs], (uint32_t)((u / RS) & 1), abort_v, st);
            ok = ok && wait_bar(&bars.a_empty[sa], (uint32_t)(((u / SA) & 1) ^ 1), abort_v, st);
            if (!__all_sync(0xffffffffu, ok)) break;
            const int nt = tiles_in(u);
#pragma unroll
            for (int t = 0; t < T; ++t) {
                if (t >= nt) break;
                const bool valid = tile_of(u, t) * kRows + r < n;
                float x[8 * KD];
                const float* src = raw + (size_t)rs * kRawUnit + ((size_t)t * kRows + r) * D;
#pragma unroll
                for (int q = 0; q < D / 4; ++q) {
                    const float4 v = valid ? *reinterpret_cast<const float4*>(src + 4 * q)
                                           : make_float4(0.f, 0.f, 0.f, 0.f);
                    x[4 * q] = v.x; x[4 * q + 1] = v.y; x[4 * q + 2] = v.z; x[4 * q + 3] = v.w;
                }
#pragma unroll
                for (int e = D; e < 8 * KD; ++e) x[e] = 0.f;
                unsigned char* a = sA + (size_t)sa * kAUnit + (size_t)t * C::ABYTES;
#pragma unroll
                for (int s = 0; s < KD; ++s) {
#pragma unroll
                    for (int kc = 0; kc < 2; ++kc) {
                        float h[4], l[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float v = x[8 * s + 4 * kc + q];
                            h[q] = tf32_hi(v);
                            l[q] = v - h[q];
                        }
                        const uint32_t off = tc::tile_offset(r, kc);
                        *reinterpret_cast<float4*>(a + (size_t)s * kStepBytes + off) =
                            make_float4(h[0], h[1], h[2], h[3]);
                        *reinterpret_cast<float4*>(a + (size_t)(KD + s) * kStepBytes + off) =
                            make_float4(l[0], l[1], l[2], l[3]);
                    }
                }
            }
            tc::fence_proxy_async();        // generic writes -> visible to the tensor core
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars.a_full[sa]);
        }
    } else if (warp == 5) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tc::instr_desc(2u, (uint32_t)npad, (uint32_t)kRows);
            uint32_t phase = 0u;             // bit b: parity of accumulator b's next use
            for (long long u = 0; u < units; ++u) {
                const int sa = (int)(u % SA);
                const int b = (int)(u & 1) * NB + (int)((u >> 1) % NB);
                if (!wait_bar(&bars.a_full[sa], (uint32_t)((u / SA) & 1), abort_v, st, ctries)) break;
                if (!wait_bar(&bars.acc_empty[b], ((phase >> b) & 1u) ^ 1u, abort_v, st, ctries)) break;
                tc::fence_after_sync();
                const int nt = tiles_in(u);
                for (int t = 0; t < nt; ++t) {
                    const uint32_t d_tmem = tmem + (uint32_t)((b * T + t) * npad);
                    const uint32_t ab = sbase + L.a_off + (uint32_t)sa * kAUnit + (uint32_t)t * C::ABYTES;
#pragma unroll
                    for (int s = 0; s < KD; ++s) {
                        const uint32_t ah = ab + (uint32_t)s * kStepBytes;
                        const uint32_t al = ab + (uint32_t)(KD + s) * kStepBytes;
                        const uint32_t bh = sbase + L.b_off + (uint32_t)((2 * s + 0) * npad * 32);
                        const uint32_t bl = sbase + L.b_off + (uint32_t)((2 * s + 1) * npad * 32);
                        tc::mma_tf32(d_tmem, tc::smem_desc(ah), tc::smem_desc(bh), idesc, s > 0 ? 1u : 0u);
                        tc::mma_tf32(d_tmem, tc::smem_desc(ah), tc::smem_desc(bl), idesc, 1u);
                        tc::mma_tf32(d_tmem, tc::smem_desc(al), tc::smem_desc(bh), idesc, 1u);
                    }
                    const uint32_t bn = sbase + L.b_off + (uint32_t)(2 * KD * npad * 32);
                    tc::mma_tf32(d_tmem, tc::smem_desc(sbase + L.ones_off), tc::smem_desc(bn), idesc, 1u);
                }
                tc::mma_commit(&bars.acc_full[b]);
                phase ^= 1u << b;
                tc::mma_commit(&bars.a_empty[sa]);
            }
            // every MMA issued by this thread has completed once `drain` flips
            tc::mma_commit(&bars.drain);
            tc::mbar_wait(&bars.drain, 0u, kWaitTries);
        }
    } else {
        // ---------------- epilogue group g: units u = g, g + 2, ...
        const int ew = warp - 6;
        const int g = ew >> 2;
        const int quarter = warp & 3;                      // TMEM lanes 32 * (warp % 4) ...
        const int row = 32 * quarter + lane;
        const uint32_t lane_addr = (uint32_t)(32 * quarter) << 16;
        const float scaleF = st->scaleF;
        const float thr_base = 2.0f * st->cmax2;
        int* rq = reinterpret_cast<int*>(smem + L.rq_off) + ew * kRecheckQ;
        int rq_n = 0;                                      // warp-uniform queue length
        // hands the queued flagged points to the global recheck list (one atomic)
        auto rq_flush = [&]() {
            if (rq_n == 0) return;
            __syncwarp();
            int base = 0;
            if (lane == 0) base = atomicAdd(&st->recheck_count, rq_n);
            base = __shfl_sync(0xffffffffu, base, 0);
            for (int e = lane; e < rq_n; e += 32) list[base + e] = rq[e];
            __syncwarp();
            rq_n = 0;
        };
        long long* sacc = reinterpret_cast<long long*>(smem + L.acc_off + (size_t)ew * L.acc_bytes);
        int* scnt = reinterpret_cast<int*>(sacc + (size_t)k * D);
        // per-warp partials hold at most 2^16 points: fold them every 2^16 / (32 T) units
        const long long flush_units = kFlushPoints / (32 * T);
        uint32_t phase = 0u;                 // bit s: parity of accumulator g NB + s's next use
        long long done = 0;
        for (long long u = g; u < units; u += 2) {
            const int slot = (int)((u >> 1) % NB);
            const int b = g * NB + slot;
            const int rs = (int)(u % RS);
            bool w = wait_bar(&bars.acc_full[b], (phase >> slot) & 1u, abort_v, st, ctries);
            w = w && wait_bar(&bars.raw_full[rs], (uint32_t)((u / RS) & 1), abort_v, st, ctries);
            if (!__all_sync(0xffffffffu, w)) break;
            tc::fence_after_sync();
            const int nt = tiles_in(u);
            float B1[T], B2[T];
            int BI[T];
            // top-2 of every tile's row, the next 32 columns loading while the
            // current ones are compared
            {
                const uint32_t cb = tmem + lane_addr + (uint32_t)(b * T * npad);
                const int chunks = nt * (npad / 32);          // 32-column blocks of this unit
                uint32_t ra[32], rb[32];
#pragma unroll
                for (int t = 0; t < T; ++t) { B1[t] = INFINITY; B2[t] = INFINITY; BI[t] = 0; }
                tc::tmem_ld32_async(cb, ra);
                tc::tmem_wait_ld();
                for (int q = 0; q < chunks; q += 2) {
                    if (q + 1 < chunks) tc::tmem_ld32_async(cb + (uint32_t)((q + 1) * 32), rb);
                    {
                        const int t = (q * 32) / npad, c0 = (q * 32) % npad;
#pragma unroll
                        for (int tt = 0; tt < T; ++tt)
                            if (tt == t) top2_cols(ra, c0, B1[tt], B2[tt], BI[tt]);
                    }
                    tc::tmem_wait_ld();
                    if (q + 1 < chunks) {
                        if (q + 2 < chunks) tc::tmem_ld32_async(cb + (uint32_t)((q + 2) * 32), ra);
                        const int t = ((q + 1) * 32) / npad, c0 = ((q + 1) * 32) % npad;
#pragma unroll
                        for (int tt = 0; tt < T; ++tt)
                            if (tt == t) top2_cols(rb, c0, B1[tt], B2[tt], BI[tt]);
                        tc::tmem_wait_ld();
                    }
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars.acc_empty[b]);
            phase ^= 1u << slot;

            // ---- decide row `row` of each tile from its raw FP32 values
#pragma unroll
            for (int t = 0; t < T; ++t) {
                if (t >= nt) break;
                const long long tile = tile_of(u, t);
                const long long p = tile * kRows + row;
                const bool valid = p < n;
                float x[D];
                const float* src = raw + (size_t)rs * kRawUnit + ((size_t)t * kRows + row) * D;
#pragma unroll
                for (int q = 0; q < D / 4; ++q) {
                    const float4 v = valid ? *reinterpret_cast<const float4*>(src + 4 * q)
                                           : make_float4(0.f, 0.f, 0.f, 0.f);
                    x[4 * q] = v.x; x[4 * q + 1] = v.y; x[4 * q + 2] = v.z; x[4 * q + 3] = v.w;
                }
                float xn2 = 0.f;
#pragma unroll
                for (int e = 0; e < D; ++e) xn2 = fmaf(x[e], x[e], xn2);
                const float thr = kappa * (thr_base + xn2) + tie_abs(3 * D + 3) +
                                  kpack * (fabsf(B1[t]) + fabsf(B2[t]));
                bool flag = valid && (B2[t] - B1[t] <= thr);
                int lab = BI[t];
                if (flag) {
                    // inside the 3xTF32 bound: re-decide with the FP32 FMA chain
                    // and its tighter bound; FP64 only if that cannot decide
                    float f1, f2;
                    fp32_top2<D>(x, c, f1, f2, lab);
                    flag = f2 - f1 <= kappa32 * (thr_base + xn2) + tie_abs(D + 1);
                }
                {
                    const unsigned m = __ballot_sync(0xffffffffu, flag);
                    if (m) {
                        if (rq_n + 32 > kRecheckQ) rq_flush();
                        if (flag) rq[rq_n + __popc(m & lanemask_lt())] = (int)p;
                        rq_n += __popc(m);
                    }
                }
                if (valid && !flag) {
                    const bool from_ring = lab_bulk && (long long)row < ((n - tile * kRows) & ~3ll);
                    const int old = (mode == kModeDelta)
                                        ? (from_ring ? lab_ring[((size_t)rs * T + t) * kRows + row]
                                                     : labels[p])
                                        : -1;
                    if (lab != old && label_ok(lab, c.k, st) && old_label_ok(old, c.k, st)) {
#pragma unroll
                        for (int e = 0; e < D; ++e) {
                            const long long val = to_fixed(x[e], scaleF);
                            if (L.sacc) {
                                atomicAdd(reinterpret_cast<unsigned long long*>(sacc + lab * D + e),
                                          (unsigned long long)val);
                                if (old >= 0)
                                    atomicAdd(reinterpret_cast<unsigned long long*>(sacc + old * D + e),
                                              (unsigned long long)(-val));
                            } else {
                                split_add(acc.s_lo + (long long)lab * D + e,
                                          acc.s_hi + (long long)lab * D + e, val);
                                if (old >= 0)
                                    split_add(acc.s_lo + (long long)old * D + e,
                                              acc.s_hi + (long long)old * D + e, -val);
                            }
                        }
                        if (L.sacc) {
                            atomicAdd(scnt + lab, 1);
                            if (old >= 0) atomicAdd(scnt + old, -1);
                        } else {
                            atomicAdd(acc.cnt + lab, 1ull);
                            if (old >= 0) atomicAdd(acc.cnt + old, ~0ull);
                        }
                        labels[p] = lab;
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars.raw_empty[rs]);
            // static flush schedule: at most 2^16 points per partial
            ++done;
            if (done % flush_units == 0 || u + 2 >= units) {
                if (L.sacc) {
                    __syncwarp();
                    for (int e = lane; e < k * D; e += 32) {
                        const long long vv = sacc[e];
                        if (vv) {
                            split_add(acc.s_lo + e, acc.s_hi + e, vv);
                            sacc[e] = 0;
                        }
                    }
                    for (int e = lane; e < k; e += 32) {
                        const int vv = scnt[e];
                        if (vv) {
                            atomicAdd(acc.cnt + e, (unsigned long long)(long long)vv);
                            scnt[e] = 0;
                        }
                    }
                    __syncwarp();
                }
            }
        }
        rq_flush();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 5) tc::tmem_dealloc(tmem, tmem_cols);
}

}  // namespace

// Per-key error bound of the 3xTF32 form, as a multiple of (2 C2 + X2),
// doubled for the two keys of the gap (derivation in the design notes):
//   split:  xh.ml' + xl'.mh misses < 3 * 2^-20 |x||m|, m = -2c  -> 3 * 2^-19 |x||c|
//   centers rounded to FP32: 2^-23 |x||c|; ||c||^2 split: (2^-24 + 2^-20) ||c||^2
//   accumulation of nt = 24 KD + 2 exact products: nt * 2^-23 * (2 |x||c| + ||c||^2)
inline float tc32_kappa(int KD)
{
    const double nt = 24.0 * KD + 2.0;
    const double a1 = 3.0 * 0x1p-19 + 0x1p-23 + 2.0 * nt * 0x1p-23;   // coefficient of |x||c|
    const double a2 = 0x1p-24 + 0x1p-20 + nt * 0x1p-23;               // coefficient of ||c||^2
    const double per_key = fmax(a1 / 2.0, (a1 / 2.0 + a2) / 2.0);
    return (float)(2.0 * per_key * 1.0625);
}

namespace {

template <int D, int T>
int launch_tc_t(const float* X, long long n, const Centers& c, int* labels, StageState* st,
                const Accum& acc, int* list, cudaStream_t s, int sm_count, int npad)
{
    using C = TcCfg<D>;
    // ring depths and per-warp partial sums, deepest first, within the budget
    TcLayout L{};
    bool found = false;
    for (int sacc = 1; sacc >= 0 && !found; --sacc)
        for (int rs = kMaxRS; rs >= 3 && !found; --rs)
            for (int sa = kMaxSA; sa >= 2 && !found; --sa) {
                if (sa > rs - 1) continue;
                L = tc_layout(D, T, npad, c.k, rs, sa, sacc);
                found = L.total <= (uint32_t)kSmemBudget;
            }
    if (!found) {
        set_last_error_text("assign_tc32: shared-memory budget too small for this shape");
        return KMEANS2_ERR_UNSUPPORTED;
    }
    L.lab_bulk = (reinterpret_cast<uintptr_t>(labels) & 15) == 0 ? 1 : 0;
    uint32_t cols = 32;
    while (cols < (uint32_t)(2 * L.nb * T * npad)) cols <<= 1;
    KM2_TRY(set_max_dynamic_smem((const void*)assign_tc32<D, T>, kSmemBudget));
    const long long tiles = (n + kRows - 1) / kRows;
    long long grid = sm_count;
    if (grid > tiles) grid = tiles;
    if (grid < 1) grid = 1;
    ++g_launches;
    assign_tc32<D, T><<<(int)grid, kThreads, L.total, s>>>(X, n, c, labels, st, acc, list,
                                                           tc32_kappa(C::KD), kPackSlack,
                                                           tie_kappa(D), npad, cols, L,
                                                           consumer_wait_tries(kWaitTries));
    KM2_CUDA(cudaGetLastError());
    return KMEANS2_OK;
}

// True if some ring depth fits T tiles per unit into the shared-memory budget.
bool tc_layout_fits(int D, int T, int npad, int k)
{
    for (int sacc = 1; sacc >= 0; --sacc)
        for (int rs = kMaxRS; rs >= 3; --rs)
            for (int sa = kMaxSA; sa >= 2; --sa)
                if (sa <= rs - 1 && tc_layout(D, T, npad, k, rs, sa, sacc).total <=
                                        (uint32_t)kSmemBudget)
                    return true;
    return false;
}

// Tiles per unit: four while a unit's accumulator stays within 128 columns,
// fewer when that many tiles do not fit into shared memory (wide D).
template <int D>
int launch_tc(const float* X, long long n, const Centers& c, int* labels, StageState* st,
              const Accum& acc, int* list, cudaStream_t s, int sm_count)
{
    const int npad = (c.k + 31) / 32 * 32;
    int T = npad <= 32 ? 4 : (npad <= 64 ? 2 : 1);
    while (T > 1 && !tc_layout_fits(D, T, npad, c.k)) T >>= 1;
    if (T == 4) return launch_tc_t<D, 4>(X, n, c, labels, st, acc, list, s, sm_count, npad);
    if (T == 2) return launch_tc_t<D, 2>(X, n, c, labels, st, acc, list, s, sm_count, npad);
    return launch_tc_t<D, 1>(X, n, c, labels, st, acc, list, s, sm_count, npad);
}

}  // namespace

int assign_tc32_supported(int d, int k, const float* X)
{
    if (k < 1 || k > 256) return 0;
    if ((reinterpret_cast<uintptr_t>(X) & 15) != 0) return 0;
    if (!(d == 4 || d == 8 || d == 16 || d == 32)) return 0;
    return tc_layout_fits(d, 1, (k + 31) / 32 * 32, k) ? 1 : 0;
}

int launch_assign_tc32(const float* X, long long n, int d, const Centers& c, int* labels,
                       StageState* st, const Accum& acc, int* list, cudaStream_t s, int sm_count)
{
    switch (d) {
        case 4: return launch_tc<4>(X, n, c, labels, st, acc, list, s, sm_count);
        case 8: return launch_tc<8>(X, n, c, labels, st, acc, list, s, sm_count);
        case 16: return launch_tc<16>(X, n, c, labels, st, acc, list, s, sm_count);
        case 32: return launch_tc<32>(X, n, c, labels, st, acc, list, s, sm_count);
        default: return KMEANS2_ERR_UNSUPPORTED;
    }
}

}  // namespace km2
