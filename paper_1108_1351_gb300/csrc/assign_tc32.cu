// assign_tc32.cu -- fused distance + nearest-center + exact-sum kernel with the
// cross term x.c on the 5th-generation tensor cores (tcgen05, kind::tf32),
// for FP32 data with d in {4, 8, 16, 32} and k <= 256.
//
// TF32 keeps 10 mantissa bits, so each FP32 operand is split exactly into a
// high part (its TF32 truncation) and the FP32 remainder: x = xh + xl,
// m = -2c = mh + ml.  Three MMAs per K-step accumulate xh.mh + xh.ml + xl.mh
// (the dropped xl.ml is below 2^-20 |x||m|), and one more K-step adds
// ||c||^2 = nh + nl against a constant [1, 1, 0, ...] A column, so the
// accumulator holds D_j = ||c_j||^2 - 2 x.c_j for all centers of a 128-point
// tile.  The CUDA cores only run the epilogue: packed-key top-2, the near-tie
// flag (a bound that covers the split, the tensor core's FP32 accumulation and
// the key packing), labels and the exact fixed-point cluster sums.
//
// Pipeline of one CTA (one warpgroup; thread t owns row t of every tile and
// TMEM lane t): cp.async fetches each thread's own point two tiles ahead;
// produce(i) splits tile i into the K-major shared A tiles and thread 0 issues
// its MMAs into TMEM buffer i % 2; the epilogue of tile i runs while the MMAs
// of tile i + 1 execute.  Every mbarrier wait is bounded: on timeout the CTA
// records an error, waits (bounded) for its own MMAs, frees TMEM and exits.
#include <cfloat>
#include <cstdint>

#include "api_internal.h"
#include "tc_common.cuh"

namespace km2 {

namespace {

constexpr int kThreads = 128;       // one warpgroup
constexpr int kRows = 128;          // points per tile (UMMA M)
constexpr int kStepBytes = kRows * 32;   // one K-step (8 TF32) of a 128-row A tile
constexpr int kWaitTries = 1 << 22;

template <int D>
struct TcCfg {
    static constexpr int KD = (D + 7) / 8;            // data K-steps
    static constexpr int XV = D >= 4 ? 4 : D;         // floats per cp.async copy
    static constexpr int NX = D / XV;                 // copies per point
    static constexpr int FLUSH_TILES = kFlushPoints / kRows;
};

__device__ __forceinline__ float tf32_hi(float v)
{
    return __uint_as_float(__float_as_uint(v) & 0xffffe000u);
}

__device__ __forceinline__ float pack_key(float v, unsigned j)
{
    return __uint_as_float((__float_as_uint(v) & ~31u) | j);
}

struct TcLayout {
    uint32_t a_off;      // 2 stages x 2 parts (hi, lo) x KD steps x kStepBytes
    uint32_t an_off;     // constant norm A tile (kStepBytes)
    uint32_t b_off;      // (2 KD + 1) x npad x 32 bytes: mh_s, ml_s ..., norm
    uint32_t xs_off;     // 2 stages x kRows x D floats (thread-major)
    uint32_t ls_off;     // 2 stages x kRows ints
    uint32_t acc_off;    // k x D int64 + k int32 (optional)
    uint32_t total;
};

__host__ __device__ inline uint32_t align_up(uint32_t v, uint32_t a) { return (v + a - 1) / a * a; }

__host__ __device__ inline TcLayout tc_layout(int D, int KD, int npad, int k, bool with_acc)
{
    TcLayout L;
    uint32_t o = 0;
    L.a_off = o;
    o += 2u * 2u * (uint32_t)KD * kStepBytes;
    L.an_off = o;
    o += kStepBytes;
    L.b_off = o;
    o += (uint32_t)(2 * KD + 1) * (uint32_t)npad * 32u;
    o = align_up(o, 128);
    L.xs_off = o;
    o += 2u * kRows * (uint32_t)D * 4u;
    L.ls_off = o;
    o += 2u * kRows * 4u;
    o = align_up(o, 16);
    L.acc_off = o;
    if (with_acc) o += (uint32_t)k * (uint32_t)D * 8u + (uint32_t)k * 4u;
    L.total = align_up(o, 16);
    return L;
}

template <int D>
__global__ void __launch_bounds__(kThreads)
assign_tc32(const float* __restrict__ X, long long n, Centers c, int* __restrict__ labels,
            StageState* st, Accum acc, int* __restrict__ list, float kappa, float kpack,
            int npad, uint32_t tmem_cols, int use_sacc)
{
    using C = TcCfg<D>;
    constexpr int KD = C::KD;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    __shared__ unsigned long long sq;

    if (st->error) return;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int k = c.k;
    const TcLayout L = tc_layout(D, KD, npad, k, use_sacc != 0);
    unsigned char* sA = smem + L.a_off;
    unsigned char* sAn = smem + L.an_off;
    unsigned char* sB = smem + L.b_off;
    float* xs = reinterpret_cast<float*>(smem + L.xs_off);
    int* ls = reinterpret_cast<int*>(smem + L.ls_off);
    long long* sacc = reinterpret_cast<long long*>(smem + L.acc_off);
    int* scnt = reinterpret_cast<int*>(sacc + (size_t)k * D);
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    const int mode = st->mode;
    const float scaleF = st->scaleF, scaleG = st->scaleG;
    const float thr_base = 2.0f * st->cmax2;
    const uint32_t idesc = tc::instr_desc(2u, (uint32_t)npad, (uint32_t)kRows);

    // ---- B operand: -2c split in TF32 hi / lo per K-step, then ||c||^2 hi / lo
    const int bitems = npad * (2 * KD + 1) * 2;        // (row, tile, chunk)
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
            const float nrm = j < k ? c.cnorm[j] : 1e30f;   // padding center: never the best
            const float h = tf32_hi(nrm);
            v[0] = h;
            v[1] = nrm - h;
        }
        *reinterpret_cast<float4*>(sB + (size_t)tile * npad * 32 + tc::tile_offset(j, kc)) =
            make_float4(v[0], v[1], v[2], v[3]);
    }
    // constant A column pair [1, 1] for the norm K-step
    *reinterpret_cast<float4*>(sAn + tc::tile_offset(tid, 0)) = make_float4(1.f, 1.f, 0.f, 0.f);
    *reinterpret_cast<float4*>(sAn + tc::tile_offset(tid, 1)) = make_float4(0.f, 0.f, 0.f, 0.f);
    if (use_sacc) {
        for (int e = tid; e < k * D; e += kThreads) sacc[e] = 0;
        for (int e = tid; e < k; e += kThreads) scnt[e] = 0;
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base, tmem_cols);
    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        sq = 0;
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;

    const long long ntiles = (n + kRows - 1) / kRows;
    const long long cnt = (long long)blockIdx.x < ntiles
                              ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

    // cp.async of this thread's own point of local tile i into stage i % 2
    auto prefetch = [&](long long i, unsigned dep) {
        asm volatile("" ::"r"(dep) : "memory");
        if (i < cnt) {
            const long long p = (blockIdx.x + i * gridDim.x) * kRows + tid;
            if (p < n) {
                const int sg = (int)(i & 1);
                const float* src = X + p * D;
#pragma unroll
                for (int q = 0; q < C::NX; ++q) {
                    float* dst = xs + ((size_t)(sg * C::NX + q) * kThreads + tid) * C::XV;
                    if constexpr (C::XV == 4) cp_async16(dst, src + 4 * q);
                    else if constexpr (C::XV == 2) cp_async8(dst, src + 2 * q);
                    else cp_async4(dst, src + q);
                }
                if (mode == kModeDelta) cp_async4(ls + sg * kThreads + tid, labels + p);
            }
        }
        cp_async_commit();
    };

    // split tile i into the A tiles of stage i % 2 and issue its MMAs
    auto produce = [&](long long i, float* xr, int& old) {
        const int sg = (int)(i & 1);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        const long long p = (blockIdx.x + i * gridDim.x) * kRows + tid;
        if (p < n) {
#pragma unroll
            for (int q = 0; q < C::NX; ++q) {
                const float* src = xs + ((size_t)(sg * C::NX + q) * kThreads + tid) * C::XV;
#pragma unroll
                for (int e = 0; e < C::XV; ++e) xr[q * C::XV + e] = src[e];
            }
            old = (mode == kModeDelta) ? ls[sg * kThreads + tid] : -1;
        } else {
#pragma unroll
            for (int t = 0; t < D; ++t) xr[t] = 0.f;
            old = -1;
        }
        unsigned dep = 0;
#pragma unroll
        for (int t = 0; t < D; ++t) dep ^= __float_as_uint(xr[t]);
        prefetch(i + 2, dep ^ (unsigned)old);
#pragma unroll
        for (int s = 0; s < KD; ++s) {
#pragma unroll
            for (int kc = 0; kc < 2; ++kc) {
                float v[4], h[4], l[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int t = 8 * s + 4 * kc + q;
                    v[q] = t < D ? xr[t] : 0.f;
                    h[q] = tf32_hi(v[q]);
                    l[q] = v[q] - h[q];
                }
                const uint32_t off = tc::tile_offset(tid, kc);
                *reinterpret_cast<float4*>(sA + ((size_t)(sg * 2 + 0) * KD + s) * kStepBytes + off) =
                    make_float4(h[0], h[1], h[2], h[3]);
                *reinterpret_cast<float4*>(sA + ((size_t)(sg * 2 + 1) * KD + s) * kStepBytes + off) =
                    make_float4(l[0], l[1], l[2], l[3]);
            }
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            const uint32_t d_tmem = tmem + (uint32_t)(sg * npad);
#pragma unroll
            for (int s = 0; s < KD; ++s) {
                const uint32_t ah = sbase + L.a_off + (uint32_t)(((sg * 2 + 0) * KD + s) * kStepBytes);
                const uint32_t al = sbase + L.a_off + (uint32_t)(((sg * 2 + 1) * KD + s) * kStepBytes);
                const uint32_t bh = sbase + L.b_off + (uint32_t)((2 * s + 0) * npad * 32);
                const uint32_t bl = sbase + L.b_off + (uint32_t)((2 * s + 1) * npad * 32);
                tc::mma_tf32(d_tmem, tc::smem_desc(ah), tc::smem_desc(bh), idesc, s > 0 ? 1u : 0u);
                tc::mma_tf32(d_tmem, tc::smem_desc(ah), tc::smem_desc(bl), idesc, 1u);
                tc::mma_tf32(d_tmem, tc::smem_desc(al), tc::smem_desc(bh), idesc, 1u);
            }
            const uint32_t bn = sbase + L.b_off + (uint32_t)(2 * KD * npad * 32);
            tc::mma_tf32(d_tmem, tc::smem_desc(sbase + L.an_off), tc::smem_desc(bn), idesc, 1u);
            tc::mma_commit(&mbar[sg]);
        }
    };

    prefetch(0, 0u);
    prefetch(1, 0u);
    float xc[D], xn[D];
    int oldc = -1, oldn = -1;
    long long qloc = 0;
    bool failed = false;
    if (cnt > 0) produce(0, xc, oldc);
    for (long long i = 0; i < cnt; ++i) {
        if (i + 1 < cnt) produce(i + 1, xn, oldn);
        const int sg = (int)(i & 1);
        bool ok = tc::mbar_wait(&mbar[sg], (uint32_t)((i >> 1) & 1), kWaitTries);
        if (!__syncthreads_and(ok)) {
            // give up: record the error, let this CTA's own MMAs finish, then leave
            if (tid == 0) atomicExch(&st->error, kErrTimeout);
            tc::mbar_wait(&mbar[sg], (uint32_t)((i >> 1) & 1), kWaitTries);
            if (i + 1 < cnt) tc::mbar_wait(&mbar[sg ^ 1], (uint32_t)(((i + 1) >> 1) & 1), kWaitTries);
            failed = true;
            break;
        }
        tc::fence_after_sync();
        // ---- epilogue of tile i
        const long long p = (blockIdx.x + i * gridDim.x) * kRows + tid;
        const bool valid = p < n;
        float B1 = INFINITY, B2 = INFINITY;
        int BI = 0;
        for (int c0 = 0; c0 < npad; c0 += 32) {
            float v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(sg * npad + c0), v);
            // four independent top-2 chains over interleaved column pairs, then merged
            float q1[4], q2[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { q1[q] = INFINITY; q2[q] = INFINITY; }
#pragma unroll
            for (int j = 0; j < 32; j += 8) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int jj = j + 2 * q;
                    const float k0 = pack_key(v[jj], (unsigned)jj);
                    const float k1 = pack_key(v[jj + 1], (unsigned)jj + 1u);
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
                BI = c0 | (int)(__float_as_uint(b1) & 31u);
            } else {
                B2 = fminf(B2, b1);
            }
        }
        tc::fence_before_sync();
        float xn2 = 0.f;
#pragma unroll
        for (int t = 0; t < D; ++t) xn2 = fmaf(xc[t], xc[t], xn2);
        const float thr = kappa * (thr_base + xn2) + kpack * (fabsf(B1) + fabsf(B2));
        const bool flag = valid && (B2 - B1 <= thr);
        if (mode == kModeFull && valid) {
#pragma unroll
            for (int t = 0; t < D; ++t) qloc += sq_fixed(xc[t], scaleG);
        }
        recheck_append(flag, (int)p, list, &st->recheck_count);
        if (valid && !flag && BI != oldc) {
            const int lab = BI, old = oldc;
#pragma unroll
            for (int t = 0; t < D; ++t) {
                const long long v = to_fixed(xc[t], scaleF);
                if (use_sacc) {
                    atomicAdd(reinterpret_cast<unsigned long long*>(sacc + lab * D + t),
                              (unsigned long long)v);
                    if (old >= 0)
                        atomicAdd(reinterpret_cast<unsigned long long*>(sacc + old * D + t),
                                  (unsigned long long)(-v));
                } else {
                    split_add(acc.s_lo + (long long)lab * D + t, acc.s_hi + (long long)lab * D + t, v);
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
            labels[p] = lab;
        }
        // static flush schedule: at most FLUSH_TILES tiles (2^16 points) per partial
        if (((i + 1) % C::FLUSH_TILES) == 0 || i + 1 == cnt) {
            if (qloc) atomicAdd(&sq, (unsigned long long)qloc);
            qloc = 0;
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
            if (tid == 0) {
                if (sq) split_add(&st->q_lo, &st->q_hi, (long long)sq);
                sq = 0;
            }
            __syncthreads();
        }
#pragma unroll
        for (int t = 0; t < D; ++t) xc[t] = xn[t];
        oldc = oldn;
    }
    (void)failed;
    cp_async_wait_all();
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, tmem_cols);
}

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

template <int D>
int launch_tc(const float* X, long long n, const Centers& c, int* labels, StageState* st,
              const Accum& acc, int* list, cudaStream_t s, int sm_count)
{
    using C = TcCfg<D>;
    const int npad = (c.k + 31) / 32 * 32;
    uint32_t cols = 32;
    while (cols < (uint32_t)(2 * npad)) cols <<= 1;
    const bool with_acc = tc_layout(D, C::KD, npad, c.k, true).total <= 160u * 1024u;
    const TcLayout L = tc_layout(D, C::KD, npad, c.k, with_acc);
    static thread_local int configured_for = -1;
    int dev = 0;
    KM2_CUDA(cudaGetDevice(&dev));
    if (configured_for != dev) {
        KM2_CUDA(cudaFuncSetAttribute(assign_tc32<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      200 * 1024));
        configured_for = dev;
    }
    // CTAs per SM from the kernel's own resources (the occupancy API does not
    // account for tensor-memory kernels the way the hardware schedules them):
    // registers, shared memory (228 KB per SM, 1 KB reserved per CTA), warps,
    // and the 512 TMEM columns each CTA takes `cols` of.
    static thread_local int regs_per_thread = 0;
    if (regs_per_thread == 0) {
        cudaFuncAttributes fa;
        KM2_CUDA(cudaFuncGetAttributes(&fa, assign_tc32<D>));
        regs_per_thread = fa.numRegs > 0 ? fa.numRegs : 255;
    }
    const int by_regs = 65536 / (((regs_per_thread * kThreads) + 255) / 256 * 256);
    const int by_smem = (int)((228u * 1024u) / (L.total + 1024u + 1024u));
    const int by_warps = 64 / (kThreads / 32);
    const int by_tmem = (int)(512u / cols);
    int per_sm = by_regs;
    if (per_sm > by_smem) per_sm = by_smem;
    if (per_sm > by_warps) per_sm = by_warps;
    if (per_sm > by_tmem) per_sm = by_tmem;
    if (per_sm < 1) return KMEANS2_ERR_UNSUPPORTED;
    const long long tiles = (n + kRows - 1) / kRows;
    long long grid = (long long)sm_count * per_sm;
    if (grid > tiles) grid = tiles;
    if (grid < 1) grid = 1;
    ++g_launches;
    assign_tc32<D><<<(int)grid, kThreads, L.total, s>>>(X, n, c, labels, st, acc, list,
                                                        tc32_kappa(C::KD), kPackSlack, npad, cols,
                                                        with_acc ? 1 : 0);
    KM2_CUDA(cudaGetLastError());
    return KMEANS2_OK;
}

}  // namespace

int assign_tc32_supported(int d, int k, const float* X)
{
    if (k < 1 || k > 256) return 0;
    if ((reinterpret_cast<uintptr_t>(X) & 15) != 0) return 0;
    return d == 4 || d == 8 || d == 16 || d == 32;
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
