// assign_bf16.cu -- the precision form: the cross term x.c on the tensor cores
// in BF16 (tcgen05 kind::f16, FP32 accumulation in TMEM), for d a multiple of
// 16 in [16, 128] and any k.  Each operand is split into two BF16 parts,
// x = xh + xl (xh = bf16(x), xl = bf16(x - xh)) and m = -2c = mh + ml, and
// three MMAs per K-step accumulate xh.mh + xh.ml + xl.mh: the error drops from
// 2^-7 |x||c| for plain BF16 to about 2^-15 |x||c| at the price of two extra
// MMAs, which the epilogue-bound kernel hides.  A near tie under the bound is
// re-decided from the FP32 master data in FP64 (recheck_kernel), so the labels
// are the same as in every other form.
//
// Data layout (global, rebuilt per stage / per iteration):
//   Xt : one contiguous block per 128-point tile: the xh tile then the xl
//        tile, each d/16 K-steps of 4 KB in the K-major core-matrix layout
//        (tc_common.cuh);
//   xn2: FP32 ||x||^2 per point (for the error bound);
//   Cb : one contiguous block per chunk of NC centers: the mh then the ml
//        chunk, each d/16 K-steps of NC * 32 bytes.
// One CTA per SM (256 threads).  Thread 0 streams A tiles and B chunks with
// 1-D bulk TMA copies into double-buffered shared memory and issues d/16 MMAs
// (M = 128, N = NC, K = 16) per (tile, chunk) into one of two TMEM
// accumulators; all 8 warps run the epilogue of the previous unit meanwhile:
// warp w reads TMEM lanes 32 (w % 4) .. +31, columns of half w / 4 of the
// chunk, adds ||c||^2 and keeps a packed-key top-2 per row.  At a tile's last
// chunk the two halves are merged through shared memory and warps 0-3 decide
// each row: near-tie flag, label, exact fixed-point cluster sums.  Every
// mbarrier wait is bounded; on timeout the CTA records an error, waits
// (bounded) for its own copies and MMAs, frees TMEM and exits.
#include <cfloat>
#include <cstdint>

#include <cuda_bf16.h>

#include "api_internal.h"
#include "tc_common.cuh"

namespace km2 {

namespace {

constexpr int kThreads = 256;
constexpr int kRows = 128;
constexpr int kWaitTries = 1 << 22;

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

// 1-D bulk copy global -> shared, completion counted on mbar (TMA unit).
__device__ __forceinline__ void bulk_load(void* sdst, const void* gsrc, uint32_t bytes,
                                          uint64_t* mbar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            (uint32_t)__cvta_generic_to_shared(sdst)),
        "l"(gsrc), "r"(bytes), "r"((uint32_t)__cvta_generic_to_shared(mbar))
        : "memory");
}

struct Bf16Args {
    const float* X;          // FP32 master rows (sums, ||x||^2 in full mode)
    const unsigned char* Xt; // BF16 tiles
    const float* xn2;        // FP32 ||x||^2 per point
    const unsigned char* Cb; // BF16 -2c chunks
    long long n;
    int d, k, nc, nch;       // chunk width NC and chunk count
    uint32_t tmem_cols;
    float kappa, kpack;
};

__global__ void __launch_bounds__(kThreads, 1)
assign_bf16(Bf16Args a, Centers c, int* __restrict__ labels, StageState* st, Accum acc,
            int* __restrict__ list)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t barA[2], barB[2], barM[2];
    __shared__ uint32_t tmem_base;
    __shared__ float xb1[kRows], xb2[kRows];
    __shared__ int xbi[kRows];

    if (st->error) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int d = a.d, NC = a.nc, nch = a.nch;
    const uint32_t Ahalf = (uint32_t)kRows * (uint32_t)d * 2u;   // one part of a tile
    const uint32_t Bhalf = (uint32_t)NC * (uint32_t)d * 2u;      // one part of a chunk
    const uint32_t Abytes = 2u * Ahalf, Bbytes = 2u * Bhalf;
    unsigned char* sA = smem;                        // 2 stages x (xh, xl)
    unsigned char* sB = smem + 2 * Abytes;           // 2 stages x (mh, ml)
    const uint32_t sAaddr = (uint32_t)__cvta_generic_to_shared(sA);
    const uint32_t sBaddr = (uint32_t)__cvta_generic_to_shared(sB);
    const int mode = st->mode;
    const float scaleF = st->scaleF, scaleG = st->scaleG;
    const float thr_base = 2.0f * st->cmax2;
    const uint32_t idesc = tc::instr_desc(1u, (uint32_t)NC, (uint32_t)kRows);
    const int ksteps = d / 16;

    if (warp == 0) tc::tmem_alloc(&tmem_base, a.tmem_cols);
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(&barA[s], 1);
            tc::mbar_init(&barB[s], 1);
            tc::mbar_init(&barM[s], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;

    const long long ntiles = (a.n + kRows - 1) / kRows;
    const long long cnt = (long long)blockIdx.x < ntiles
                              ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const long long U = cnt * nch;

    auto issue_loads = [&](long long u) {
        const long long i = u / nch;
        const int ch = (int)(u % nch);
        const long long tile = blockIdx.x + i * gridDim.x;
        if (ch == 0) {
            const int sa = (int)(i & 1);
            mbar_expect_tx(&barA[sa], Abytes);
            bulk_load(sA + (size_t)sa * Abytes, a.Xt + (size_t)tile * Abytes, Abytes, &barA[sa]);
        }
        const int sb = (int)(u & 1);
        mbar_expect_tx(&barB[sb], Bbytes);
        bulk_load(sB + (size_t)sb * Bbytes, a.Cb + (size_t)ch * Bbytes, Bbytes, &barB[sb]);
    };
    // returns false on a timed-out wait
    auto issue_mma = [&](long long u) -> bool {
        const long long i = u / nch;
        const int sa = (int)(i & 1), sb = (int)(u & 1);
        if (!tc::mbar_wait(&barA[sa], (uint32_t)((i >> 1) & 1), kWaitTries)) return false;
        if (!tc::mbar_wait(&barB[sb], (uint32_t)((u >> 1) & 1), kWaitTries)) return false;
        tc::fence_after_sync();
        const uint32_t dt = tmem + (uint32_t)(sb * NC);
        for (int s = 0; s < ksteps; ++s) {
            const uint32_t ah = sAaddr + (uint32_t)sa * Abytes + (uint32_t)s * 4096u;
            const uint32_t bh = sBaddr + (uint32_t)sb * Bbytes + (uint32_t)(s * NC * 32);
            tc::mma_bf16(dt, tc::smem_desc(ah), tc::smem_desc(bh), idesc, s > 0 ? 1u : 0u);
            tc::mma_bf16(dt, tc::smem_desc(ah), tc::smem_desc(bh + Bhalf), idesc, 1u);
            tc::mma_bf16(dt, tc::smem_desc(ah + Ahalf), tc::smem_desc(bh), idesc, 1u);
        }
        tc::mma_commit(&barM[sb]);
        return true;
    };

    bool ok = true;
    bool next_issued = false;        // thread 0: MMA of unit u + 1 issued
    if (tid == 0 && U > 0) {
        issue_loads(0);
        if (U > 1) issue_loads(1);
        ok = issue_mma(0);
    }
    // per-row running top-2 across the chunks of the current tile
    float B1 = INFINITY, B2 = INFINITY;
    int BI = 0;
    const int half = warp >> 2;                 // which half of each chunk's columns
    const int row = 32 * (warp & 3) + lane;     // TMEM lane = tile row
    long long qloc = 0;
    long long u = 0;
    for (; u < U; ++u) {
        next_issued = false;
        if (tid == 0 && ok && u + 1 < U) {
            ok = issue_mma(u + 1);
            next_issued = ok;
        }
        const int sb = (int)(u & 1);
        bool mine = ok && tc::mbar_wait(&barM[sb], (uint32_t)((u >> 1) & 1), kWaitTries);
        if (!__syncthreads_and(mine)) break;
        tc::fence_after_sync();
        if (tid == 0 && u + 2 < U) issue_loads(u + 2);

        const long long i = u / nch;
        const int ch = (int)(u % nch);
        // ---- epilogue of unit u: my half of the chunk's NC columns
        const int cols = NC / 2;
        for (int c0 = 0; c0 < cols; c0 += 32) {
            float v[32];
            const int col = half * cols + c0;          // column within the chunk
            tc::tmem_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(sb * NC + col), v);
            const int j0 = ch * NC + col;              // center index of v[0]
            const float4* cn4 = reinterpret_cast<const float4*>(c.cnorm + j0);
            float q1[4], q2[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { q1[q] = INFINITY; q2[q] = INFINITY; }
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                const float4 cn = __ldg(cn4 + g);
                const float w0 = v[4 * g] + cn.x, w1 = v[4 * g + 1] + cn.y;
                const float w2 = v[4 * g + 2] + cn.z, w3 = v[4 * g + 3] + cn.w;
                const int q = g & 3;
                {
                    const float k0 = pack_key(w0, 4u * g), k1 = pack_key(w1, 4u * g + 1u);
                    const float lo = fminf(k0, k1), hi = fmaxf(k0, k1);
                    q2[q] = fmin3(q2[q], hi, fmaxf(q1[q], lo));
                    q1[q] = fminf(q1[q], lo);
                }
                {
                    const float k0 = pack_key(w2, 4u * g + 2u), k1 = pack_key(w3, 4u * g + 3u);
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
        tc::fence_before_sync();
        if (ch == nch - 1) {
            // merge the two halves of each row, then warps 0-3 decide the row
            if (half == 1) { xb1[row] = B1; xb2[row] = B2; xbi[row] = BI; }
            __syncthreads();
            if (half == 0) {
                const float o1 = xb1[row], o2 = xb2[row];
                const int oi = xbi[row];
                if (o1 < B1 || (o1 == B1 && oi < BI)) {
                    B2 = fminf(B1, o2);
                    B1 = o1;
                    BI = oi;
                } else {
                    B2 = fminf(B2, o1);
                }
                const long long p = (blockIdx.x + i * gridDim.x) * kRows + row;
                const bool valid = p < a.n;
                if ((i & 255) == 255) {
                    // keep each ||x||^2 partial below 2^62: fold it every 256 tiles
                    long long qs = qloc;
                    for (int o = 16; o; o >>= 1) qs += __shfl_xor_sync(0xffffffffu, qs, o);
                    if (lane == 0 && qs) split_add(&st->q_lo, &st->q_hi, qs);
                    qloc = 0;
                }
                const float xx = valid ? __ldg(a.xn2 + p) : 0.0f;
                const float thr = a.kappa * (thr_base + xx) + a.kpack * (fabsf(B1) + fabsf(B2));
                const bool flag = valid && (B2 - B1 <= thr);
                recheck_append(flag, (int)p, list, &st->recheck_count);
                const float* xr = a.X + p * d;
                if (mode == kModeFull && valid)
                    for (int t = 0; t < d; ++t) qloc += sq_fixed(__ldg(xr + t), scaleG);
                if (valid && !flag) {
                    const int old = (mode == kModeDelta) ? labels[p] : -1;
                    if (BI != old) {
                        for (int t = 0; t < d; ++t) {
                            const long long val = to_fixed(__ldg(xr + t), scaleF);
                            split_add(acc.s_lo + (long long)BI * d + t, acc.s_hi + (long long)BI * d + t, val);
                            if (old >= 0)
                                split_add(acc.s_lo + (long long)old * d + t,
                                          acc.s_hi + (long long)old * d + t, -val);
                        }
                        atomicAdd(acc.cnt + BI, 1ull);
                        if (old >= 0) atomicAdd(acc.cnt + old, ~0ull);
                        labels[p] = BI;
                    }
                }
            }
            B1 = INFINITY;
            B2 = INFINITY;
            BI = 0;
        }
        __syncthreads();
    }
    if (u < U) {
        // a wait gave up: record it, let this CTA's own copies and MMAs finish, then leave
        if (tid == 0) {
            atomicExch(&st->error, kErrTimeout);
            tc::mbar_wait(&barM[u & 1], (uint32_t)((u >> 1) & 1), kWaitTries);
            if (u + 1 < U) {
                const long long v = u + 1, vi = v / nch;
                tc::mbar_wait(&barB[v & 1], (uint32_t)((v >> 1) & 1), kWaitTries);
                if (v % nch == 0) tc::mbar_wait(&barA[vi & 1], (uint32_t)((vi >> 1) & 1), kWaitTries);
                if (next_issued) tc::mbar_wait(&barM[v & 1], (uint32_t)((v >> 1) & 1), kWaitTries);
            }
        }
        __syncthreads();
    }
    // one partial of ||x||^2 per warp (warps 0-3 hold them; each is below 2^62)
    for (int o = 16; o; o >>= 1) qloc += __shfl_xor_sync(0xffffffffu, qloc, o);
    if (lane == 0 && qloc) split_add(&st->q_lo, &st->q_hi, qloc);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, a.tmem_cols);
}

// X -> BF16 tiles (K-major core-matrix layout) and FP32 ||x||^2; one warp per row.
__global__ void convert_x_kernel(const float* __restrict__ X, long long n, int d,
                                 unsigned char* __restrict__ Xt, float* __restrict__ xn2,
                                 long long ntiles)
{
    const int lane = threadIdx.x & 31;
    const long long nrows = ntiles * kRows;
    long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const size_t Ahalf = (size_t)kRows * d * 2;
    for (; w < nrows; w += nw) {
        const long long tile = w / kRows;
        const int r = (int)(w - tile * kRows);
        unsigned char* base = Xt + (size_t)tile * 2 * Ahalf;
        float s2 = 0.f;
        for (int t0 = 4 * lane; t0 < d; t0 += 128) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (w < n) v = __ldg(reinterpret_cast<const float4*>(X + w * d + t0));
            s2 = fmaf(v.x, v.x, s2); s2 = fmaf(v.y, v.y, s2);
            s2 = fmaf(v.z, v.z, s2); s2 = fmaf(v.w, v.w, s2);
            const int s = t0 >> 4, kc = (t0 >> 3) & 1, e = t0 & 7;
            __nv_bfloat162 h0 = __floats2bfloat162_rn(v.x, v.y);
            __nv_bfloat162 h1 = __floats2bfloat162_rn(v.z, v.w);
            const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
            __nv_bfloat162 l0 = __floats2bfloat162_rn(v.x - f0.x, v.y - f0.y);
            __nv_bfloat162 l1 = __floats2bfloat162_rn(v.z - f1.x, v.w - f1.y);
            uint2 ph, pl;
            ph.x = *reinterpret_cast<uint32_t*>(&h0);
            ph.y = *reinterpret_cast<uint32_t*>(&h1);
            pl.x = *reinterpret_cast<uint32_t*>(&l0);
            pl.y = *reinterpret_cast<uint32_t*>(&l1);
            const size_t off = (size_t)s * 4096 + tc::tile_offset(r, kc) + e * 2;
            *reinterpret_cast<uint2*>(base + off) = ph;
            *reinterpret_cast<uint2*>(base + Ahalf + off) = pl;
        }
        for (int o = 16; o; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        if (lane == 0 && w < n) xn2[w] = s2;
    }
}

// -2c -> BF16 chunks of NC centers (padding centers are zero).
__global__ void convert_c_kernel(const float* __restrict__ c32, int k, int d, int NC, int nch,
                                 unsigned char* __restrict__ Cb)
{
    const long long total = (long long)nch * NC * d;
    const size_t Bhalf = (size_t)NC * d * 2;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e / d), t = (int)(e - (long long)j * d);
        const int ch = j / NC, jj = j - ch * NC;
        const float m = j < k ? -2.0f * c32[(long long)j * d + t] : 0.0f;
        const int s = t >> 4, kc = (t >> 3) & 1, el = t & 7;
        const __nv_bfloat16 h = __float2bfloat16_rn(m);
        const __nv_bfloat16 l = __float2bfloat16_rn(m - __bfloat162float(h));
        const size_t off = (size_t)ch * 2 * Bhalf + (size_t)s * NC * 32 + tc::tile_offset(jj, kc) + el * 2;
        *reinterpret_cast<__nv_bfloat16*>(Cb + off) = h;
        *reinterpret_cast<__nv_bfloat16*>(Cb + off + Bhalf) = l;
    }
}

}  // namespace

// Per key (derivation in the design notes): with |x - xh - xl| <= 2^-18 |x| and
// |m - mh - ml| <= 2^-18 |m| (two round-to-nearest BF16 steps), the three
// products miss xl.ml, (x - xh - xl) m and (xh + xl)(m - mh - ml): at most
// 3.02 * 2^-18 |x_t||m_t| per dimension, i.e. 6.04 * 2^-18 sum_t |x_t||c_t|.
// The FP32 accumulation of nt = 3d + 1 exact products (truncation assumed):
// nt * 2^-23 (2 |x||c| + ||c||^2); FP32 centers and ||c||^2: 2^-23 |x||c| and
// 2^-23 ||c||^2.  With 2 |x||c| <= X2 + C2 the sum is below k_b (2 C2 + X2).
// Two keys of a gap, 1.0625 slack.
float bf16_kappa(int d)
{
    const double nt = 3.0 * d + 1.0;
    const double a1 = 6.04 * 0x1p-18 + 2.0 * nt * 0x1p-23 + 0x1p-23;   // |x||c|
    const double a2 = nt * 0x1p-23 + 0x1p-23;                            // ||c||^2
    const double kb = fmax(a1 / 2.0, (a1 / 2.0 + a2) / 2.0);
    return (float)(2.0 * kb * 1.0625);
}

int bf16_fits(int d)
{
    return 2 * 2 * 128 * d * 2 + 2 * 2 * 64 * d * 2 <= 200 * 1024;
}

int assign_bf16_supported(int d, int k, const float* X)
{
    (void)k;
    if ((reinterpret_cast<uintptr_t>(X) & 15) != 0) return 0;
    return d >= 16 && d % 16 == 0 && bf16_fits(d);
}

// Chunk width NC in {64, 128, 256} (a divisor of 256, so NC * chunks never
// exceeds k rounded up to 256, the length of the padded ||c||^2 array):
// halved while k fits in half a chunk or the two A and two B stages would
// exceed 200 KB of shared memory.
int bf16_chunk(int d, int k)
{
    int nc = 256;
    while (nc > 64 && nc / 2 >= k) nc /= 2;
    while (nc > 64 && 2 * 2 * 128 * d * 2 + 2 * 2 * nc * d * 2 > 200 * 1024) nc /= 2;
    return nc;
}

size_t bf16_xt_bytes(long long n, int d)
{
    return (size_t)((n + kRows - 1) / kRows) * kRows * (size_t)d * 2 * 2;
}

size_t bf16_cb_bytes(int d, int k)
{
    const int nc = bf16_chunk(d, k);
    const int nch = (k + nc - 1) / nc;
    return (size_t)nch * nc * (size_t)d * 2 * 2;
}

int launch_convert_x_bf16(const float* X, long long n, int d, unsigned char* Xt, float* xn2,
                          cudaStream_t s, int sm_count)
{
    const long long ntiles = (n + kRows - 1) / kRows;
    long long blocks = (ntiles * kRows * 32 + 255) / 256;
    if (blocks > (long long)sm_count * 16) blocks = (long long)sm_count * 16;
    ++g_launches;
    convert_x_kernel<<<(int)blocks, 256, 0, s>>>(X, n, d, Xt, xn2, ntiles);
    KM2_CUDA(cudaGetLastError());
    return KMEANS2_OK;
}

int launch_assign_bf16(const float* X, const unsigned char* Xt, const float* xn2,
                       unsigned char* Cb, long long n, int d, const Centers& c, int* labels,
                       StageState* st, const Accum& acc, int* list, cudaStream_t s, int sm_count)
{
    const int NC = bf16_chunk(d, c.k);
    const int nch = (c.k + NC - 1) / NC;
    // this iteration's centers into BF16 chunks
    {
        const long long total = (long long)nch * NC * d;
        long long blocks = (total + 255) / 256;
        if (blocks > 4096) blocks = 4096;
        ++g_launches;
        convert_c_kernel<<<(int)blocks, 256, 0, s>>>(c.c32, c.k, d, NC, nch, Cb);
        KM2_CUDA(cudaGetLastError());
    }
    uint32_t cols = 32;
    while (cols < (uint32_t)(2 * NC)) cols <<= 1;
    const size_t smem = (size_t)2 * 2 * kRows * d * 2 + (size_t)2 * 2 * NC * d * 2;
    static thread_local int configured_for = -1;
    int dev = 0;
    KM2_CUDA(cudaGetDevice(&dev));
    if (configured_for != dev) {
        KM2_CUDA(cudaFuncSetAttribute(assign_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      210 * 1024));
        configured_for = dev;
    }
    const long long tiles = (n + kRows - 1) / kRows;
    long long grid = sm_count;
    if (grid > tiles) grid = tiles;
    if (grid < 1) grid = 1;
    Bf16Args a;
    a.X = X;
    a.Xt = Xt;
    a.xn2 = xn2;
    a.Cb = Cb;
    a.n = n;
    a.d = d;
    a.k = c.k;
    a.nc = NC;
    a.nch = nch;
    a.tmem_cols = cols;
    a.kappa = bf16_kappa(d);
    a.kpack = kPackSlack;
    ++g_launches;
    assign_bf16<<<(int)grid, kThreads, smem, s>>>(a, c, labels, st, acc, list);
    KM2_CUDA(cudaGetLastError());
    return KMEANS2_OK;
}

}  // namespace km2
