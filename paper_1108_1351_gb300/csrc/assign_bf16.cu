// assign_bf16.cu -- the precision form: the cross term x.c on the tensor cores
// in BF16 (tcgen05 kind::f16, FP32 accumulation in TMEM), for d a multiple of
// 16 in [16, 128] and any k.  Each operand is split into two BF16 parts,
// x = xh + xl (xh = bf16(x), xl = bf16(x - xh)) and m = -2c = mh + ml, and
// three MMAs per K-step accumulate xh.mh + xh.ml + xl.mh: the error drops from
// 2^-7 |x||c| for plain BF16 to about 2^-15 |x||c| at the price of two extra
// MMAs.  A near tie under the bound is re-decided from the FP32 master data in
// FP64 (recheck_kernel), so the labels are the same as in every other form.
//
// Data layout (global, rebuilt per stage / per iteration):
//   Xt : one contiguous block per 128-point tile: the xh tile then the xl
//        tile, each d/16 K-steps of 4 KB in the K-major core-matrix layout
//        (tc_common.cuh);
//   xn2: FP32 ||x||^2 per point (for the error bound);
//   Cb : one contiguous slice per (chunk of NC centers, K-step): the mh then
//        the ml part, NC * 32 bytes each; after a chunk's d/16 data slices a
//        norm slice holds ||c_j||^2 = nh + nm + nl (three exact BF16 parts) in
//        the first three columns of row j, multiplied by a constant A tile of
//        ones, so the accumulator holds ||c||^2 - 2 x.c with no epilogue add.
//
// Warp-specialised pipeline, one CTA per SM, 11 warps:
//   warp 0  A producer: one bulk TMA copy per tile into a 2-stage ring;
//   warp 1  B producer: one bulk TMA copy per ring slot (SB <= 8 slots) of
//           one (chunk, K-step) slice, five of a chunk in the single pass;
//   warp 2  MMA issuer: tiles go in pairs (one per epilogue group and A
//           stage); per (pair, chunk) unit and K-step it issues 3 MMAs
//           (M 128, N NC, K 16) for each tile of the pair into its TMEM
//           accumulator, so each B slice is read from L2 once for 256 points;
//           tcgen05.commit frees each slot and both tiles and hands the
//           accumulators to the epilogues;
//   warps 3-6, 7-10  two epilogue groups taking alternate tiles, each with its
//           own two TMEM accumulators (4 x NC columns in all): a thread owns
//           one row (TMEM lane) of the tile, keeps a packed-key top-2 across
//           the chunks (the next 32 columns load while the current ones are
//           compared) and decides the row (near-tie flag, label, exact
//           fixed-point cluster sums).
// Roles are coupled only by mbarriers (full / empty per ring slot and per
// accumulator), so copies, MMAs and epilogues of different units overlap.
// Every wait is bounded; on timeout the CTA records an error, each role lets
// its own copies or MMAs finish (bounded), TMEM is freed and the CTA exits.
#include <cfloat>
#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "api_internal.h"
#include "tc_common.cuh"

namespace km2 {

namespace {

constexpr int kEpiGroups = 2;
constexpr int kEpiWarps = 4 * kEpiGroups;
constexpr int kThreads = 32 * (3 + kEpiWarps);
constexpr int kRows = 128;
constexpr int kSA = 2;                 // A ring depth (tiles)
constexpr int kMaxSB = 8;              // B ring depth (slices)
constexpr int kSmemBudget = 226 * 1024;    // dynamic + static shared memory of the CTA
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

__device__ __forceinline__ void mbar_arrive(uint64_t* mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(mbar))
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
    const long long* n_dev;  // when set, the row count is read here (n is its bound)
    const unsigned char* Xt; // BF16 tiles
    const float* xn2;        // FP32 ||x||^2 per point
    const unsigned char* Cb; // BF16 -2c slices
    long long n;
    int d, k, nc, nch, sb;   // chunk width NC, chunk count, B ring depth (slots)
    int kps;                 // K-steps per B ring slot
    int lab_bulk;            // old labels can be bulk-copied (16-byte aligned)
    uint32_t tmem_cols;
    float kappa, kpack;
    float kabs;              // single-pass form: coefficient of the bound's absolute term
    int ctries;              // wait limit of the consumer roles (MMA issuer, epilogue)
};

// Scales of the single-pass FP16 operands: x as x 2^-a with a = E - 14, where
// max|x| < 2^E (the stage's recorded max|x|), and m = -2c as m 2^-b with
// b = Em + 1 - 14, where 2 sqrt(C2) < 2^Em for C2 = st->cmax2 >= max_j
// ||c_j||^2 (one extra bit covers the rounding of sqrtf).  Every scaled operand
// stays below 2^14 in magnitude, inside the FP16 range; the accumulator then
// holds D 2^-(a + b), whose argmin is D's.  The conversion kernels and the
// epilogue derive a, b and E the same way.
__device__ __forceinline__ void f16_scales(const StageState* st, int& ea, int& eb, int& E)
{
    E = 0;
    const float mx = __uint_as_float(st->maxabs_bits);
    if (mx > 0.0f) frexpf(mx, &E);
    ea = E - 14;
    int em = 0;
    frexpf(2.0f * sqrtf(st->cmax2), &em);
    eb = em + 1 - 14;
}

// Accumulators per epilogue group: two (MMAs of the next chunk overlap the
// epilogue of this one) while 2 groups x 2 x NC columns fit in TMEM's 512;
// one for NC = 256 (the wider MMAs then alternate with the epilogue).
template <int NC>
constexpr int kAccBufs = NC >= 256 ? 1 : 2;

constexpr int kSR = 4;                 // side ring depth (tiles): ||x||^2 and old labels
constexpr int kRecheckQ = 256;         // flagged points staged per epilogue warp

struct Bars {
    uint64_t a_full[kSA], a_empty[kSA];
    uint64_t b_full[kMaxSB], b_empty[kMaxSB];
    uint64_t acc_full[2 * kEpiGroups], acc_empty[2 * kEpiGroups];
    uint64_t side_full[kSR], side_empty[kSR];
    uint64_t drain;
};

// Per-tile values the row decisions need, loaded with each tile by bulk
// copies, whose shared-memory destinations must be 16-byte aligned.
struct __align__(128) SideRing {
    float xn2[kSR][kRows];
    int lab[kSR][kRows];
};
static_assert(sizeof(float) * kRows % 16 == 0, "side ring rows must keep 16-byte alignment");

// Static shared memory of the kernel (barriers, side ring, recheck queues),
// rounded up; the dynamic part must fit beside it.
constexpr int kStaticSmem = 16 * 1024;
static_assert(sizeof(Bars) + sizeof(SideRing) + kEpiWarps * kRecheckQ * 4 + 64 <= kStaticSmem,
              "static shared memory estimate too small");

// Bounded wait for the phase of `parity`; gives up early once another role
// has aborted.  On its own timeout it raises the abort flag and the error.
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
// folded into the running (B1, B2, BI) of a row.  Eight independent chains
// of two column pairs each keep the dependent path short.
__device__ __forceinline__ void top2_cols(const uint32_t* r, int j0, float& B1, float& B2, int& BI)
{
    float q1[8], q2[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) { q1[q] = INFINITY; q2[q] = INFINITY; }
#pragma unroll
    for (int j = 0; j < 32; j += 16) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int jj = j + 2 * q;
            const float k0 = pack_key(__uint_as_float(r[jj]), (unsigned)jj);
            const float k1 = pack_key(__uint_as_float(r[jj + 1]), (unsigned)jj + 1u);
            const float lo = fminf(k0, k1), hi = fmaxf(k0, k1);
            q2[q] = fmin3(q2[q], hi, fmaxf(q1[q], lo));
            q1[q] = fminf(q1[q], lo);
        }
    }
    // pairwise merge of the chains: (a1, a2) + (b1, b2) -> (min, second)
#pragma unroll
    for (int w = 4; w >= 1; w >>= 1) {
#pragma unroll
        for (int q = 0; q < w; ++q) {
            const float m = fmin3(q2[q], q2[q + w], fmaxf(q1[q], q1[q + w]));
            q1[q] = fminf(q1[q], q1[q + w]);
            q2[q] = m;
        }
    }
    const float b1 = q1[0], b2 = q2[0];
    if (b1 < B1) {
        B2 = fminf(B1, b2);
        B1 = b1;
        BI = j0 + (int)(__float_as_uint(b1) & 31u);
    } else {
        B2 = fminf(B2, b1);
    }
}

// SINGLE = 0: split BF16 (two parts per operand, three MMAs per K-step);
// SINGLE = 1: one FP16 part per operand (scaled, f16_scales), one MMA per K-step.
// The norm slice is BF16 in both (its own MMA against the BF16 ones tile).
template <int NC, int SINGLE>
__global__ void __launch_bounds__(kThreads, 1)
assign_bf16(Bf16Args a, Centers c, int* __restrict__ labels, StageState* st, Accum acc,
            int* __restrict__ list)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ Bars bars;
    __shared__ __align__(128) SideRing side;
    __shared__ int rqs[kEpiWarps][kRecheckQ];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    if (st->error) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int d = a.d, nch = a.nch, SB = a.sb;
    const long long n = a.n_dev ? min(*a.n_dev, a.n) : a.n;
    const int ctries = a.ctries;
    const int mode = st->mode;
    const bool lab_bulk = a.lab_bulk != 0 && mode == kModeDelta;
    const int ksteps = d / 16;
    const int kslices = ksteps + 1;                              // data K-steps + the norm slice
    constexpr uint32_t kParts = SINGLE ? 1u : 2u;                // operand parts
    const uint32_t Ahalf = (uint32_t)ksteps * 4096u;             // one part of a tile
    const uint32_t Abytes = kParts * Ahalf;
    // A slot of the B ring holds kps consecutive (chunk, K-step) slices of one
    // chunk (contiguous in Cb): one bulk copy and one commit per slot, so the
    // commits per chunk drop from d/16 + 1 to (d/16 + 1) / kps.  The split
    // form keeps one slice per slot (a compile-time 1, no extra issuer work).
    const int kPerSlot = SINGLE ? a.kps : 1;
    const uint32_t Kbytes = (uint32_t)NC * 32u * kParts;         // one (chunk, K-step) slice
    const uint32_t Sbytes = Kbytes * (uint32_t)kPerSlot;         // one slot of the B ring
    const int kunits = (kslices + kPerSlot - 1) / kPerSlot;      // slots per chunk
    unsigned char* sA = smem;                                    // kSA x Abytes
    unsigned char* sB = smem + kSA * Abytes;                     // SB x Sbytes
    unsigned char* sOnes = sB + (size_t)SB * Sbytes;             // 128 x 16 BF16: [1, 1, 1, 0, ...]
    const uint32_t sAaddr = (uint32_t)__cvta_generic_to_shared(sA);
    const uint32_t sBaddr = (uint32_t)__cvta_generic_to_shared(sB);
    const uint32_t sOnesAddr = (uint32_t)__cvta_generic_to_shared(sOnes);
    volatile int* abort_v = &abort_flag;

    // constant A tile of the norm K-step: row r = [1, 1, 1, 0, ..., 0] (BF16)
    if (tid < kRows) {
        *reinterpret_cast<uint4*>(sOnes + tc::tile_offset(tid, 0)) =
            make_uint4(0x3f803f80u, 0x00003f80u, 0u, 0u);
        *reinterpret_cast<uint4*>(sOnes + tc::tile_offset(tid, 1)) = make_uint4(0u, 0u, 0u, 0u);
    }
    tc::fence_proxy_async();
    if (warp == 2) tc::tmem_alloc(&tmem_base, a.tmem_cols);
    if (tid == 0) {
        for (int s = 0; s < kSA; ++s) {
            tc::mbar_init(&bars.a_full[s], 1);
            tc::mbar_init(&bars.a_empty[s], 1);
        }
        for (int s = 0; s < kMaxSB; ++s) {
            tc::mbar_init(&bars.b_full[s], 1);
            tc::mbar_init(&bars.b_empty[s], 1);
        }
        for (int b = 0; b < 2 * kEpiGroups; ++b) {
            tc::mbar_init(&bars.acc_full[b], 1);
            tc::mbar_init(&bars.acc_empty[b], 4);   // the 4 warps of the owning group
        }
        for (int r = 0; r < kSR; ++r) {
            tc::mbar_init(&bars.side_full[r], 1);
            tc::mbar_init(&bars.side_empty[r], 4);  // the 4 warps of the consuming group
        }
        tc::mbar_init(&bars.drain, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;

    const long long ntiles = (n + kRows - 1) / kRows;
    const long long cnt = (long long)blockIdx.x < ntiles
                              ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

    if (warp == 0) {
        // ---------------- A producer: tile i -> stage i % 2
        if (lane == 0) {
            long long issued = 0;
            for (long long i = 0; i < cnt; ++i) {
                const int s = (int)(i & 1), r = (int)(i % kSR);
                if (!wait_bar(&bars.a_empty[s], (uint32_t)(((i >> 1) & 1) ^ 1), abort_v, st)) break;
                if (!wait_bar(&bars.side_empty[r], (uint32_t)(((i / kSR) & 1) ^ 1), abort_v, st)) break;
                const long long tile = blockIdx.x + i * gridDim.x;
                mbar_expect_tx(&bars.a_full[s], Abytes);
                bulk_load(sA + (size_t)s * Abytes, a.Xt + (size_t)tile * Abytes, Abytes,
                          &bars.a_full[s]);
                // ||x||^2 and old labels of the tile's first rows & ~3 points
                const long long rows = n - tile * kRows < kRows ? n - tile * kRows : kRows;
                const uint32_t vb = (uint32_t)(rows & ~3ll) * 4u;
                const uint32_t lb = lab_bulk ? vb : 0u;
                mbar_expect_tx(&bars.side_full[r], vb + lb);
                if (vb) bulk_load(side.xn2[r], a.xn2 + tile * kRows, vb, &bars.side_full[r]);
                if (lb) bulk_load(side.lab[r], labels + tile * kRows, lb, &bars.side_full[r]);
                issued = i + 1;
            }
            // let this CTA's own copies land before it can exit
            for (long long i = issued > kSA ? issued - kSA : 0; i < issued; ++i)
                tc::mbar_wait(&bars.a_full[i & 1], (uint32_t)((i >> 1) & 1), kWaitTries);
            for (long long i = issued > kSR ? issued - kSR : 0; i < issued; ++i)
                tc::mbar_wait(&bars.side_full[i % kSR], (uint32_t)((i / kSR) & 1), kWaitTries);
        }
    } else if (warp == 1) {
        // ---------------- B producer: slot q = (pair, chunk, K-step group) -> stage q % SB
        if (lane == 0) {
            // slices go once per PAIR of tiles (both tiles' MMAs read each slice)
            const long long total = ((cnt + 1) / 2) * nch * kunits;
            long long q = 0;
            for (; q < total; ++q) {
                const int slot = (int)(q % SB);
                if (!wait_bar(&bars.b_empty[slot], (uint32_t)(((q / SB) & 1) ^ 1), abort_v, st))
                    break;
                const long long unit = q / kunits;
                const int ch = (int)(unit % nch), ks0 = (int)(q % kunits) * kPerSlot;
                const uint32_t bytes = Kbytes * (uint32_t)min(kPerSlot, kslices - ks0);
                mbar_expect_tx(&bars.b_full[slot], bytes);
                bulk_load(sB + (size_t)slot * Sbytes, a.Cb + ((size_t)ch * kslices + ks0) * Kbytes,
                          bytes, &bars.b_full[slot]);
            }
            for (long long r = q > SB ? q - SB : 0; r < q; ++r)
                tc::mbar_wait(&bars.b_full[r % SB], (uint32_t)((r / SB) & 1), kWaitTries);
        }
    } else if (warp == 2) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tc::instr_desc(1u, (uint32_t)NC, (uint32_t)kRows);     // BF16
            const uint32_t idesc16 = tc::instr_desc(0u, (uint32_t)NC, (uint32_t)kRows);   // FP16
            uint32_t phase = 0u;             // bit b: parity of accumulator b's next use
            long long q = 0;
            bool ok = true;
            // tiles go in pairs (2 pr -> A stage 0 and epilogue group 0, 2 pr + 1 ->
            // stage 1 and group 1): each B slice feeds both tiles' MMAs
            const long long npairs = (cnt + 1) / 2;
            for (long long pr = 0; pr < npairs && ok; ++pr) {
                const bool two = 2 * pr + 1 < cnt;
                const uint32_t par = (uint32_t)(pr & 1);
                if (!(ok = wait_bar(&bars.a_full[0], par, abort_v, st, ctries))) break;
                if (two && !(ok = wait_bar(&bars.a_full[1], par, abort_v, st, ctries))) break;
                tc::fence_after_sync();
                for (int ch = 0; ch < nch && ok; ++ch) {
                    const int b0 = ch % kAccBufs<NC>, b1 = kAccBufs<NC> + ch % kAccBufs<NC>;
                    if (!(ok = wait_bar(&bars.acc_empty[b0], ((phase >> b0) & 1u) ^ 1u, abort_v, st, ctries))) break;
                    if (two && !(ok = wait_bar(&bars.acc_empty[b1], ((phase >> b1) & 1u) ^ 1u, abort_v, st, ctries)))
                        break;
                    tc::fence_after_sync();
                    const uint32_t d0 = tmem + (uint32_t)(b0 * NC), d1 = tmem + (uint32_t)(b1 * NC);
                    for (int u = 0; u < kunits; ++u, ++q) {
                        const int slot = (int)(q % SB);
                        if (!(ok = wait_bar(&bars.b_full[slot], (uint32_t)((q / SB) & 1), abort_v, st, ctries)))
                            break;
                        tc::fence_after_sync();
                        const int ks0 = u * kPerSlot, ks1 = min(ks0 + kPerSlot, kslices);
                        for (int ks = ks0; ks < ks1; ++ks) {
                            const uint32_t bh = sBaddr + (uint32_t)slot * Sbytes + (uint32_t)(ks - ks0) * Kbytes;
                            if (ks < ksteps && SINGLE) {
#pragma unroll
                                for (int t = 0; t < 2; ++t) {
                                    if (t == 1 && !two) break;
                                    const uint32_t dt = t ? d1 : d0;
                                    const uint32_t ah = sAaddr + (uint32_t)t * Abytes + (uint32_t)ks * 4096u;
                                    tc::mma_bf16(dt, tc::smem_desc(ah), tc::smem_desc(bh), idesc16, ks > 0 ? 1u : 0u);
                                }
                            } else if (ks < ksteps) {
                                const uint32_t bl = bh + (uint32_t)NC * 32u;
#pragma unroll
                                for (int t = 0; t < 2; ++t) {
                                    if (t == 1 && !two) break;
                                    const uint32_t dt = t ? d1 : d0;
                                    const uint32_t ah = sAaddr + (uint32_t)t * Abytes + (uint32_t)ks * 4096u;
                                    tc::mma_bf16(dt, tc::smem_desc(ah), tc::smem_desc(bh), idesc, ks > 0 ? 1u : 0u);
                                    tc::mma_bf16(dt, tc::smem_desc(ah), tc::smem_desc(bl), idesc, 1u);
                                    tc::mma_bf16(dt, tc::smem_desc(ah + Ahalf), tc::smem_desc(bh), idesc, 1u);
                                }
                            } else {
                                // + ||c||^2: ones x (nh, nm, nl)
                                tc::mma_bf16(d0, tc::smem_desc(sOnesAddr), tc::smem_desc(bh), idesc, 1u);
                                if (two) tc::mma_bf16(d1, tc::smem_desc(sOnesAddr), tc::smem_desc(bh), idesc, 1u);
                            }
                        }
                        tc::mma_commit(&bars.b_empty[slot]);
                    }
                    if (!ok) break;
                    tc::mma_commit(&bars.acc_full[b0]);
                    phase ^= 1u << b0;
                    if (two) {
                        tc::mma_commit(&bars.acc_full[b1]);
                        phase ^= 1u << b1;
                    }
                }
                if (ok) {
                    tc::mma_commit(&bars.a_empty[0]);
                    if (two) tc::mma_commit(&bars.a_empty[1]);
                }
            }
            // every MMA issued by this thread has completed once `drain` flips
            tc::mma_commit(&bars.drain);
            tc::mbar_wait(&bars.drain, 0u, kWaitTries);
        }
    } else {
        // ---------------- epilogue group g: tiles i = g, g + 2, ...
        const int ew = warp - 3;
        const int g = ew >> 2;
        const int quarter = warp & 3;                     // TMEM lanes 32 * (warp % 4) ...
        const int row = 32 * quarter + lane;
        const uint32_t lane_addr = (uint32_t)(32 * quarter) << 16;
        const float scaleF = st->scaleF;
        const float thr_base = 2.0f * st->cmax2;
        // single-pass form: the keys are D 2^-(ea + eb); the bound is formed in
        // unscaled units (with its floor) and scaled the same way
        const float tabs = tie_abs(SINGLE ? d + 3 : 3 * d + 3);   // products per key
        int kexp = 0;
        float kabs = 0.0f;
        if (SINGLE) {
            int ea, eb, E;
            f16_scales(st, ea, eb, E);
            kexp = -(ea + eb);
            kabs = ldexpf(a.kabs, 2 * E + kexp) + ldexpf(a.kabs * st->cmax2, kexp) + tabs;
        }
        int* rq = rqs[ew];
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
        uint32_t phase = 0u;                 // bit s: parity of accumulator 2 g + s's next use
        bool ok = true;
        for (long long i = g; i < cnt && ok; i += kEpiGroups) {
            float B1 = INFINITY, B2 = INFINITY;
            int BI = 0;
            for (int ch = 0; ch < nch; ++ch) {
                const int b = g * kAccBufs<NC> + ch % kAccBufs<NC>;
                bool w = wait_bar(&bars.acc_full[b], (phase >> (ch % kAccBufs<NC>)) & 1u, abort_v,
                                  st, ctries);
                if (!__all_sync(0xffffffffu, w)) { ok = false; break; }
                tc::fence_after_sync();
                // 32 columns at a time through three register buffers: block i + 2
                // loads while block i is compared, and the accumulator is handed
                // back to the MMA issuer as soon as its last block is in registers
                // (the last two blocks are compared after that).
                constexpr int NB = NC / 32;
                uint32_t rr[3][32];
                const uint32_t cb = tmem + lane_addr + (uint32_t)(b * NC);
                auto release = [&]() {
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&bars.acc_empty[b]);
                };
                tc::tmem_ld32_async(cb, rr[0]);
                if (NB > 1) tc::tmem_ld32_async(cb + 32u, rr[1]);
                tc::tmem_wait_ld();
                if (NB <= 2) release();
#pragma unroll
                for (int i = 0; i < NB; ++i) {
                    if (i + 2 < NB) tc::tmem_ld32_async(cb + (uint32_t)(32 * (i + 2)), rr[(i + 2) % 3]);
                    top2_cols(rr[i % 3], ch * NC + 32 * i, B1, B2, BI);
                    if (i + 2 < NB) {
                        tc::tmem_wait_ld();
                        if (i + 3 == NB) release();
                    }
                }
                phase ^= 1u << (ch % kAccBufs<NC>);
            }
            if (!ok) break;
            // ---- decide row `row` of tile i
            const long long tile = blockIdx.x + i * gridDim.x;
            const long long p = tile * kRows + row;
            const bool valid = p < n;
            const int r = (int)(i % kSR);
            {
                const bool w = wait_bar(&bars.side_full[r], (uint32_t)((i / kSR) & 1), abort_v, st, ctries);
                if (!__all_sync(0xffffffffu, w)) break;
            }
            const bool in_ring = (long long)row < ((n - tile * kRows) & ~3ll);
            const float xx = valid ? (in_ring ? side.xn2[r][row] : __ldg(a.xn2 + p)) : 0.0f;
            const float thr = ldexpf(a.kappa * (thr_base + xx) + tabs, kexp) + kabs +
                              a.kpack * (fabsf(B1) + fabsf(B2));
            const bool flag = valid && (B2 - B1 <= thr);
            {
                const unsigned m = __ballot_sync(0xffffffffu, flag);
                if (m) {
                    if (rq_n + 32 > kRecheckQ) rq_flush();
                    if (flag) rq[rq_n + __popc(m & lanemask_lt())] = (int)p;
                    rq_n += __popc(m);
                }
            }
            int old = -1;
            if (mode == kModeDelta && valid)
                old = (lab_bulk && in_ring) ? side.lab[r][row] : labels[p];
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars.side_empty[r]);
            const bool moved = valid && !flag && label_ok(BI, a.k, st) && old_label_ok(old, a.k, st) &&
                               BI != old;
            if (moved) {
                atomicAdd(acc.cnt + BI, 1ull);
                if (old >= 0) atomicAdd(acc.cnt + old, ~0ull);
                labels[p] = BI;
            }
            // Sums: one moved row at a time, the warp's lanes over its
            // coordinates, so each atomic instruction touches a few contiguous
            // lines of s_lo / s_hi and each row is read coalesced.
            const unsigned mmov = __ballot_sync(0xffffffffu, moved);
            for (unsigned m = mmov; m; m &= m - 1) {
                const int src = __ffs(m) - 1;
                const long long pj = __shfl_sync(0xffffffffu, p, src);
                const int bj = __shfl_sync(0xffffffffu, BI, src);
                const int oj = __shfl_sync(0xffffffffu, old, src);
                const float* xr = a.X + pj * d;
                for (int t = lane; t < d; t += 32) {
                    const long long val = to_fixed(__ldg(xr + t), scaleF);
                    split_add(acc.s_lo + (long long)bj * d + t, acc.s_hi + (long long)bj * d + t, val);
                    if (oj >= 0)
                        split_add(acc.s_lo + (long long)oj * d + t,
                                  acc.s_hi + (long long)oj * d + t, -val);
                }
            }
        }
        rq_flush();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 2) tc::tmem_dealloc(tmem, a.tmem_cols);
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

// -2c -> BF16 slices: for each chunk of NC centers and K-step, the mh part then
// the ml part (NC * 32 bytes each); padding centers are zero.
__global__ void convert_c_kernel(const float* __restrict__ c32, int k, int d, int NC, int nch,
                                 unsigned char* __restrict__ Cb)
{
    const long long total = (long long)nch * NC * d;
    const int kslices = d / 16 + 1;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e / d), t = (int)(e - (long long)j * d);
        const int ch = j / NC, jj = j - ch * NC;
        const float m = j < k ? -2.0f * c32[(long long)j * d + t] : 0.0f;
        const int s = t >> 4, kc = (t >> 3) & 1, el = t & 7;
        const __nv_bfloat16 h = __float2bfloat16_rn(m);
        const __nv_bfloat16 l = __float2bfloat16_rn(m - __bfloat162float(h));
        const size_t off = ((size_t)ch * kslices + s) * NC * 64 + tc::tile_offset(jj, kc) + el * 2;
        *reinterpret_cast<__nv_bfloat16*>(Cb + off) = h;
        *reinterpret_cast<__nv_bfloat16*>(Cb + off + (size_t)NC * 32) = l;
    }
}

// Norm slice of every chunk: row j = [nh, nm, nl, 0, ...] with nh + nm + nl =
// ||c_j||^2 up to 2^-27 relative (three round-to-nearest BF16 parts of the FP32
// value, each residual exact in FP32); its ml half and the other columns are
// zero.  A padding center gets the largest finite BF16, so it never wins.
__global__ void convert_norm_kernel(const float* __restrict__ cnorm, int k, int d, int NC, int nch,
                                    unsigned char* __restrict__ Cb)
{
    const int kslices = d / 16 + 1;
    const int total = nch * NC;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < total; j += gridDim.x * blockDim.x) {
        const int ch = j / NC, jj = j - ch * NC;
        const float nrm = j < k ? cnorm[j] : 3.3895313892515355e38f;
        const __nv_bfloat16 nh = __float2bfloat16_rn(nrm);
        const float r1 = nrm - __bfloat162float(nh);
        const __nv_bfloat16 nm = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(nm);
        const __nv_bfloat16 nl = __float2bfloat16_rn(r2);
        unsigned char* base = Cb + ((size_t)ch * kslices + (kslices - 1)) * NC * 64;
        uint4 v0;
        v0.x = (uint32_t)__bfloat16_as_ushort(nh) | ((uint32_t)__bfloat16_as_ushort(nm) << 16);
        v0.y = (uint32_t)__bfloat16_as_ushort(nl);
        v0.z = 0u;
        v0.w = 0u;
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(base + tc::tile_offset(jj, 0)) = v0;
        *reinterpret_cast<uint4*>(base + tc::tile_offset(jj, 1)) = z;
        *reinterpret_cast<uint4*>(base + (size_t)NC * 32 + tc::tile_offset(jj, 0)) = z;
        *reinterpret_cast<uint4*>(base + (size_t)NC * 32 + tc::tile_offset(jj, 1)) = z;
    }
}


// Single-pass form: X -> one FP16 part per tile, x 2^-ea (f16_scales), in the
// K-major core-matrix layout, and FP32 ||x||^2 (unscaled); one warp per row.
__global__ void convert_x_f16_kernel(const float* __restrict__ X, long long n, int d,
                                     unsigned char* __restrict__ Xt, float* __restrict__ xn2,
                                     long long ntiles, const StageState* st)
{
    const int lane = threadIdx.x & 31;
    int ea, eb, E;
    f16_scales(st, ea, eb, E);
    const long long nrows = ntiles * kRows;
    long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const size_t Apart = (size_t)kRows * d * 2;
    for (; w < nrows; w += nw) {
        const long long tile = w / kRows;
        const int r = (int)(w - tile * kRows);
        unsigned char* base = Xt + (size_t)tile * Apart;
        float s2 = 0.f;
        for (int t0 = 4 * lane; t0 < d; t0 += 128) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (w < n) v = __ldg(reinterpret_cast<const float4*>(X + w * d + t0));
            s2 = fmaf(v.x, v.x, s2); s2 = fmaf(v.y, v.y, s2);
            s2 = fmaf(v.z, v.z, s2); s2 = fmaf(v.w, v.w, s2);
            const int ks = t0 >> 4, kc = (t0 >> 3) & 1, e = t0 & 7;
            const __half2 h0 = __floats2half2_rn(ldexpf(v.x, -ea), ldexpf(v.y, -ea));
            const __half2 h1 = __floats2half2_rn(ldexpf(v.z, -ea), ldexpf(v.w, -ea));
            uint2 ph;
            ph.x = *reinterpret_cast<const uint32_t*>(&h0);
            ph.y = *reinterpret_cast<const uint32_t*>(&h1);
            *reinterpret_cast<uint2*>(base + (size_t)ks * 4096 + tc::tile_offset(r, kc) + e * 2) = ph;
        }
        for (int o = 16; o; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        if (lane == 0 && w < n) xn2[w] = s2;
    }
}

// Single-pass form: -2c 2^-eb -> FP16 slices (NC * 32 bytes per chunk and
// K-step); padding centers are zero.
__global__ void convert_c_f16_kernel(const float* __restrict__ c32, int k, int d, int NC, int nch,
                                     unsigned char* __restrict__ Cb, const StageState* st)
{
    int ea, eb, E;
    f16_scales(st, ea, eb, E);
    const long long total = (long long)nch * NC * d;
    const int kslices = d / 16 + 1;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e / d), t = (int)(e - (long long)j * d);
        const int ch = j / NC, jj = j - ch * NC;
        const float m = j < k ? -2.0f * c32[(long long)j * d + t] : 0.0f;
        const int ks = t >> 4, kc = (t >> 3) & 1, el = t & 7;
        const size_t off = ((size_t)ch * kslices + ks) * NC * 32 + tc::tile_offset(jj, kc) + el * 2;
        *reinterpret_cast<__half*>(Cb + off) = __float2half_rn(ldexpf(m, -eb));
    }
}

// Single-pass form: the norm slice of every chunk, ||c_j||^2 2^-(ea + eb) as
// three BF16 parts in the first columns of row j (BF16 operands: the norm MMA
// runs with a BF16 instruction descriptor against the BF16 ones tile).
__global__ void convert_norm_single_kernel(const float* __restrict__ cnorm, int k, int d, int NC,
                                           int nch, unsigned char* __restrict__ Cb,
                                           const StageState* st)
{
    int ea, eb, E;
    f16_scales(st, ea, eb, E);
    const int kslices = d / 16 + 1;
    const int total = nch * NC;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < total; j += gridDim.x * blockDim.x) {
        const int ch = j / NC, jj = j - ch * NC;
        const float nrm = j < k ? ldexpf(cnorm[j], -(ea + eb)) : 3.3895313892515355e38f;
        const __nv_bfloat16 nh = __float2bfloat16_rn(nrm);
        const float r1 = nrm - __bfloat162float(nh);
        const __nv_bfloat16 nm = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(nm);
        const __nv_bfloat16 nl = __float2bfloat16_rn(r2);
        unsigned char* base = Cb + ((size_t)ch * kslices + (kslices - 1)) * NC * 32;
        uint4 v0;
        v0.x = (uint32_t)__bfloat16_as_ushort(nh) | ((uint32_t)__bfloat16_as_ushort(nm) << 16);
        v0.y = (uint32_t)__bfloat16_as_ushort(nl);
        v0.z = 0u;
        v0.w = 0u;
        *reinterpret_cast<uint4*>(base + tc::tile_offset(jj, 0)) = v0;
        *reinterpret_cast<uint4*>(base + tc::tile_offset(jj, 1)) = make_uint4(0u, 0u, 0u, 0u);
    }
}


// ---- second pass of the single-pass form: the rows its bound could not
// decide go through the split-BF16 kernel (a bound 2^-7 of the single pass's),
// and only the rows that one cannot decide reach the FP64 recheck.

// *nb = the number of listed rows when they fit the pass's buffers (cap), else
// 0 (the FP64 recheck then takes them all); st2 = the stage state with an
// empty list of its own.
__global__ void stageb_prep_kernel(StageState* st, StageState* st2, long long* nb, long long cap)
{
    const int count = st->recheck_count;
    const bool run = st->error == 0 && count > 0 && (long long)count <= cap;
    *nb = run ? (long long)count : 0ll;
    st->undecided16_total += count;
    *st2 = *st;
    st2->recheck_count = 0;
}

// Compact copies of the listed rows: FP32 rows (the pass's sums read them),
// split-BF16 tiles, FP32 ||x||^2 and the old labels; rows past the count up to
// the tile boundary are zero.  One warp per row.
__global__ void stageb_compact_kernel(const float* __restrict__ X, int d, const int* __restrict__ list,
                                      const long long* nb, const int* __restrict__ labels,
                                      const StageState* st, float* __restrict__ Xc,
                                      unsigned char* __restrict__ Xt, float* __restrict__ xn2,
                                      int* __restrict__ lab)
{
    const long long count = *nb;
    const int lane = threadIdx.x & 31;
    const bool delta = st->mode == kModeDelta;
    const long long nrows = (count + kRows - 1) / kRows * kRows;
    const size_t Ahalf = (size_t)kRows * d * 2;
    long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (; w < nrows; w += nw) {
        const long long tile = w / kRows;
        const int r = (int)(w - tile * kRows);
        unsigned char* base = Xt + (size_t)tile * 2 * Ahalf;
        const bool live = w < count;
        const long long i = live ? (long long)list[w] : 0;
        float s2 = 0.f;
        for (int t0 = 4 * lane; t0 < d; t0 += 128) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (live) {
                v = __ldg(reinterpret_cast<const float4*>(X + i * d + t0));
                *reinterpret_cast<float4*>(Xc + w * d + t0) = v;
            }
            s2 = fmaf(v.x, v.x, s2); s2 = fmaf(v.y, v.y, s2);
            s2 = fmaf(v.z, v.z, s2); s2 = fmaf(v.w, v.w, s2);
            const int ks = t0 >> 4, kc = (t0 >> 3) & 1, e = t0 & 7;
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
            const size_t off = (size_t)ks * 4096 + tc::tile_offset(r, kc) + e * 2;
            *reinterpret_cast<uint2*>(base + off) = ph;
            *reinterpret_cast<uint2*>(base + Ahalf + off) = pl;
        }
        for (int o = 16; o; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        if (lane == 0 && live) {
            xn2[w] = s2;
            lab[w] = delta ? labels[i] : -1;
        }
    }
}

// The pass's decisions back to the stage: labels of the compact rows, and its
// own list of undecided rows (compact indices) turned into row indices.
__global__ void stageb_scatter_kernel(const int* __restrict__ list, const long long* nb,
                                      const int* __restrict__ lab, int* __restrict__ labels,
                                      int* __restrict__ list2, const StageState* st2)
{
    const long long count = *nb;
    if (count == 0) return;
    const long long c2 = st2->recheck_count;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += stride)
        labels[list[e]] = lab[e];
    for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < c2; f += stride)
        list2[f] = list[list2[f]];
}

// The stage's recheck list and count become the pass's (error carried over).
__global__ void stageb_finish_kernel(int* __restrict__ list, const int* __restrict__ list2,
                                     const long long* nb, StageState* st, const StageState* st2)
{
    if (*nb == 0) return;
    const long long c2 = st2->recheck_count;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < c2; f += stride)
        list[f] = list2[f];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->recheck_count = (int)c2;
        if (st2->error) st->error = st2->error;
    }
}
}  // namespace

// Per key (derivation in the design notes): with |x - xh - xl| <= 2^-18 |x| and
// |m - mh - ml| <= 2^-18 |m| (two round-to-nearest BF16 steps), the three
// products miss xl.ml, (x - xh - xl) m and (xh + xl)(m - mh - ml): at most
// 3.02 * 2^-18 |x_t||m_t| per dimension, i.e. 6.04 * 2^-18 sum_t |x_t||c_t|.
// The FP32 accumulation of nt = 3d + 3 exact products (the data K-steps and
// the three norm parts; truncation assumed): nt * 2^-23 (2 |x||c| + ||c||^2);
// FP32 centers and ||c||^2: 2^-23 |x||c| and 2^-23 ||c||^2; the BF16 parts of
// ||c||^2: 2^-27 ||c||^2.  With 2 |x||c| <= X2 + C2 the sum is below
// k_b (2 C2 + X2).  Two keys of a gap, 1.0625 slack.
float bf16_kappa(int d)
{
    const double nt = 3.0 * d + 3.0;
    const double a1 = 6.04 * 0x1p-18 + 2.0 * nt * 0x1p-23 + 0x1p-23;           // |x||c|
    const double a2 = nt * 0x1p-23 + 0x1p-23 + 0x1p-27;                         // ||c||^2
    const double kb = fmax(a1 / 2.0, (a1 / 2.0 + a2) / 2.0);
    return (float)(2.0 * kb * 1.0625);
}

// Single-pass FP16 form, per key.  Rounding the scaled operands to FP16 costs
// at most u = 2^-11 relative plus eta = 2^-14 absolute (scaled units; eta also
// covers FP16 subnormals flushed to zero).  The relative part leaves (2u + u^2)
// |x_t||m_t| per dimension, i.e. 2 (2u + u^2) sum_t |x_t||c_t|; the FP32
// accumulation of nt = d + 3 exact products (an FP16 x FP16 product is exact
// in FP32): nt 2^-23 (2 |x||c| + ||c||^2); FP32 centers and ||c||^2 and the BF16
// norm parts as in the split form.  The absolute part, back in unscaled units
// with 2^b <= sqrt(C2) 2^-11, 2^a = 2^(E - 14), sum_t |x_t| <= sqrt(d) |x| and
// sum_t |m_t| <= 2 sqrt(d) sqrt(C2):
//   eta (1 + u) sqrt(d) |x| sqrt(C2) 2^-11   <= (1 + u) sqrt(d) 2^-26 (X2 + C2)
//   eta (1 + u) 2 sqrt(d) sqrt(C2) 2^(E-14)  <= (1 + u) sqrt(d) 2^-28 (4^E + C2)
//   d eta^2 2^(a + b)                        <= d 2^-55 (4^E + C2)
// The first joins the relative coefficient; the other two, for two keys, are
// f16_kabs x (4^E + C2).
float f16_kappa(int d)
{
    const double u = 0x1p-11, nt = d + 3.0;
    const double a1 = 2.0 * (2.0 * u + u * u) + 2.0 * nt * 0x1p-23 + 0x1p-23;   // |x||c|
    const double a2 = nt * 0x1p-23 + 0x1p-23 + 0x1p-27;                         // ||c||^2
    const double kb = fmax(a1 / 2.0, (a1 / 2.0 + a2) / 2.0) + (1.0 + u) * sqrt((double)d) * 0x1p-26;
    return (float)(2.0 * kb * 1.0625);
}

float f16_kabs(int d)
{
    const double u = 0x1p-11;
    return (float)(2.0 * ((1.0 + u) * sqrt((double)d) * 0x1p-28 + d * 0x1p-55) * 1.0625);
}

// Two A stages of a 128-row tile (hi + lo parts) and at least two B slices of
// the widest chunk must fit into the shared-memory budget.
int bf16_fits(int d)
{
    return d <= 128 && kSA * 4 * kRows * d + 2 * 128 * 64 + 4096 <= kSmemBudget - kStaticSmem;
}

int assign_bf16_supported(int d, int k, const float* X)
{
    (void)k;
    if ((reinterpret_cast<uintptr_t>(X) & 15) != 0) return 0;
    return d >= 16 && d % 16 == 0 && bf16_fits(d);
}

// Chunk width NC: 64 when k fits in 64, 256 from k = 512 on (one M128 x N256
// MMA per part and K-step: half the instructions and a wider B operand per
// A read), else 128.  Two epilogue groups x kAccBufs accumulators x NC
// columns fill at most the 512 TMEM columns of the SM.  Columns past k hold
// zero centers with the padding norm, so they never win.
int bf16_chunk(int d, int k, int single)
{
    (void)d;
    (void)single;
    return k <= 64 ? 64 : (k >= 512 ? 256 : 128);
}

size_t bf16_xt_bytes(long long n, int d, int single)
{
    return (size_t)((n + kRows - 1) / kRows) * kRows * (size_t)d * 2 * (single ? 1 : 2);
}

size_t bf16_cb_bytes(int d, int k, int single)
{
    const int nc = bf16_chunk(d, k, single);
    const int nch = (k + nc - 1) / nc;
    return (size_t)nch * nc * (single ? 32 : 64) * (size_t)(d / 16 + 1);
}

int launch_convert_x_bf16(const float* X, long long n, int d, unsigned char* Xt, float* xn2,
                          const StageState* st, int single, cudaStream_t s, int sm_count)
{
    const long long ntiles = (n + kRows - 1) / kRows;
    long long blocks = (ntiles * kRows * 32 + 255) / 256;
    if (blocks > (long long)sm_count * 16) blocks = (long long)sm_count * 16;
    ++g_launches;
    if (single)
        convert_x_f16_kernel<<<(int)blocks, 256, 0, s>>>(X, n, d, Xt, xn2, ntiles, st);
    else
        convert_x_kernel<<<(int)blocks, 256, 0, s>>>(X, n, d, Xt, xn2, ntiles);
    KM2_CUDA(cudaGetLastError());
    return KMEANS2_OK;
}

int launch_assign_bf16(const float* X, const unsigned char* Xt, const float* xn2,
                       unsigned char* Cb, long long n, int d, const Centers& c, int* labels,
                       StageState* st, const Accum& acc, int* list, int single, cudaStream_t s,
                       int sm_count, const long long* n_dev)
{
    const int NC = bf16_chunk(d, c.k, single);
    const int nch = (c.k + NC - 1) / NC;
    // this iteration's centers into BF16 (FP16) chunks
    {
        const long long total = (long long)nch * NC * d;
        long long blocks = (total + 255) / 256;
        if (blocks > 4096) blocks = 4096;
        ++g_launches;
        if (single)
            convert_c_f16_kernel<<<(int)blocks, 256, 0, s>>>(c.c32, c.k, d, NC, nch, Cb, st);
        else
            convert_c_kernel<<<(int)blocks, 256, 0, s>>>(c.c32, c.k, d, NC, nch, Cb);
        KM2_CUDA(cudaGetLastError());
        ++g_launches;
        if (single)
            convert_norm_single_kernel<<<(nch * NC + 255) / 256, 256, 0, s>>>(c.cnorm, c.k, d, NC,
                                                                               nch, Cb, st);
        else
            convert_norm_kernel<<<(nch * NC + 255) / 256, 256, 0, s>>>(c.cnorm, c.k, d, NC, nch,
                                                                        Cb);
        KM2_CUDA(cudaGetLastError());
    }
    uint32_t cols = 32;
    while (cols < (uint32_t)(kEpiGroups * (NC >= 256 ? 1 : 2) * NC)) cols <<= 1;
    const size_t parts = single ? 1 : 2;
    const size_t abytes = parts * 2 * kRows * d, kbytes = (size_t)NC * 32 * parts;
    // a B ring slot holds kps K-steps of a chunk: five in the single-pass form
    // (fewer when the ring would drop below two slots), one in the split form
    int kps = single ? 5 : 1, sb = 0;
    for (; kps >= 1; --kps) {
        sb = (int)((kSmemBudget - kStaticSmem - kSA * abytes - 4096) / (kbytes * kps));
        if (sb >= 2) break;
    }
    if (kps < 1 || sb < 2) {
        set_last_error_text("assign_bf16: shared-memory budget too small for this d");
        return KMEANS2_ERR_UNSUPPORTED;
    }
    if (sb > kMaxSB) sb = kMaxSB;
    const size_t sbytes = kbytes * kps;
    const size_t smem = kSA * abytes + (size_t)sb * sbytes + 4096;
    // one fixed limit for both instantiations (the static part holds the
    // barriers, the side ring and the recheck queues)
    KM2_TRY(set_max_dynamic_smem((const void*)assign_bf16<64, 0>, kSmemBudget - kStaticSmem));
    KM2_TRY(set_max_dynamic_smem((const void*)assign_bf16<128, 0>, kSmemBudget - kStaticSmem));
    KM2_TRY(set_max_dynamic_smem((const void*)assign_bf16<256, 0>, kSmemBudget - kStaticSmem));
    KM2_TRY(set_max_dynamic_smem((const void*)assign_bf16<64, 1>, kSmemBudget - kStaticSmem));
    KM2_TRY(set_max_dynamic_smem((const void*)assign_bf16<128, 1>, kSmemBudget - kStaticSmem));
    KM2_TRY(set_max_dynamic_smem((const void*)assign_bf16<256, 1>, kSmemBudget - kStaticSmem));
    const long long tiles = (n + kRows - 1) / kRows;
    long long grid = sm_count;
    if (grid > tiles) grid = tiles;
    if (grid < 1) grid = 1;
    Bf16Args a;
    a.X = X;
    a.n_dev = n_dev;
    a.Xt = Xt;
    a.xn2 = xn2;
    a.Cb = Cb;
    a.n = n;
    a.d = d;
    a.k = c.k;
    a.nc = NC;
    a.nch = nch;
    a.sb = sb;
    a.kps = kps;
    a.lab_bulk = (reinterpret_cast<uintptr_t>(labels) & 15) == 0 ? 1 : 0;
    a.tmem_cols = cols;
    a.kappa = single ? f16_kappa(d) : bf16_kappa(d);
    a.kabs = single ? f16_kabs(d) : 0.0f;
    a.kpack = kPackSlack;
    a.ctries = consumer_wait_tries(kWaitTries);
    ++g_launches;
    if (single) {
        if (NC == 64)
            assign_bf16<64, 1><<<(int)grid, kThreads, smem, s>>>(a, c, labels, st, acc, list);
        else if (NC == 128)
            assign_bf16<128, 1><<<(int)grid, kThreads, smem, s>>>(a, c, labels, st, acc, list);
        else
            assign_bf16<256, 1><<<(int)grid, kThreads, smem, s>>>(a, c, labels, st, acc, list);
    } else {
        if (NC == 64)
            assign_bf16<64, 0><<<(int)grid, kThreads, smem, s>>>(a, c, labels, st, acc, list);
        else if (NC == 128)
            assign_bf16<128, 0><<<(int)grid, kThreads, smem, s>>>(a, c, labels, st, acc, list);
        else
            assign_bf16<256, 0><<<(int)grid, kThreads, smem, s>>>(a, c, labels, st, acc, list);
    }
    KM2_CUDA(cudaGetLastError());
    return KMEANS2_OK;
}

// Rows the second pass takes at most: a quarter of the stage (more undecided
// rows than that go to the FP64 recheck; a single pass that leaves so many is
// the wrong form for the data anyway).
long long stage_b_cap(long long n)
{
    const long long cap = n / 4 + 1024;
    return cap < n ? cap : n;
}

int launch_stage_b(const float* X, int d, const Centers& c, int* labels, StageState* st,
                   const Accum& acc, int* list, const StageB& b, cudaStream_t s, int sm_count)
{
    g_launches += 4;
    stageb_prep_kernel<<<1, 1, 0, s>>>(st, b.st, b.nb, b.cap);
    KM2_CUDA(cudaGetLastError());
    const long long rows = (b.cap + kRows - 1) / kRows * kRows;
    long long blocks = (rows * 32 + 255) / 256;
    if (blocks > (long long)sm_count * 16) blocks = (long long)sm_count * 16;
    stageb_compact_kernel<<<(int)blocks, 256, 0, s>>>(X, d, list, b.nb, labels, st, b.Xc, b.Xt,
                                                      b.xn2, b.lab);
    KM2_CUDA(cudaGetLastError());
    KM2_TRY(launch_assign_bf16(b.Xc, b.Xt, b.xn2, b.cb, b.cap, d, c, b.lab, b.st, acc, b.list, 0,
                               s, sm_count, b.nb));
    long long sb = (b.cap + 255) / 256;
    if (sb > (long long)sm_count * 8) sb = (long long)sm_count * 8;
    stageb_scatter_kernel<<<(int)sb, 256, 0, s>>>(list, b.nb, b.lab, labels, b.list, b.st);
    KM2_CUDA(cudaGetLastError());
    stageb_finish_kernel<<<(int)sb, 256, 0, s>>>(list, b.list, b.nb, st, b.st);
    KM2_CUDA(cudaGetLastError());
    return KMEANS2_OK;
}

}  // namespace km2
