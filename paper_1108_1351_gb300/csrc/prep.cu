// prep.cu -- the small kernels around the distance kernels:
//   maxabs      max |x| over a stage's data (fixed-point scale, finiteness check)
//   qsum        exact sum of s^2 over a stage's coordinates, s = round(x 2^F)
//               (the integer that J is formed from, Eq. 3)
//   gather      X_s = rows of X at the subset indices (Algorithm: the per% subset)
//   init        initial centers = chosen points of X_s (Algorithm: random initial centers)
//   center_prep FP32 / transposed copies of the FP64 centers and ||c||^2
//   stage_init  fixed-point scales and loop state of one stage
//   finalize    new centers = cluster means (Lloyd's method, Section 4.1), the
//               largest movement (stop test, Sections 5-6), J (Eq. 3)
//   recheck     FP64 re-evaluation of near-tie points (ties -> lowest index)
#include <cstdint>

#include "api_internal.h"
#include "stage_dev.cuh"

namespace km2 {

namespace {

__device__ __forceinline__ unsigned int abs_bits(float v)
{
    return __float_as_uint(v) & 0x7fffffffu;   // NaN keeps a payload above +inf
}

__device__ __forceinline__ unsigned int warp_max_u32(unsigned int v)
{
    for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__global__ void maxabs_kernel(const float* __restrict__ X, long long count, int vec4,
                              StageState* st)
{
    unsigned int m = 0;
    long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    long long done = 0;
    if (vec4) {
        const float4* X4 = reinterpret_cast<const float4*>(X);
        long long n4 = count >> 2;
        for (long long i = tid; i < n4; i += stride) {
            float4 v = __ldg(X4 + i);
            m = max(m, max(max(abs_bits(v.x), abs_bits(v.y)), max(abs_bits(v.z), abs_bits(v.w))));
        }
        done = n4 << 2;
    }
    for (long long i = done + tid; i < count; i += stride) m = max(m, abs_bits(__ldg(X + i)));
    m = warp_max_u32(m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(&st->maxabs_bits, m);
}

// Exact sum of s^2 over count coordinates, s = to_fixed(x, 2^F) (the same
// integers the cluster sums add), into st->q.  Each thread sums < 2^26
// squares below 2^92 in 128 bits; one wide_add4 per warp.
__global__ void qsum_kernel(const float* __restrict__ X, long long count, int vec4,
                            StageState* st)
{
    if (st->error) return;
    const float scale = st->scaleF;
    unsigned __int128 a = 0;
    long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    long long done = 0;
    if (vec4) {
        const float4* X4 = reinterpret_cast<const float4*>(X);
        long long n4 = count >> 2;
        for (long long i = tid; i < n4; i += stride) {
            float4 v = __ldg(X4 + i);
            a += sq_fixed(v.x, scale) + sq_fixed(v.y, scale) + sq_fixed(v.z, scale) +
                 sq_fixed(v.w, scale);
        }
        done = n4 << 2;
    }
    for (long long i = done + tid; i < count; i += stride) a += sq_fixed(__ldg(X + i), scale);
    a = warp_sum_u128(a);
    if ((threadIdx.x & 31) == 0 && a) wide_add4(st->q, a);
}

__global__ void gather_kernel(const float* __restrict__ X, int d,
                              const long long* __restrict__ subset, long long m,
                              float* __restrict__ Xs, StageState* st)
{
    unsigned int mx = 0;
    long long total = m * (long long)d;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        long long p = e / d;
        int t = (int)(e - p * d);
        float v = X[subset[p] * (long long)d + t];
        Xs[e] = v;
        mx = max(mx, abs_bits(v));
    }
    mx = warp_max_u32(mx);
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(&st->maxabs_bits, mx);
}

__global__ void init_centers_kernel(const float* __restrict__ Xs, int d,
                                    const long long* __restrict__ pos, int k,
                                    double* __restrict__ c64)
{
    long long total = (long long)k * d;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        long long j = e / d;
        int t = (int)(e - j * d);
        c64[e] = (double)Xs[pos[j] * (long long)d + t];
    }
}

// One CTA: FP32 copies and ||c_j||^2 of every center.
__global__ void center_prep_kernel(Centers c, StageState* st)
{
    __shared__ double red[1024];
    center_prep_block(c, st, red);
}

__global__ void stage_init_kernel(StageState* st, int d, double tol, int max_iter)
{
    stage_init_dev(st, d, tol, max_iter);
}

// One CTA.  New centers, movement, J; loop control for the next iteration.
__global__ void __launch_bounds__(1024) finalize_kernel(Accum acc, Centers c, StageState* st,
                                                        TrajDev tr, double* clus,
                                                        unsigned long long handle, int use_cond)
{
    __shared__ FinalizeSmem sm;
    if (st->error) {
        if (threadIdx.x == 0) {
            st->done = 1;
            if (use_cond) cudaGraphSetConditional(handle, 0u);
        }
        return;
    }
    finalize_block(acc, c, st, tr, clus, sm);
    if (threadIdx.x == 0 && use_cond) cudaGraphSetConditional(handle, st->done ? 0u : 1u);
}

// Many CTAs: the new centers, one warp per center (large k * d).
__global__ void __launch_bounds__(256) finalize_centers_kernel(Accum acc, Centers c,
                                                               StageState* st, TrajDev tr,
                                                               double* clus)
{
    if (st->error) return;
    const double inv = st->inv_scaleF;
    const int it = st->iter;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    for (int j = gw; j < c.k; j += nw) finalize_center_warp(acc, c, inv, j, clus, tr, it);
}

// One CTA after finalize_centers_kernel: movement, J, loop control.
__global__ void __launch_bounds__(1024) finalize_reduce_kernel(int k, StageState* st,
                                                               TrajDev tr, const double* clus,
                                                               unsigned long long handle,
                                                               int use_cond)
{
    __shared__ FinalizeSmem sm;
    if (st->error) {
        if (threadIdx.x == 0) {
            st->done = 1;
            if (use_cond) cudaGraphSetConditional(handle, 0u);
        }
        return;
    }
    finalize_reduce_block(k, st, tr, clus, sm);
    if (threadIdx.x == 0 && use_cond) cudaGraphSetConditional(handle, st->done ? 0u : 1u);
}

constexpr int kRecheckThreads = 256;
constexpr int kRecheckCache = 1024;     // pass-1 values kept per warp (k <= 1024)

// Warps of the grid share the listed points (see recheck_warps).
__global__ void __launch_bounds__(kRecheckThreads) recheck_kernel(const float* __restrict__ X, int d, Centers c,
                               int* __restrict__ labels, const int* __restrict__ list,
                               StageState* st, Accum acc)
{
    __shared__ float cache[kRecheckThreads / 32][kRecheckCache];
    if (st->error) return;
    long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    recheck_warps(X, d, c, labels, list, st, acc, gw, nw, cache[threadIdx.x >> 5], kRecheckCache);
}

}  // namespace

static int grid_for(long long work, int threads, int sm_count, int per_sm)
{
    long long g = (work + threads - 1) / threads;
    long long cap = (long long)sm_count * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

int launch_maxabs(const float* X, long long n, int d, StageState* st, cudaStream_t s,
                  int sm_count)
{
    const long long count = n * d;
    int vec4 = ((reinterpret_cast<uintptr_t>(X) & 15) == 0) ? 1 : 0;
    ++g_launches;
    maxabs_kernel<<<grid_for(count / 4 + 1, 256, sm_count, 8), 256, 0, s>>>(X, count, vec4, st);
    KM2_CUDA(cudaGetLastError());
    return KMEANS2_OK;
}

int launch_qsum(const float* X, long long n, int d, StageState* st, cudaStream_t s, int sm_count)
{
    const long long count = n * d;
    if (count <= 0) return KMEANS2_OK;
    int vec4 = ((reinterpret_cast<uintptr_t>(X) & 15) == 0) ? 1 : 0;
    ++g_launches;
    qsum_kernel<<<grid_for(count / 4 + 1, 256, sm_count, 8), 256, 0, s>>>(X, count, vec4, st);
    KM2_CUDA(cudaGetLastError());
    return KMEANS2_OK;
}

__global__ void recheck_reset_kernel(StageState* st)
{
    st->rechecked_total += st->recheck_count;
    st->recheck_count = 0;
}

int launch_recheck_reset(StageState* st, cudaStream_t s)
{
    ++g_launches;
    recheck_reset_kernel<<<1, 1, 0, s>>>(st);
    KM2_CUDA(cudaGetLastError());
    return KMEANS2_OK;
}

int launch_gather(const float* X, int d, const long long* subset, long long m, float* Xs,
                  StageState* st, cudaStream_t s, int sm_count)
{
    ++g_launches;
    gather_kernel<<<grid_for(m * d, 256, sm_count, 8), 256, 0, s>>>(X, d, subset, m, Xs, st);
    KM2_CUDA(cudaGetLastError());
    return KMEANS2_OK;
}

int launch_init_centers(const float* Xs, int d, const long long* pos, int k, double* c64,
                        cudaStream_t s)
{
    long long total = (long long)k * d;
    int grid = (int)((total + 255) / 256);
    if (grid > 4096) grid = 4096;
    ++g_launches;
    init_centers_kernel<<<grid, 256, 0, s>>>(Xs, d, pos, k, c64);
    KM2_CUDA(cudaGetLastError());
    return KMEANS2_OK;
}

int launch_center_prep(const Centers& c, StageState* st, cudaStream_t s)
{
    ++g_launches;
    center_prep_kernel<<<1, 1024, 0, s>>>(c, st);
    KM2_CUDA(cudaGetLastError());
    return KMEANS2_OK;
}

int launch_stage_init(StageState* st, int d, double tol, int max_iter, cudaStream_t s)
{
    ++g_launches;
    stage_init_kernel<<<1, 1, 0, s>>>(st, d, tol, max_iter);
    KM2_CUDA(cudaGetLastError());
    return KMEANS2_OK;
}

// k * d from which the center updates run on many CTAs instead of one.
constexpr long long kSplitFinalizeWork = 16384;

int launch_finalize(const Accum& acc, const Centers& c, StageState* st, const TrajDev& tr,
                    double* clus, unsigned long long cond_handle, int use_cond, cudaStream_t s)
{
    if ((long long)c.k * c.d >= kSplitFinalizeWork) {
        // spread the k center updates over the GPU, then reduce in one CTA
        // (the same per-center arithmetic and reduction order as one CTA)
        int blocks = (c.k + 7) / 8;
        if (blocks > 1024) blocks = 1024;
        g_launches += 2;
        finalize_centers_kernel<<<blocks, 256, 0, s>>>(acc, c, st, tr, clus);
        KM2_CUDA(cudaGetLastError());
        finalize_reduce_kernel<<<1, 1024, 0, s>>>(c.k, st, tr, clus, cond_handle, use_cond);
        KM2_CUDA(cudaGetLastError());
        return KMEANS2_OK;
    }
    ++g_launches;
    finalize_kernel<<<1, 1024, 0, s>>>(acc, c, st, tr, clus, cond_handle, use_cond);
    KM2_CUDA(cudaGetLastError());
    return KMEANS2_OK;
}

int launch_recheck(const float* X, int d, const Centers& c, int* labels, const int* list,
                   StageState* st, const Accum& acc, cudaStream_t s, int sm_count)
{
    ++g_launches;
    recheck_kernel<<<sm_count * 4, kRecheckThreads, 0, s>>>(X, d, c, labels, list, st, acc);
    KM2_CUDA(cudaGetLastError());
    return KMEANS2_OK;
}

}  // namespace km2
