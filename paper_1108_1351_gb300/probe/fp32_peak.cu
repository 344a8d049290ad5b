// fp32_peak.cu -- FP32 FMA throughput probe: the denominator of the CUDA-core
// distance kernels' roofline.  Not part of the k-means library; bench.py loads
// it (libfp32peak.so) to measure the peak on the GPU it runs on, under the
// clocks of that run.  A second probe times the inner loop of the small-d
// distance kernel alone (see select_loop below): the ceiling that its mix of
// packed FMAs and top-2 selection instructions allows.
//
// Every thread advances NACC independent FMA chains (enough to cover the FMA
// latency at full occupancy) for `iters` rounds, either as scalar fmaf or as
// packed fma.rn.f32x2 (two FMAs per instruction).  The chains stay bounded
// (a <- a * b + c with |b| < 1) and their sum is stored so that nothing is
// optimised away.  FMAs executed = grid * block * iters * NACC (* 2 packed).
#include <cuda_runtime.h>

namespace {

constexpr int kNacc = 16;

__global__ void __launch_bounds__(256) fma_scalar(long long iters, float b, float c, float* out)
{
    float a[kNacc];
#pragma unroll
    for (int i = 0; i < kNacc; ++i) a[i] = (float)(threadIdx.x + i) * 1e-3f;
    for (long long r = 0; r < iters; ++r) {
#pragma unroll
        for (int i = 0; i < kNacc; ++i) a[i] = fmaf(a[i], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kNacc; ++i) s += a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) fma_packed(long long iters, float b, float c, float* out)
{
    float2 a[kNacc];
#pragma unroll
    for (int i = 0; i < kNacc; ++i) a[i] = make_float2((float)(threadIdx.x + i) * 1e-3f, (float)i * 1e-3f);
    const float2 bb = make_float2(b, b), cc = make_float2(c, c);
    for (long long r = 0; r < iters; ++r) {
#pragma unroll
        for (int i = 0; i < kNacc; ++i) a[i] = __ffma2_rn(a[i], bb, cc);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kNacc; ++i) s += a[i].x + a[i].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The inner loop of the small-d distance kernel at d = 8 with nothing else:
// 2 points per thread in registers, 32 centers per chunk held as interleaved
// pairs in shared memory (-2 c, read as broadcast 128-bit loads) with their
// squared norms, one packed FMA per coordinate and center pair.  MODE 0 keeps
// the kernel's exact top-2 over packed keys (index in the 5 low mantissa
// bits); MODE 1 replaces the selection by one three-way minimum per pair, so
// its time is that of the loads and FMAs alone.  No global memory is touched
// inside the loop.  FMAs executed = grid * block * iters * 16 pairs * 2 points
// * 8 coordinates * 2.
__device__ __forceinline__ float select_key(float v, unsigned j)
{
    return __uint_as_float((__float_as_uint(v) & ~31u) | j);
}

__device__ __forceinline__ float min_of3(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

template <int MODE>
__global__ void __launch_bounds__(256, 4) select_loop(long long iters, float seed, float* out)
{
    __shared__ __align__(16) float sc[32 * 8];
    __shared__ __align__(16) float sn[32];
    for (int e = threadIdx.x; e < 32 * 8; e += blockDim.x) sc[e] = seed * (float)(e % 37) - 1.0f;
    if (threadIdx.x < 32) sn[threadIdx.x] = seed * (float)threadIdx.x;
    __syncthreads();
    float x[2][8];
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int t = 0; t < 8; ++t) x[p][t] = (float)((threadIdx.x * 7 + p * 3 + t) % 13) * seed;
    float b1[2] = {INFINITY, INFINITY}, b2[2] = {INFINITY, INFINITY};
    for (long long r = 0; r < iters; ++r) {
#pragma unroll 4
        for (unsigned jj = 0; jj < 32; jj += 2) {
            float2 cp[8];
            const float4* q = reinterpret_cast<const float4*>(sc + jj * 8);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const float4 v = q[h];
                cp[2 * h] = make_float2(v.x, v.y);
                cp[2 * h + 1] = make_float2(v.z, v.w);
            }
            const float2 n01 = *reinterpret_cast<const float2*>(sn + jj);
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                float2 dd = n01;
#pragma unroll
                for (int t = 0; t < 8; ++t) dd = __ffma2_rn(make_float2(x[p][t], x[p][t]), cp[t], dd);
                if (MODE == 0) {
                    const float k0 = select_key(dd.x, jj), k1 = select_key(dd.y, jj | 1u);
                    const float lo = fminf(k0, k1), hi = fmaxf(k0, k1);
                    b2[p] = min_of3(b2[p], hi, fmaxf(b1[p], lo));
                    b1[p] = fminf(b1[p], lo);
                } else {
                    b1[p] = min_of3(b1[p], dd.x, dd.y);
                }
            }
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = b1[0] + b1[1] + b2[0] + b2[1];
}

}  // namespace

extern "C" {

// Runs one probe launch of `blocks` x 256 threads on `stream`; out: device
// buffer of blocks * 256 floats.  *ms = its CUDA-event time; *fmas = the FMAs
// it executed.  Returns 0 or the CUDA error code.
__attribute__((visibility("default"))) int fp32_fma_probe(int packed, int blocks, long long iters,
                                                          float* out, void* stream, float* ms,
                                                          double* fmas)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return (int)e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) { cudaEventDestroy(e0); return (int)e; }
    cudaEventRecord(e0, s);
    if (packed) fma_packed<<<blocks, 256, 0, s>>>(iters, 0.999999f, 1e-6f, out);
    else fma_scalar<<<blocks, 256, 0, s>>>(iters, 0.999999f, 1e-6f, out);
    cudaEventRecord(e1, s);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *fmas = (double)blocks * 256.0 * (double)iters * kNacc * (packed ? 2.0 : 1.0);
    return (int)e;
}

// Runs one launch of the small-d inner loop (select_loop<mode>, mode 0 or 1)
// with `blocks` x 256 threads on `stream`; out: device buffer of blocks * 256
// floats.  *ms = its CUDA-event time; *fmas = the FMAs it executed.  Returns 0
// or the CUDA error code (cudaErrorInvalidValue for another mode).
__attribute__((visibility("default"))) int fp32_select_probe(int mode, int blocks, long long iters,
                                                             float* out, void* stream, float* ms,
                                                             double* fmas)
{
    if (mode != 0 && mode != 1) return (int)cudaErrorInvalidValue;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return (int)e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) { cudaEventDestroy(e0); return (int)e; }
    cudaEventRecord(e0, s);
    if (mode == 0) select_loop<0><<<blocks, 256, 0, s>>>(iters, 1e-3f, out);
    else select_loop<1><<<blocks, 256, 0, s>>>(iters, 1e-3f, out);
    cudaEventRecord(e1, s);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *fmas = (double)blocks * 256.0 * (double)iters * 16.0 * 2.0 * 8.0 * 2.0;
    return (int)e;
}

}  // extern "C"
