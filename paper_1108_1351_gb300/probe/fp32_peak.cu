// fp32_peak.cu -- FP32 FMA throughput probe: the denominator of the CUDA-core
// distance kernels' roofline.  Not part of the k-means library; bench.py loads
// it (libfp32peak.so) to measure the peak on the GPU it runs on, under the
// clocks of that run.
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

}  // extern "C"
