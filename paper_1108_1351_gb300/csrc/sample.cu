// sample.cu -- the Algorithm's two random draws (the per% subset S_s and the
// initial centers picked at random from it), done on the GPU.
//
// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) serves as a counter-based
// generator: key_i = mix64(seed + (i + 1) * GAMMA).  mix64 is a bijection, so
// keys never tie.  S_s = the m smallest keys of stream positions [0, n); the
// initial centers = the k smallest keys of positions [n, n + m).  Selecting
// the m smallest of a range is an exact radix select: one histogram pass over
// the top 11 key bits, a collection of the keys in the bucket that holds the
// m-th smallest, 11-bit narrowing passes over those candidates down to the
// exact m-th key T, then an order-preserving compaction of {i : key_i <= T}.
// Keys are recomputed on the fly in every pass, so nothing of size n is stored.
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "api_internal.h"

namespace km2 {

namespace {

constexpr int kBins = 2048;           // 11-bit digits
constexpr int kThreads = 256;
constexpr int kChunkItems = 4096;     // indices per compaction chunk (16 per thread)

__device__ __forceinline__ unsigned long long key_at(unsigned long long seed,
                                                     unsigned long long pos)
{
    return splitmix64_at(seed, pos);
}

struct SelectState {
    unsigned long long prefix;   // fixed high bits of the threshold key T
    long long need;              // rank (1-based) of T among keys sharing `prefix`
    int free_bits;               // low bits of T not yet fixed
    unsigned int cand_count;     // candidates collected
    unsigned int hist[kBins];
};

// Histogram of the top 11 bits over the full range.
__global__ void hist_top(unsigned long long seed, unsigned long long offset, long long count,
                         unsigned int* ghist)
{
    __shared__ unsigned int h[kBins];
    for (int b = threadIdx.x; b < kBins; b += blockDim.x) h[b] = 0;
    __syncthreads();
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        unsigned long long key = key_at(seed, offset + (unsigned long long)i);
        atomicAdd(&h[key >> 53], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kBins; b += blockDim.x)
        if (h[b]) atomicAdd(&ghist[b], h[b]);
}

// Single CTA: find the bucket of the need-th key in st->hist, fix its digit.
// `shift` is the bit position of the digit's least significant bit.
__global__ void find_bucket(SelectState* st, int shift, int width)
{
    __shared__ unsigned int part[kThreads];
    __shared__ long long base[kThreads + 1];
    int nb = 1 << width;
    int per = (nb + kThreads - 1) / kThreads;
    unsigned int s = 0;
    for (int b = threadIdx.x * per; b < min(nb, (int)(threadIdx.x + 1) * per); ++b) s += st->hist[b];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long acc = 0;
        for (int t = 0; t < kThreads; ++t) { base[t] = acc; acc += part[t]; }
        base[kThreads] = acc;
    }
    __syncthreads();
    long long need = st->need;
    long long lo = base[threadIdx.x];
    long long hi = base[threadIdx.x + 1];
    if (need > lo && need <= hi) {
        long long acc = lo;
        for (int b = threadIdx.x * per; b < min(nb, (int)(threadIdx.x + 1) * per); ++b) {
            long long c = st->hist[b];
            if (need <= acc + c) {
                st->prefix |= (unsigned long long)b << shift;
                st->need = need - acc;
                st->free_bits = shift;
                break;
            }
            acc += c;
        }
    }
}

// Collect the keys whose top 11 bits equal the chosen bucket.
__global__ void collect(unsigned long long seed, unsigned long long offset, long long count,
                        SelectState* st, unsigned long long* cand, unsigned int cap)
{
    unsigned long long want = st->prefix >> 53;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        unsigned long long key = key_at(seed, offset + (unsigned long long)i);
        if ((key >> 53) == want) {
            unsigned int slot = atomicAdd(&st->cand_count, 1u);
            if (slot < cap) cand[slot] = key;
        }
    }
}

// Histogram of the digit [shift, shift + width) over candidates matching the prefix.
__global__ void hist_cand(const unsigned long long* cand, SelectState* st, int shift, int width)
{
    __shared__ unsigned int h[kBins];
    int nb = 1 << width;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) h[b] = 0;
    __syncthreads();
    unsigned int cnt = st->cand_count;
    int hi_shift = shift + width;
    unsigned long long want = st->prefix >> hi_shift;
    for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += gridDim.x * blockDim.x) {
        unsigned long long key = cand[i];
        if ((key >> hi_shift) == want)
            atomicAdd(&h[(key >> shift) & (unsigned long long)(nb - 1)], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        if (h[b]) atomicAdd(&st->hist[b], h[b]);
}

// Per-chunk count of keys <= T.
__global__ void count_sel(unsigned long long seed, unsigned long long offset, long long count,
                          const SelectState* st, unsigned int* chunk_counts, long long nchunks)
{
    __shared__ unsigned int wsum[kThreads / 32];
    unsigned long long T = st->prefix;
    for (long long c = blockIdx.x; c < nchunks; c += gridDim.x) {
        long long base = c * kChunkItems;
        unsigned int local = 0;
        for (int it = 0; it < kChunkItems / kThreads; ++it) {
            long long i = base + (long long)it * kThreads + threadIdx.x;
            if (i < count && key_at(seed, offset + (unsigned long long)i) <= T) ++local;
        }
        for (int o = 16; o; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
        if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = local;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned int s = 0;
            for (int w = 0; w < kThreads / 32; ++w) s += wsum[w];
            chunk_counts[c] = s;
        }
        __syncthreads();
    }
}

// Exclusive scan of chunk counts (single CTA, sequential over thread slices).
__global__ void scan_counts(const unsigned int* counts, long long nchunks, long long* offsets)
{
    __shared__ long long part[1024];
    long long per = (nchunks + blockDim.x - 1) / blockDim.x;
    long long b0 = threadIdx.x * per, b1 = min(nchunks, b0 + per);
    long long s = 0;
    for (long long c = b0; c < b1; ++c) s += counts[c];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long acc = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) { long long v = part[t]; part[t] = acc; acc += v; }
    }
    __syncthreads();
    long long acc = part[threadIdx.x];
    for (long long c = b0; c < b1; ++c) { offsets[c] = acc; acc += counts[c]; }
}

// Write the selected positions in ascending order.
__global__ void write_sel(unsigned long long seed, unsigned long long offset, long long count,
                          const SelectState* st, const long long* offsets, long long nchunks,
                          long long* out)
{
    __shared__ unsigned int wcnt[kThreads / 32];
    __shared__ long long running;
    unsigned long long T = st->prefix;
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long c = blockIdx.x; c < nchunks; c += gridDim.x) {
        if (threadIdx.x == 0) running = offsets[c];
        __syncthreads();
        long long base = c * kChunkItems;
        for (int it = 0; it < kChunkItems / kThreads; ++it) {
            long long i = base + (long long)it * kThreads + threadIdx.x;
            bool sel = i < count && key_at(seed, offset + (unsigned long long)i) <= T;
            unsigned mask = __ballot_sync(0xffffffffu, sel);
            if (lane == 0) wcnt[warp] = __popc(mask);
            __syncthreads();
            long long before = running;
            for (int w = 0; w < warp; ++w) before += wcnt[w];
            if (sel) out[before + __popc(mask & lanemask_lt())] = i;
            __syncthreads();
            if (threadIdx.x == 0) {
                long long s = 0;
                for (int w = 0; w < kThreads / 32; ++w) s += wcnt[w];
                running += s;
            }
            __syncthreads();
        }
    }
}

// Order k selected positions by their key (rank = number of smaller keys).
__global__ void order_by_key(unsigned long long seed, unsigned long long offset,
                             const long long* sel, int k, long long* out)
{
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < k; a += gridDim.x * blockDim.x) {
        unsigned long long ka = key_at(seed, offset + (unsigned long long)sel[a]);
        int rank = 0;
        for (int b = 0; b < k; ++b)
            rank += key_at(seed, offset + (unsigned long long)sel[b]) < ka;
        out[rank] = sel[a];
    }
}

}  // namespace

// m smallest keys of stream positions [offset, offset + count), written as
// ascending positions relative to `offset` into out (device, m entries).
static unsigned int* hist_of(SelectState* st)
{
    return reinterpret_cast<unsigned int*>(reinterpret_cast<char*>(st) +
                                           offsetof(SelectState, hist));
}

static int select_smallest(unsigned long long seed, unsigned long long offset, long long count,
                           long long m, long long* out, cudaStream_t s, DeviceScratch& ws)
{
    SelectState* st = nullptr;
    KM2_TRY(ws.alloc((void**)&st, sizeof(SelectState), s));
    KM2_CUDA(cudaMemsetAsync(st, 0, sizeof(SelectState), s));
    SelectState h0{};
    h0.need = m;
    h0.free_bits = 64;
    KM2_CUDA(cudaMemcpyAsync(st, &h0, offsetof(SelectState, hist), cudaMemcpyHostToDevice, s));
    int grid = ws.sm_count * 4;
    ++g_launches;
    hist_top<<<grid, kThreads, 0, s>>>(seed, offset, count, hist_of(st));
    KM2_CUDA(cudaGetLastError());
    ++g_launches;
    find_bucket<<<1, kThreads, 0, s>>>(st, 53, 11);
    // size the candidate buffer from the chosen bucket's count
    unsigned int hsel = 0;
    {
        unsigned int hist[kBins];
        SelectState hs;
        KM2_CUDA(cudaMemcpyAsync(&hs, st, offsetof(SelectState, hist), cudaMemcpyDeviceToHost, s));
        KM2_CUDA(cudaMemcpyAsync(hist, hist_of(st), sizeof(hist), cudaMemcpyDeviceToHost, s));
        KM2_CUDA(cudaStreamSynchronize(s));
        hsel = hist[hs.prefix >> 53];
    }
    unsigned long long* cand = nullptr;
    KM2_TRY(ws.alloc((void**)&cand, sizeof(unsigned long long) * (size_t)(hsel ? hsel : 1), s));
    ++g_launches;
    collect<<<grid, kThreads, 0, s>>>(seed, offset, count, st, cand, hsel);
    KM2_CUDA(cudaGetLastError());
    const int shifts[5] = {42, 31, 20, 9, 0};
    const int widths[5] = {11, 11, 11, 11, 9};
    int cgrid = (int)((hsel + kThreads - 1) / kThreads);
    if (cgrid < 1) cgrid = 1;
    if (cgrid > ws.sm_count * 4) cgrid = ws.sm_count * 4;
    for (int p = 0; p < 5; ++p) {
        KM2_CUDA(cudaMemsetAsync(hist_of(st), 0, sizeof(unsigned int) * kBins, s));
        ++g_launches;
        hist_cand<<<cgrid, kThreads, 0, s>>>(cand, st, shifts[p], widths[p]);
        ++g_launches;
        find_bucket<<<1, kThreads, 0, s>>>(st, shifts[p], widths[p]);
    }
    KM2_CUDA(cudaGetLastError());
    long long nchunks = (count + kChunkItems - 1) / kChunkItems;
    unsigned int* counts = nullptr;
    long long* offs = nullptr;
    KM2_TRY(ws.alloc((void**)&counts, sizeof(unsigned int) * (size_t)nchunks, s));
    KM2_TRY(ws.alloc((void**)&offs, sizeof(long long) * (size_t)nchunks, s));
    int g2 = (int)(nchunks < (long long)ws.sm_count * 8 ? nchunks : (long long)ws.sm_count * 8);
    ++g_launches;
    count_sel<<<g2, kThreads, 0, s>>>(seed, offset, count, st, counts, nchunks);
    ++g_launches;
    scan_counts<<<1, 1024, 0, s>>>(counts, nchunks, offs);
    ++g_launches;
    write_sel<<<g2, kThreads, 0, s>>>(seed, offset, count, st, offs, nchunks, out);
    KM2_CUDA(cudaGetLastError());
    return KMEANS2_OK;
}

int sample_device(long long n, int k, long long m, unsigned long long seed, long long* subset,
                  long long* init_pos, cudaStream_t s, DeviceScratch& ws)
{
    KM2_TRY(select_smallest(seed, 0ull, n, m, subset, s, ws));
    long long* sel = nullptr;
    KM2_TRY(ws.alloc((void**)&sel, sizeof(long long) * (size_t)k, s));
    KM2_TRY(select_smallest(seed, (unsigned long long)n, m, k, sel, s, ws));
    int grid = (k + kThreads - 1) / kThreads;
    ++g_launches;
    order_by_key<<<grid, kThreads, 0, s>>>(seed, (unsigned long long)n, sel, k, init_pos);
    KM2_CUDA(cudaGetLastError());
    return KMEANS2_OK;
}

}  // namespace km2
