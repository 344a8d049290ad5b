// api_internal.h -- host-side plumbing shared by the translation units of libkmeans2.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/kmeans2.h"
#include "common.cuh"

namespace km2 {

// Kernels launched by the calling thread (every launch site increments it).
extern thread_local long long g_launches;

// Thread-local text of the last CUDA failure, returned by kmeans2_last_error().
void set_last_error(const char* where, cudaError_t e);
void set_last_error_text(const char* text);

#define KM2_CUDA(call)                                                     \
    do {                                                                   \
        cudaError_t km2_e_ = (call);                                       \
        if (km2_e_ != cudaSuccess) {                                       \
            ::km2::set_last_error(#call, km2_e_);                          \
            return (km2_e_ == cudaErrorMemoryAllocation) ? KMEANS2_ERR_NOMEM \
                                                         : KMEANS2_ERR_CUDA; \
        }                                                                  \
    } while (0)

#define KM2_TRY(expr)                        \
    do {                                     \
        int km2_rc_ = (expr);                \
        if (km2_rc_ != KMEANS2_OK) return km2_rc_; \
    } while (0)

// A private blocking stream of the calling thread for `device` (capturable,
// unlike the legacy default stream).
cudaStream_t private_stream(int device);

// The library's stream-ordered memory pool on `device` (freed memory stays
// mapped for reuse; kmeans2_release_memory trims it); null if it cannot be made.
cudaMemPool_t library_pool(int device);
// cudaMallocAsync from the library pool of the current device.
cudaError_t pool_malloc_async(void** p, size_t bytes, cudaStream_t s);

// Stream-ordered scratch: every allocation is released (cudaFreeAsync on the
// same stream) when the object goes out of scope.
struct DeviceScratch {
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    int device = 0;
    std::vector<void*> ptrs;

    // Arena mode: alloc() carves 256-byte-aligned pieces out of [arena, arena +
    // arena_bytes) and never calls the allocator; nothing is freed.
    unsigned char* arena = nullptr;
    size_t arena_bytes = 0;
    size_t arena_used = 0;

    explicit DeviceScratch(cudaStream_t s);
    DeviceScratch(cudaStream_t s, void* arena_base, size_t bytes);
    ~DeviceScratch();
    int alloc(void** p, size_t bytes, cudaStream_t s);
    DeviceScratch(const DeviceScratch&) = delete;
    DeviceScratch& operator=(const DeviceScratch&) = delete;
};

// Wait limit (mbarrier try_wait rounds) of the consumer roles of the
// tensor-core kernels -- the MMA issuer and the epilogues -- given the
// kernel's normal limit.  Debug builds (KM2_DEBUG_CHECKS) take it from the
// environment variable KMEANS2_DEBUG_WAIT_TRIES when set, so that a test can
// make those waits run out and check the timeout status; producers and the
// drain waits that let every issued copy and MMA finish keep their limits.
int consumer_wait_tries(int normal);

// Raises a kernel's dynamic shared-memory limit to `bytes` once per (kernel,
// device) for the whole process, under a lock.  The value must be fixed per
// kernel: worker threads that launch the same kernel concurrently then never
// see the limit change under them.
int set_max_dynamic_smem(const void* kernel, int bytes);

// sample.cu
int sample_device(long long n, int k, long long m, unsigned long long seed, long long* subset,
                  long long* init_pos, cudaStream_t s, DeviceScratch& ws);

// prep.cu
// max |x| of n rows of d values, into st->maxabs_bits.
int launch_maxabs(const float* X, long long n, int d, StageState* st, cudaStream_t s,
                  int sm_count);
// Exact sum of s^2 over n rows of d values into st->q (after stage_init: needs F).
int launch_qsum(const float* X, long long n, int d, StageState* st, cudaStream_t s, int sm_count);
int launch_gather(const float* X, int d, const long long* subset, long long m, float* Xs,
                  StageState* st, cudaStream_t s, int sm_count);
int launch_init_centers(const float* Xs, int d, const long long* pos, int k, double* c64,
                        cudaStream_t s);
int launch_center_prep(const Centers& c, StageState* st, cudaStream_t s);
int launch_stage_init(StageState* st, int d, double tol, int max_iter, cudaStream_t s);
// clus: kClusSlots*k doubles of scratch; tr: the stage's optional per-iteration records.
int launch_finalize(const Accum& acc, const Centers& c, StageState* st, const TrajDev& tr,
                    double* clus, unsigned long long cond_handle, int use_cond, cudaStream_t s);
int launch_recheck(const float* X, int d, const Centers& c, int* labels, const int* list,
                   StageState* st, const Accum& acc, cudaStream_t s, int sm_count);
// Folds this pass's recheck count into the stage total and empties the list
// (between the chunks of a streamed pass, whose indices are chunk-relative).
int launch_recheck_reset(StageState* st, cudaStream_t s);

// assign_tc32.cu: tensor-core (3xTF32) form for FP32 data, d in {4, 8, 16, 32}, k <= 256
int assign_tc32_supported(int d, int k, const float* X);
int launch_assign_tc32(const float* X, long long n, int d, const Centers& c, int* labels,
                       StageState* st, const Accum& acc, int* list, cudaStream_t s,
                       int sm_count);

// assign_bf16.cu: tensor-core split-BF16 form, d a multiple of 16 in [16, 128]
int assign_bf16_supported(int d, int k, const float* X);
// single = 1: the single-pass FP16 variant (one operand part, scaled by powers
// of two taken from the stage's fixed-point exponent and max ||c||^2)
size_t bf16_xt_bytes(long long n, int d, int single);
size_t bf16_cb_bytes(int d, int k, int single);
int launch_convert_x_bf16(const float* X, long long n, int d, unsigned char* Xt, float* xn2,
                          const StageState* st, int single, cudaStream_t s, int sm_count);
int launch_assign_bf16(const float* X, const unsigned char* Xt, const float* xn2,
                       unsigned char* Cb, long long n, int d, const Centers& c, int* labels,
                       StageState* st, const Accum& acc, int* list, int single, cudaStream_t s,
                       int sm_count, const long long* n_dev = nullptr);
// Second pass of the single-pass FP16 form: buffers for up to `cap` rows that
// its bound could not decide, re-run through the split-BF16 kernel.
struct StageB {
    long long cap = 0;
    float* Xc = nullptr;          // cap x d FP32 rows
    unsigned char* Xt = nullptr;  // their split-BF16 tiles
    float* xn2 = nullptr;         // cap
    int* lab = nullptr;           // cap
    int* list = nullptr;          // cap: the pass's own undecided rows
    StageState* st = nullptr;     // the pass's stage state
    long long* nb = nullptr;      // rows the pass takes (device)
    unsigned char* cb = nullptr;  // split-BF16 center slices
};
long long stage_b_cap(long long n);
int launch_stage_b(const float* X, int d, const Centers& c, int* labels, StageState* st,
                   const Accum& acc, int* list, const StageB& b, cudaStream_t s, int sm_count);
// the two 16-bit tensor-core forms share the kernel, its tiles and its sizes
inline bool tc16_form(int form)
{
    return form == KMEANS2_PRECISION_BF16 || form == KMEANS2_PRECISION_FP16;
}

// assign_fp32.cu
int assign_fp32_supported(int d, int k);
int launch_assign_fp32(const float* X, long long n, int d, const Centers& c, int* labels,
                       StageState* st, const Accum& acc, int* list, cudaStream_t s,
                       int sm_count);

// ---------------------------------------------------------------- stage plumbing (api.cu)
// Per-stage device state of one fit: centers, exact sums, loop state, near-tie list.
struct Workspace {
    int form = KMEANS2_PRECISION_FP32;   // distance-kernel form used by this call
    Centers c{};
    Accum acc{};
    StageState* st = nullptr;
    int* list = nullptr;
    double* clus = nullptr;
    double* traj_J = nullptr;      // max_iter
    double* traj_shift = nullptr;  // max_iter
    double* traj_c = nullptr;      // max_iter * k * d (only when requested)
    long long* traj_n = nullptr;   // max_iter * k (only when requested)
    TrajDev traj() const { return TrajDev{traj_J, traj_shift, traj_c, traj_n}; }
    int max_iter = 0;
    DeviceScratch* ws = nullptr;   // the call's scratch (per-stage buffers)
    // BF16 form: the stage's points as BF16 tiles, their ||x||^2, the centers' chunks
    unsigned char* xt = nullptr;
    float* xn2 = nullptr;
    unsigned char* cb = nullptr;
    StageB sb{};                   // FP16 form: its second pass
};

int alloc_workspace(Workspace& w, DeviceScratch& ws, long long list_cap, int k, int d,
                    int max_iter, cudaStream_t s);
// BF16 form: per-stage BF16 tiles and ||x||^2 of the stage's points (no-op otherwise).
int prepare_stage_points(const float* X, long long n, int d, Workspace& w, DeviceScratch& ws,
                         cudaStream_t s);
// The fused distance kernel of w.form over n points.
int launch_assign(const float* X, long long n, int d, Workspace& w, int* labels, cudaStream_t s,
                  int sm_count);
// Resolves a requested precision to the form this shape runs in.
int choose_form(int requested, int d, int k, const float* X, int* form);
int map_stage_error(int err);
bool valid_shape(long long n, int d, int k);
bool is_device_ptr(const void* p);
// Device-resident, 16-byte aligned view of X (staged through scratch when needed).
int device_view(const float* X, long long count, const float** out, DeviceScratch& ws,
                cudaStream_t s);
struct Resolved {
    cudaStream_t stream;
    kmeans2_options opt;
};
Resolved resolve_options(const kmeans2_options* opt);

}  // namespace km2
