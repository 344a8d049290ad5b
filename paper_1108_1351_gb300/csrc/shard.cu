// shard.cu -- the two-stage method (Section 2) split over the rows of S_n, the
// way a data-parallel group of GPUs runs it: every rank keeps its own rows,
// labels, exact cluster sums and near-tie list, and a replicated copy of the
// centers.  The ranks exchange data at three kinds of points, each an
// all-reduce of one small buffer that the caller performs (NCCL, gloo, or the
// in-process reduction of kmeans2_fit_sharded):
//   * the initial centers (the Algorithm's random draw from S_s): every
//     rank writes the chosen rows of X_s that it owns and -0.0 elsewhere; the
//     FP64 sum is exact in any order (x + -0.0 = x for every x);
//   * max |x| of a stage's points, which fixes the stage's fixed-point scales;
//   * per Lloyd iteration (Section 4.1), the integer partials of the update:
//     the split sums S_j, the counts N_j and, in the first iteration of a
//     stage, the exact sum of the squared fixed-point coordinates (for J).  Integer sums are order-independent, so every rank
//     runs the same finalize on the same totals and all replicas, labels and
//     iteration counts equal those of one unsharded fit bit for bit.
// Sampling needs no exchange: the keys that choose S_s depend only on the
// global positions, so every rank draws S_s itself and keeps the part that
// falls in its rows (a contiguous piece of X_s, S_s being in ascending order).
#include <chrono>
#include <cstring>
#include <memory>
#include <vector>

#include "api_internal.h"

namespace km2 {
namespace {

constexpr int kMaxShards = 64;

// Number of entries of subset[0, m) below lo and below hi (subset ascending).
__global__ void bounds_kernel(const long long* subset, long long m, long long lo, long long hi,
                              long long* out)
{
    if (threadIdx.x > 1) return;
    const long long v = threadIdx.x == 0 ? lo : hi;
    long long a = 0, b = m;
    while (a < b) {
        long long mid = a + (b - a) / 2;
        if (subset[mid] < v) a = mid + 1; else b = mid;
    }
    out[threadIdx.x] = a;
}

__global__ void localize_kernel(long long* idx, long long count, long long row0)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        idx[i] -= row0;
}

// This rank's part of the initial centers: row pos[j] of X_s where this rank
// holds it (X_s positions [a, a + rows)), -0.0 elsewhere.
__global__ void init_contrib_kernel(const float* Xs, long long a, long long rows, int d,
                                    const long long* pos, int k, double* out)
{
    const long long total = (long long)k * d;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long j = e / d, t = e - j * d;
        const long long p = pos[j] - a;
        out[e] = (p >= 0 && p < rows) ? (double)Xs[p * d + t] : -0.0;
    }
}

// Exchange layout of the per-iteration partials (int64 entries):
//   [0, kd) low words of S | [kd, 2kd) high words of S | [2kd, 2kd + k) N |
//   q[0..3] (sum of s^2, first iteration of a stage) | one flag per device
//   error kind (1..3)
__host__ __device__ inline long long partials_count(int k, int d)
{
    return 2ll * k * d + k + 4 + 3;
}

// Carries each local low word into its high word (value unchanged) and copies
// the rank's partials into the exchange buffer; after the carry every low
// word is below 2^32, so the integer sum over up to 2^31 ranks cannot wrap.
__global__ void pack_partials_kernel(Accum acc, int k, int d, const StageState* st,
                                     unsigned long long* x)
{
    const long long kd = (long long)k * d;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < kd + k;
         e += (long long)gridDim.x * blockDim.x) {
        if (e < kd) {
            const unsigned long long lo = acc.s_lo[e], hi = acc.s_hi[e] + (lo >> 32);
            acc.s_lo[e] = lo & 0xffffffffull;
            acc.s_hi[e] = hi;
            x[e] = lo & 0xffffffffull;
            x[kd + e] = hi;
        } else {
            x[kd + e] = acc.cnt[e - kd];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // the sum of s^2 with its words carried (q[0..2] < 2^32, value
        // unchanged), so the sum over ranks cannot wrap either
        unsigned long long q[4] = {0ull, 0ull, 0ull, 0ull};
        if (st->mode == kModeFull)
            for (int w = 0; w < 4; ++w) q[w] = st->q[w];
        for (int w = 0; w < 3; ++w) {
            q[w + 1] += q[w] >> 32;
            q[w] &= 0xffffffffull;
        }
        for (int w = 0; w < 4; ++w) x[2 * kd + k + w] = q[w];
        for (int e = 1; e <= 3; ++e) x[2 * kd + k + 3 + e] = (st->error == e) ? 1ull : 0ull;
    }
}

// Totals of all ranks -> the accumulators finalize reads and the stage state.
__global__ void unpack_partials_kernel(const unsigned long long* x, Accum tot, int k, int d,
                                       StageState* st)
{
    const long long kd = (long long)k * d;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < kd + k;
         e += (long long)gridDim.x * blockDim.x) {
        if (e < kd) {
            tot.s_lo[e] = x[e];
            tot.s_hi[e] = x[kd + e];
        } else {
            tot.cnt[e - kd] = x[kd + e];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (st->mode == kModeFull)
            for (int w = 0; w < 4; ++w) st->q[w] = x[2 * kd + k + w];
        for (int e = 1; e <= 3; ++e)
            if (x[2 * kd + k + 3 + e] != 0ull && st->error == 0) st->error = e;
    }
}

__global__ void maxabs_xchg_kernel(StageState* st, unsigned long long* x, int to_buffer)
{
    if (to_buffer) x[0] = st->maxabs_bits;
    else st->maxabs_bits = (unsigned int)x[0];
}

struct XchgPtrs {
    unsigned long long* p[kMaxShards];
};

// The all-reduce of an in-process shard group, in shard order, written back
// to every shard's buffer.
__global__ void xchg_reduce_kernel(XchgPtrs ptrs, int P, long long count, int op)
{
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (long long)gridDim.x * blockDim.x) {
        if (op == KMEANS2_XCHG_SUM_F64) {
            double a = reinterpret_cast<const double*>(ptrs.p[0])[e];
            for (int r = 1; r < P; ++r) a += reinterpret_cast<const double*>(ptrs.p[r])[e];
            for (int r = 0; r < P; ++r) reinterpret_cast<double*>(ptrs.p[r])[e] = a;
        } else {
            unsigned long long a = ptrs.p[0][e];
            for (int r = 1; r < P; ++r) {
                const unsigned long long v = ptrs.p[r][e];
                if (op == KMEANS2_XCHG_SUM_I64) a += v;
                else a = ((long long)v > (long long)a) ? v : a;
            }
            for (int r = 0; r < P; ++r) ptrs.p[r][e] = a;
        }
    }
}

int grid_for(long long count)
{
    long long g = (count + 255) / 256;
    if (g < 1) g = 1;
    if (g > 1024) g = 1024;
    return (int)g;
}

}  // namespace
}  // namespace km2

using namespace km2;

// Phases of a shard between exchanges.
enum ShardPhase {
    kPhStart = 0,
    kPhInitCenters,   // waiting for the initial-centers sum
    kPhMaxabs,        // waiting for the stage's max |x|
    kPhIter,          // waiting for the iteration's partials
    kPhDone,
    kPhFailed,
};

struct kmeans2_shard {
    kmeans2_options opt{};
    cudaStream_t s = nullptr;
    std::unique_ptr<DeviceScratch> ws;
    Workspace w;
    Accum tot{};
    const float* X = nullptr;      // this rank's rows of S_n (device, aligned)
    long long n_local = 0, row0 = 0, n_total = 0, m = 0;
    long long fast_a = 0, m_local = 0;   // this rank's rows of X_s: [fast_a, fast_a + m_local)
    int d = 0, k = 0, max_iter = 0;
    double tol = 0.0, tol_fast = 0.0;
    float* Xs = nullptr;
    int* labels = nullptr;
    int* labels_s = nullptr;
    long long* pos = nullptr;
    unsigned long long* x = nullptr;     // the caller's exchange buffer
    int phase = kPhStart;
    int stage = 0;                       // 0 fast, 1 slow
    int status = KMEANS2_OK;
    kmeans2_result rr{};
    long long launches0 = 0;
    std::chrono::steady_clock::time_point t0;

    const float* stage_X() const { return stage == 0 ? Xs : X; }
    long long stage_rows() const { return stage == 0 ? m_local : n_local; }
    int* stage_labels() const { return stage == 0 ? labels_s : labels; }
};

namespace {

int fail(kmeans2_shard* sh, int rc)
{
    sh->phase = kPhFailed;
    sh->status = rc;
    return rc;
}

// Start stage sh->stage: local max |x|, sent for the max-reduction.
int begin_stage(kmeans2_shard* sh, kmeans2_exchange* next)
{
    cudaStream_t s = sh->s;
    KM2_CUDA(cudaMemsetAsync(sh->w.st, 0, sizeof(StageState), s));
    if (sh->stage_rows() > 0)
        KM2_TRY(launch_maxabs(sh->stage_X(), sh->stage_rows(), sh->d, sh->w.st, s,
                              sh->ws->sm_count));
    ++g_launches;
    maxabs_xchg_kernel<<<1, 1, 0, s>>>(sh->w.st, sh->x, 1);
    KM2_CUDA(cudaGetLastError());
    KM2_CUDA(cudaStreamSynchronize(s));
    sh->phase = kPhMaxabs;
    next->op = KMEANS2_XCHG_MAX_I64;
    next->count = 1;
    return KMEANS2_PENDING;
}

// Assign + recheck on this rank's rows, partials into the exchange buffer.
int run_local_pass(kmeans2_shard* sh, kmeans2_exchange* next)
{
    cudaStream_t s = sh->s;
    const long long rows = sh->stage_rows();
    if (rows > 0) {
        KM2_TRY(launch_assign(sh->stage_X(), rows, sh->d, sh->w, sh->stage_labels(), s,
                              sh->ws->sm_count));
        KM2_TRY(launch_recheck(sh->stage_X(), sh->d, sh->w.c, sh->stage_labels(), sh->w.list,
                               sh->w.st, sh->w.acc, s, sh->ws->sm_count));
    }
    const long long count = partials_count(sh->k, sh->d);
    ++g_launches;
    pack_partials_kernel<<<grid_for((long long)sh->k * sh->d + sh->k), 256, 0, s>>>(
        sh->w.acc, sh->k, sh->d, sh->w.st, sh->x);
    KM2_CUDA(cudaGetLastError());
    KM2_CUDA(cudaStreamSynchronize(s));
    sh->phase = kPhIter;
    next->op = KMEANS2_XCHG_SUM_I64;
    next->count = count;
    return KMEANS2_PENDING;
}

// The reduced max |x| is in the buffer: scales, loop state, first pass.
int resume_maxabs(kmeans2_shard* sh, kmeans2_exchange* next)
{
    cudaStream_t s = sh->s;
    const size_t kd = (size_t)sh->k * sh->d;
    ++g_launches;
    maxabs_xchg_kernel<<<1, 1, 0, s>>>(sh->w.st, sh->x, 0);
    KM2_CUDA(cudaGetLastError());
    KM2_CUDA(cudaMemsetAsync(sh->w.acc.s_lo, 0, kd * 8, s));
    KM2_CUDA(cudaMemsetAsync(sh->w.acc.s_hi, 0, kd * 8, s));
    KM2_CUDA(cudaMemsetAsync(sh->w.acc.cnt, 0, (size_t)sh->k * 8, s));
    KM2_TRY(launch_center_prep(sh->w.c, sh->w.st, s));
    KM2_TRY(launch_stage_init(sh->w.st, sh->d, sh->stage == 0 ? sh->tol_fast : sh->tol,
                              sh->max_iter, s));
    StageState st;
    KM2_CUDA(cudaMemcpyAsync(&st, sh->w.st, sizeof(st), cudaMemcpyDeviceToHost, s));
    KM2_CUDA(cudaStreamSynchronize(s));
    if (st.error) return map_stage_error(st.error);   // the same on every rank
    if (sh->stage_rows() > 0) {
        KM2_TRY(launch_qsum(sh->stage_X(), sh->stage_rows(), sh->d, sh->w.st, s,
                            sh->ws->sm_count));
        KM2_TRY(prepare_stage_points(sh->stage_X(), sh->stage_rows(), sh->d, sh->w, *sh->ws, s));
    }
    return run_local_pass(sh, next);
}

int resume_iter(kmeans2_shard* sh, kmeans2_exchange* next)
{
    cudaStream_t s = sh->s;
    const long long kd = (long long)sh->k * sh->d;
    ++g_launches;
    unpack_partials_kernel<<<grid_for(kd + sh->k), 256, 0, s>>>(sh->x, sh->tot, sh->k, sh->d,
                                                                 sh->w.st);
    KM2_CUDA(cudaGetLastError());
    KM2_TRY(launch_finalize(sh->tot, sh->w.c, sh->w.st, sh->w.traj(),
                            sh->w.clus, 0ull, 0, s));
    StageState st;
    KM2_CUDA(cudaMemcpyAsync(&st, sh->w.st, sizeof(st), cudaMemcpyDeviceToHost, s));
    KM2_CUDA(cudaStreamSynchronize(s));
    if (st.error) return map_stage_error(st.error);
    if (!st.done) return run_local_pass(sh, next);
    // stage finished
    const kmeans2_options& o = sh->opt;
    double* tj = sh->stage == 0 ? o.traj_J_fast : o.traj_J_slow;
    double* ts = sh->stage == 0 ? o.traj_shift_fast : o.traj_shift_slow;
    if (tj && st.iter > 0)
        KM2_CUDA(cudaMemcpyAsync(tj, sh->w.traj_J, sizeof(double) * st.iter,
                                 cudaMemcpyDeviceToHost, s));
    if (ts && st.iter > 0)
        KM2_CUDA(cudaMemcpyAsync(ts, sh->w.traj_shift, sizeof(double) * st.iter,
                                 cudaMemcpyDeviceToHost, s));
    KM2_CUDA(cudaStreamSynchronize(s));
    sh->rr.rechecked_points += st.rechecked_total;
    if (sh->stage == 0) {
        sh->rr.iters_fast = st.iter;
        sh->rr.converged_fast = st.converged;
        sh->rr.shift_fast = st.shift;
        sh->stage = 1;
        return begin_stage(sh, next);
    }
    sh->rr.iters_slow = st.iter;
    sh->rr.converged_slow = st.converged;
    sh->rr.shift_slow = st.shift;
    sh->rr.J = st.J;
    sh->rr.empty_clusters = st.empty;
    sh->rr.distance_evals = (int64_t)sh->rr.iters_fast * sh->m * sh->k +
                            (int64_t)sh->rr.iters_slow * sh->n_total * sh->k;
    sh->phase = kPhDone;
    return KMEANS2_OK;
}

int shard_setup(kmeans2_shard* sh, const float* X_local, double subset_fraction, uint64_t seed,
                const double* init_centers)
{
    cudaStream_t s = sh->s;
    DeviceScratch& ws = *sh->ws;
    const int d = sh->d, k = sh->k;
    if (sh->n_local > 0)
        KM2_TRY(device_view(X_local, sh->n_local * d, &sh->X, ws, s));
    // the form depends on (precision, d, k) only: X is aligned device memory
    // on every rank after device_view
    const float* aligned = reinterpret_cast<const float*>(static_cast<uintptr_t>(256));
    KM2_TRY(choose_form(sh->opt.precision, d, k, aligned, &sh->w.form));
    sh->m = kmeans2_subset_size(sh->n_total, k, subset_fraction);
    long long* subset = nullptr;
    long long* bnd = nullptr;
    KM2_TRY(ws.alloc((void**)&subset, sizeof(long long) * (size_t)sh->m, s));
    KM2_TRY(ws.alloc((void**)&sh->pos, sizeof(long long) * (size_t)k, s));
    KM2_TRY(ws.alloc((void**)&bnd, 2 * sizeof(long long), s));
    KM2_TRY(sample_device(sh->n_total, k, sh->m, seed, subset, sh->pos, s, ws));
    ++g_launches;
    bounds_kernel<<<1, 32, 0, s>>>(subset, sh->m, sh->row0, sh->row0 + sh->n_local, bnd);
    KM2_CUDA(cudaGetLastError());
    long long hb[2] = {0, 0};
    KM2_CUDA(cudaMemcpyAsync(hb, bnd, sizeof(hb), cudaMemcpyDeviceToHost, s));
    KM2_CUDA(cudaStreamSynchronize(s));
    sh->fast_a = hb[0];
    sh->m_local = hb[1] - hb[0];
    const long long list_cap = std::max(sh->n_local, sh->m_local);
    KM2_TRY(alloc_workspace(sh->w, ws, list_cap, k, d, sh->max_iter, s));
    const size_t kd = (size_t)k * d;
    KM2_TRY(ws.alloc((void**)&sh->tot.s_lo, kd * 8, s));
    KM2_TRY(ws.alloc((void**)&sh->tot.s_hi, kd * 8, s));
    KM2_TRY(ws.alloc((void**)&sh->tot.cnt, (size_t)k * 8, s));
    KM2_TRY(ws.alloc((void**)&sh->labels, sizeof(int) * (size_t)sh->n_local, s));
    KM2_TRY(ws.alloc((void**)&sh->labels_s, sizeof(int) * (size_t)sh->m_local, s));
    KM2_TRY(ws.alloc((void**)&sh->Xs, sizeof(float) * (size_t)sh->m_local * d, s));
    if (sh->m_local > 0) {
        long long* mine = subset + sh->fast_a;
        ++g_launches;
        localize_kernel<<<grid_for(sh->m_local), 256, 0, s>>>(mine, sh->m_local, sh->row0);
        KM2_CUDA(cudaGetLastError());
        KM2_CUDA(cudaMemsetAsync(sh->w.st, 0, sizeof(StageState), s));
        KM2_TRY(launch_gather(sh->X, d, mine, sh->m_local, sh->Xs, sh->w.st, s, ws.sm_count));
    }
    if (init_centers)
        KM2_CUDA(cudaMemcpyAsync(sh->w.c.c64, init_centers, sizeof(double) * kd,
                                 is_device_ptr(init_centers) ? cudaMemcpyDeviceToDevice
                                                             : cudaMemcpyHostToDevice, s));
    KM2_CUDA(cudaStreamSynchronize(s));
    return KMEANS2_OK;
}

}  // namespace

extern "C" {

int64_t kmeans2_shard_exchange_elems(int32_t d, int32_t k)
{
    if (d < 1 || k < 1) return -1;
    return partials_count(k, d);
}

int kmeans2_shard_create(const float* X_local, int64_t n_local, int64_t row0, int64_t n_total,
                         int32_t d, int32_t k, double subset_fraction, uint64_t seed, double tol,
                         int32_t max_iter, void* exchange_buf, const kmeans2_options* opt,
                         kmeans2_shard** out)
{
    if (!out) return KMEANS2_ERR_INVALID;
    *out = nullptr;
    if (!valid_shape(n_total, d, k) || n_local < 0 || row0 < 0 || row0 + n_local > n_total ||
        (n_local > 0 && !X_local) || !exchange_buf || !(tol >= 0.0) || max_iter < 1 ||
        !(subset_fraction > 0.0 && subset_fraction <= 1.0))
        return KMEANS2_ERR_INVALID;
    if (!is_device_ptr(exchange_buf) || (reinterpret_cast<uintptr_t>(exchange_buf) & 7) != 0) {
        set_last_error_text("kmeans2_shard_create: the exchange buffer must be 8-byte aligned "
                            "device memory");
        return KMEANS2_ERR_INVALID;
    }
    Resolved r = resolve_options(opt);
    if (r.opt.start_stage != 0 && r.opt.start_stage != 1) return KMEANS2_ERR_INVALID;
    if (r.opt.start_stage == 1 && !r.opt.init_centers) return KMEANS2_ERR_INVALID;
    std::unique_ptr<kmeans2_shard> sh(new kmeans2_shard());
    sh->t0 = std::chrono::steady_clock::now();
    sh->launches0 = g_launches;
    sh->opt = r.opt;
    sh->s = r.stream;
    sh->ws.reset(new DeviceScratch(sh->s));
    sh->n_local = n_local;
    sh->row0 = row0;
    sh->n_total = n_total;
    sh->d = d;
    sh->k = k;
    sh->max_iter = max_iter;
    sh->tol = tol;
    sh->tol_fast = (r.opt.tol_fast > 0.0) ? r.opt.tol_fast : tol;
    sh->x = static_cast<unsigned long long*>(exchange_buf);
    KM2_TRY(shard_setup(sh.get(), X_local, subset_fraction, seed, r.opt.init_centers));
    sh->rr.precision_used = sh->w.form;
    sh->rr.subset_size = sh->m;
    sh->stage = r.opt.start_stage;
    *out = sh.release();
    return KMEANS2_OK;
}

int kmeans2_shard_advance(kmeans2_shard* sh, kmeans2_exchange* next)
{
    if (!sh || !next) return KMEANS2_ERR_INVALID;
    std::memset(next, 0, sizeof(*next));
    if (sh->phase == kPhDone) return KMEANS2_OK;
    if (sh->phase == kPhFailed) return sh->status;
    int rc = KMEANS2_OK;
    switch (sh->phase) {
        case kPhStart:
            if (sh->stage == 0 && !sh->opt.init_centers) {
                const long long kd = (long long)sh->k * sh->d;
                ++g_launches;
                init_contrib_kernel<<<grid_for(kd), 256, 0, sh->s>>>(
                    sh->Xs, sh->fast_a, sh->m_local, sh->d, sh->pos, sh->k,
                    reinterpret_cast<double*>(sh->x));
                cudaError_t e = cudaGetLastError();
                if (e == cudaSuccess) e = cudaStreamSynchronize(sh->s);
                if (e != cudaSuccess) {
                    set_last_error("kmeans2_shard_advance", e);
                    return fail(sh, KMEANS2_ERR_CUDA);
                }
                sh->phase = kPhInitCenters;
                next->op = KMEANS2_XCHG_SUM_F64;
                next->count = kd;
                return KMEANS2_PENDING;
            }
            rc = begin_stage(sh, next);
            break;
        case kPhInitCenters: {
            cudaError_t e = cudaMemcpyAsync(sh->w.c.c64, sh->x, sizeof(double) * sh->k * sh->d,
                                            cudaMemcpyDeviceToDevice, sh->s);
            if (e != cudaSuccess) {
                set_last_error("kmeans2_shard_advance", e);
                return fail(sh, KMEANS2_ERR_CUDA);
            }
            rc = begin_stage(sh, next);
            break;
        }
        case kPhMaxabs: rc = resume_maxabs(sh, next); break;
        case kPhIter: rc = resume_iter(sh, next); break;
        default: rc = KMEANS2_ERR_INVALID;
    }
    if (rc != KMEANS2_OK && rc != KMEANS2_PENDING) return fail(sh, rc);
    return rc;
}

int kmeans2_shard_result(kmeans2_shard* sh, double* centers_out, int32_t* labels_out,
                         kmeans2_result* res)
{
    if (!sh) return KMEANS2_ERR_INVALID;
    if (sh->phase != kPhDone) {
        set_last_error_text("kmeans2_shard_result: the fit has not finished");
        return sh->phase == kPhFailed ? sh->status : KMEANS2_ERR_INVALID;
    }
    cudaStream_t s = sh->s;
    if (centers_out)
        KM2_CUDA(cudaMemcpyAsync(centers_out, sh->w.c.c64, sizeof(double) * sh->k * sh->d,
                                 is_device_ptr(centers_out) ? cudaMemcpyDeviceToDevice
                                                            : cudaMemcpyDeviceToHost, s));
    if (labels_out && sh->n_local > 0)
        KM2_CUDA(cudaMemcpyAsync(labels_out, sh->labels, sizeof(int) * sh->n_local,
                                 is_device_ptr(labels_out) ? cudaMemcpyDeviceToDevice
                                                           : cudaMemcpyDeviceToHost, s));
    KM2_CUDA(cudaStreamSynchronize(s));
    if (res) {
        *res = sh->rr;
        res->seconds =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - sh->t0).count();
    }
    if (sh->opt.profile) sh->opt.profile->kernel_launches += g_launches - sh->launches0;
    return KMEANS2_OK;
}

void kmeans2_shard_destroy(kmeans2_shard* sh)
{
    if (!sh) return;
    cudaStreamSynchronize(sh->s);
    delete sh;
}

int kmeans2_fit_sharded(const float* X, int64_t n, int32_t d, int32_t k, double subset_fraction,
                        uint64_t seed, double tol, int32_t max_iter, int32_t shards,
                        double* centers_out, int32_t* labels_out, kmeans2_result* res,
                        const kmeans2_options* opt)
{
    auto t0 = std::chrono::steady_clock::now();
    if (!X || !centers_out || !labels_out || !valid_shape(n, d, k) || shards < 1 ||
        shards > kMaxShards || !(subset_fraction > 0.0 && subset_fraction <= 1.0) ||
        !(tol >= 0.0) || max_iter < 1)
        return KMEANS2_ERR_INVALID;
    Resolved r = resolve_options(opt);
    cudaStream_t s = r.stream;
    DeviceScratch ws(s);
    const float* Xd = nullptr;
    KM2_TRY(device_view(X, (long long)n * d, &Xd, ws, s));
    const int P = shards;
    // shard r holds rows [row0[r], row0[r + 1]); boundaries on multiples of 4
    // rows keep every shard 16-byte aligned
    std::vector<long long> row0(P + 1);
    for (int i = 0; i <= P; ++i) row0[i] = (i == P) ? n : ((long long)n * i / P) & ~3ll;
    const long long E = partials_count(k, d);
    XchgPtrs ptrs{};
    for (int i = 0; i < P; ++i)
        KM2_TRY(ws.alloc((void**)&ptrs.p[i], (size_t)E * 8, s));
    kmeans2_options so = r.opt;
    so.stream = s;
    so.profile = nullptr;
    std::vector<kmeans2_shard*> sh(P, nullptr);
    struct Guard {
        std::vector<kmeans2_shard*>& v;
        ~Guard() { for (auto* p : v) kmeans2_shard_destroy(p); }
    } guard{sh};
    for (int i = 0; i < P; ++i) {
        kmeans2_options oi = so;
        if (i > 0) oi.traj_J_fast = oi.traj_J_slow = oi.traj_shift_fast = oi.traj_shift_slow = nullptr;
        KM2_TRY(kmeans2_shard_create(Xd + (size_t)row0[i] * d, row0[i + 1] - row0[i], row0[i], n,
                                     d, k, subset_fraction, seed, tol, max_iter, ptrs.p[i], &oi,
                                     &sh[i]));
    }
    std::vector<kmeans2_exchange> xs(P);
    for (;;) {
        int rc0 = 0;
        for (int i = 0; i < P; ++i) {
            int rc = kmeans2_shard_advance(sh[i], &xs[i]);
            if (rc < 0) return rc;
            if (i == 0) rc0 = rc;
            if (rc != rc0 || xs[i].op != xs[0].op || xs[i].count != xs[0].count) {
                set_last_error_text("kmeans2_fit_sharded: shards disagree on the next exchange");
                return KMEANS2_ERR_CUDA;
            }
        }
        if (rc0 == KMEANS2_OK) break;
        ++g_launches;
        xchg_reduce_kernel<<<grid_for(xs[0].count), 256, 0, s>>>(ptrs, P, xs[0].count, xs[0].op);
        KM2_CUDA(cudaGetLastError());
    }
    // every replica holds the same centers
    const size_t kd = (size_t)k * d;
    std::vector<double> c0(kd), ci(kd);
    kmeans2_result rr{};
    for (int i = 0; i < P; ++i) {
        kmeans2_result ri{};
        KM2_TRY(kmeans2_shard_result(sh[i], i == 0 ? c0.data() : ci.data(),
                                     labels_out + row0[i], &ri));
        if (i == 0) rr = ri;
        else {
            rr.rechecked_points += ri.rechecked_points;
            if (std::memcmp(c0.data(), ci.data(), kd * sizeof(double)) != 0) {
                set_last_error_text("kmeans2_fit_sharded: shard replicas diverged");
                return KMEANS2_ERR_CUDA;
            }
        }
    }
    KM2_CUDA(cudaMemcpyAsync(centers_out, c0.data(), kd * sizeof(double),
                             is_device_ptr(centers_out) ? cudaMemcpyHostToDevice
                                                        : cudaMemcpyHostToHost, s));
    KM2_CUDA(cudaStreamSynchronize(s));
    rr.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (res) *res = rr;
    return KMEANS2_OK;
}

}  // extern "C"
