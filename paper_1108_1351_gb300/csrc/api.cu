// api.cu -- the C ABI of libkmeans2 and the host-side orchestration of the
// two-stage method (Section 2, Algorithm): draw S_s and the initial centers,
// run the Lloyd loop on S_s (fast stage), then on S_n from the fast stage's
// final centers (slow stage).
//
// One stage = stage_init, then per iteration: assign (fused distance, argmin,
// exact sums) -> recheck (FP64 near ties) -> finalize (means, movement, J,
// loop control).  With use_graph the iteration body is captured once into the
// body of a CUDA-graph WHILE node whose condition finalize sets on the device,
// so a whole stage is one graph launch with no host round trip per iteration.
#include <algorithm>
#include <cfloat>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "api_internal.h"

namespace km2 {

// NVTX range for the lifetime of the object (header-only NVTX v3: a no-op
// unless a profiler is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

thread_local long long g_launches = 0;

namespace {
thread_local char g_last_error[512] = "";
}

void set_last_error(const char* where, cudaError_t e)
{
    std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%d)", where, cudaGetErrorString(e),
                  (int)e);
}

void set_last_error_text(const char* text)
{
    std::snprintf(g_last_error, sizeof(g_last_error), "%s", text);
}

const char* last_error() { return g_last_error; }

namespace {
std::mutex g_attr_mu;
std::vector<std::pair<const void*, int>> g_attr_done;   // (kernel, device) already raised
}

int set_max_dynamic_smem(const void* kernel, int bytes)
{
    int dev = 0;
    KM2_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_attr_mu);
    for (const auto& e : g_attr_done)
        if (e.first == kernel && e.second == dev) return KMEANS2_OK;
    KM2_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    g_attr_done.emplace_back(kernel, dev);
    return KMEANS2_OK;
}

int consumer_wait_tries(int normal)
{
#ifdef KM2_DEBUG_CHECKS
    const char* v = std::getenv("KMEANS2_DEBUG_WAIT_TRIES");
    if (v && *v) {
        const long t = std::strtol(v, nullptr, 10);
        if (t >= 0 && t < normal) return (int)t;
    }
#endif
    return normal;
}

// A private blocking stream per thread and device, used when the caller passes
// the legacy default stream (which cannot be captured into a graph).
cudaStream_t private_stream(int device)
{
    static thread_local cudaStream_t streams[64] = {};
    if (device < 0 || device >= 64) return nullptr;
    if (!streams[device]) cudaStreamCreate(&streams[device]);
    return streams[device];
}

namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {};
}

// The library's stream-ordered pool on `device`: it keeps freed memory mapped
// (no release threshold), so repeated calls reuse their scratch instead of
// mapping it again each time (kmeans2_release_memory trims it).
cudaMemPool_t library_pool(int device)
{
    if (device < 0 || device >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[device]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        unsigned long long keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pools[device] = pool;
    }
    return g_pools[device];
}

cudaError_t pool_malloc_async(void** p, size_t bytes, cudaStream_t s)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaMemPool_t pool = library_pool(dev);
    return pool ? cudaMallocFromPoolAsync(p, bytes, pool, s) : cudaMallocAsync(p, bytes, s);
}

DeviceScratch::DeviceScratch(cudaStream_t s) : stream(s)
{
    cudaGetDevice(&device);
    cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, device);
    if (sm_count < 1) sm_count = 1;
}

DeviceScratch::DeviceScratch(cudaStream_t s, void* arena_base, size_t bytes)
    : DeviceScratch(s)
{
    arena = static_cast<unsigned char*>(arena_base);
    arena_bytes = bytes;
}

DeviceScratch::~DeviceScratch()
{
    for (void* p : ptrs) cudaFreeAsync(p, stream);
}

int DeviceScratch::alloc(void** p, size_t bytes, cudaStream_t s)
{
    if (bytes == 0) bytes = 16;
    if (arena) {
        size_t off = (arena_used + 255) & ~(size_t)255;
        if (off + bytes > arena_bytes) {
            set_last_error_text("fixed scratch area too small for this call");
            *p = nullptr;
            return KMEANS2_ERR_INVALID;
        }
        *p = arena + off;
        arena_used = off + bytes;
        return KMEANS2_OK;
    }
    cudaMemPool_t pool = library_pool(device);
    cudaError_t e = pool ? cudaMallocFromPoolAsync(p, bytes, pool, s) : cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        set_last_error("cudaMallocFromPoolAsync", e);
        cudaGetLastError();
        *p = nullptr;
        return KMEANS2_ERR_NOMEM;
    }
    ptrs.push_back(*p);
    return KMEANS2_OK;
}

// ---------------------------------------------------------------- stage plumbing

__global__ void fill_f32_kernel(float* p, long long count, float v)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

int fill_f32(float* p, long long count, float v, cudaStream_t s)
{
    if (count <= 0) return KMEANS2_OK;
    int grid = (int)((count + 255) / 256);
    if (grid > 1024) grid = 1024;
    ++g_launches;
    fill_f32_kernel<<<grid, 256, 0, s>>>(p, count, v);
    KM2_CUDA(cudaGetLastError());
    return KMEANS2_OK;
}

// True if p is memory the current device addresses as device memory.
bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}


int alloc_workspace(Workspace& w, DeviceScratch& ws, long long list_cap, int k, int d,
                    int max_iter, cudaStream_t s)
{
    w.c.k = k;
    w.c.d = d;
    w.c.kpad = (k + 127) / 128 * 128;
    w.c.dpad = (d + 7) / 8 * 8;
    w.max_iter = max_iter;
    w.ws = &ws;
    size_t kd = (size_t)k * d;
    KM2_TRY(ws.alloc((void**)&w.c.c64, kd * sizeof(double), s));
    KM2_TRY(ws.alloc((void**)&w.c.c32, kd * sizeof(float), s));
    KM2_TRY(ws.alloc((void**)&w.c.c32t, (size_t)w.c.dpad * w.c.kpad * sizeof(float), s));
    const long long cn_len = std::max((long long)w.c.kpad, (long long)(k + 255) / 256 * 256);
    KM2_TRY(ws.alloc((void**)&w.c.cnorm, (size_t)cn_len * sizeof(float), s));
    KM2_TRY(ws.alloc((void**)&w.acc.s_lo, kd * 8, s));
    KM2_TRY(ws.alloc((void**)&w.acc.s_hi, kd * 8, s));
    KM2_TRY(ws.alloc((void**)&w.acc.cnt, (size_t)k * 8, s));
    KM2_TRY(ws.alloc((void**)&w.st, sizeof(StageState), s));
    KM2_TRY(ws.alloc((void**)&w.list, (size_t)(list_cap > 0 ? list_cap : 1) * sizeof(int), s));
    KM2_TRY(ws.alloc((void**)&w.clus, (size_t)kClusSlots * k * sizeof(double), s));
    KM2_TRY(ws.alloc((void**)&w.traj_J, (size_t)max_iter * sizeof(double), s));
    KM2_TRY(ws.alloc((void**)&w.traj_shift, (size_t)max_iter * sizeof(double), s));
    KM2_CUDA(cudaMemsetAsync(w.c.c32t, 0, (size_t)w.c.dpad * w.c.kpad * sizeof(float), s));
    // padding centers: the largest finite key, so that packing an index into
    // its low mantissa bits never makes a NaN and it never wins or ties
    KM2_TRY(fill_f32(w.c.cnorm, cn_len, FLT_MAX, s));
    // (the split layout: a fit may switch from FP16 to split BF16 between stages)
    if (tc16_form(w.form)) KM2_TRY(ws.alloc((void**)&w.cb, bf16_cb_bytes(d, k, 0), s));
    return KMEANS2_OK;
}

// 16-bit tensor-core forms: per-stage copy of the stage's points as BF16
// (FP16) tiles + ||x||^2.  After stage_init: the FP16 scale depends on F.
int prepare_stage_points(const float* X, long long n, int d, Workspace& w, DeviceScratch& ws,
                         cudaStream_t s)
{
    if (!tc16_form(w.form)) return KMEANS2_OK;
    const int single = w.form == KMEANS2_PRECISION_FP16;
    KM2_TRY(ws.alloc((void**)&w.xt, bf16_xt_bytes(n, d, single), s));
    KM2_TRY(ws.alloc((void**)&w.xn2, (size_t)n * sizeof(float), s));
    if (single) {
        // the second pass's buffers for this stage's undecided rows
        StageB& b = w.sb;
        b.cap = stage_b_cap(n);
        KM2_TRY(ws.alloc((void**)&b.Xc, (size_t)b.cap * d * sizeof(float), s));
        KM2_TRY(ws.alloc((void**)&b.Xt, bf16_xt_bytes(b.cap, d, 0), s));
        KM2_TRY(ws.alloc((void**)&b.xn2, (size_t)b.cap * sizeof(float), s));
        KM2_TRY(ws.alloc((void**)&b.lab, (size_t)b.cap * sizeof(int), s));
        KM2_TRY(ws.alloc((void**)&b.list, (size_t)b.cap * sizeof(int), s));
        KM2_TRY(ws.alloc((void**)&b.st, sizeof(StageState), s));
        KM2_TRY(ws.alloc((void**)&b.nb, sizeof(long long), s));
        if (!b.cb) KM2_TRY(ws.alloc((void**)&b.cb, bf16_cb_bytes(d, w.c.k, 0), s));
    }
    return launch_convert_x_bf16(X, n, d, w.xt, w.xn2, w.st, single, s, ws.sm_count);
}

// The fused distance kernel of the chosen form.
int launch_assign(const float* X, long long n, int d, Workspace& w, int* labels, cudaStream_t s,
                  int sm_count)
{
    if (w.form == KMEANS2_PRECISION_TF32X3)
        return launch_assign_tc32(X, n, d, w.c, labels, w.st, w.acc, w.list, s, sm_count);
    if (w.form == KMEANS2_PRECISION_FP16) {
        KM2_TRY(launch_assign_bf16(X, w.xt, w.xn2, w.cb, n, d, w.c, labels, w.st, w.acc, w.list,
                                   1, s, sm_count));
        return launch_stage_b(X, d, w.c, labels, w.st, w.acc, w.list, w.sb, s, sm_count);
    }
    if (tc16_form(w.form))
        return launch_assign_bf16(X, w.xt, w.xn2, w.cb, n, d, w.c, labels, w.st, w.acc, w.list,
                                  0, s, sm_count);
    return launch_assign_fp32(X, n, d, w.c, labels, w.st, w.acc, w.list, s, sm_count);
}

// Resolve the requested precision to the form this shape runs in.
int choose_form(int requested, int d, int k, const float* X, int* form)
{
    const bool tc = assign_tc32_supported(d, k, X) != 0;
    const bool bf = assign_bf16_supported(d, k, X) != 0;
    switch (requested) {
        case KMEANS2_PRECISION_FP32: *form = KMEANS2_PRECISION_FP32; return KMEANS2_OK;
        case KMEANS2_PRECISION_BF16:
            if (!bf) {
                set_last_error_text("the BF16 tensor-core form needs d a multiple of 16 in "
                                    "[16, 128] and 16-byte aligned X");
                return KMEANS2_ERR_UNSUPPORTED;
            }
            *form = KMEANS2_PRECISION_BF16;
            return KMEANS2_OK;
        case KMEANS2_PRECISION_FP16:
            if (!bf) {
                set_last_error_text("the FP16 tensor-core form needs d a multiple of 16 in "
                                    "[16, 128] and 16-byte aligned X");
                return KMEANS2_ERR_UNSUPPORTED;
            }
            *form = KMEANS2_PRECISION_FP16;
            return KMEANS2_OK;
        case KMEANS2_PRECISION_TF32X3:
            if (!tc) {
                set_last_error_text("the 3xTF32 tensor-core form needs d in {4, 8, 16, 32}, "
                                    "k <= 256 and 16-byte aligned X");
                return KMEANS2_ERR_UNSUPPORTED;
            }
            *form = KMEANS2_PRECISION_TF32X3;
            return KMEANS2_OK;
        case KMEANS2_PRECISION_AUTO:
            // For d <= 32 the CUDA-core form is as fast per launch as the tensor-core
            // forms and flags far fewer near ties (measured).  From d = 64 on the
            // BF16 tensor-core form wins once k is large (k >= 512: 1.1-2.5x
            // faster fits); with fewer centers the CUDA-core kernel is fast
            // enough that the BF16 form's 5-10x more near-tie rechecks lose
            // (measured on Gaussian mixtures of 4 to 1024 components).
            *form = (bf && d >= 64 && k >= 512) ? KMEANS2_PRECISION_BF16 : KMEANS2_PRECISION_FP32;
            return KMEANS2_OK;
        default:
            set_last_error_text("unknown precision form");
            return KMEANS2_ERR_UNSUPPORTED;
    }
}

// One Lloyd iteration: assign -> recheck -> finalize.
int launch_iteration(const float* X, long long n, int d, Workspace& w, int* labels,
                     unsigned long long handle, int use_cond, cudaStream_t s, int sm_count)
{
    KM2_TRY(launch_assign(X, n, d, w, labels, s, sm_count));
    KM2_TRY(launch_recheck(X, d, w.c, labels, w.list, w.st, w.acc, s, sm_count));
    KM2_TRY(launch_finalize(w.acc, w.c, w.st, w.traj(), w.clus, handle, use_cond,
                            s));
    return KMEANS2_OK;
}

// The stage loop as one graph: a WHILE conditional node whose body is one iteration.
int run_loop_graph(const float* X, long long n, int d, Workspace& w, int* labels, cudaStream_t s,
                   int sm_count)
{
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int rc = KMEANS2_OK;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e != cudaSuccess) { set_last_error("cudaGraphCreate", e); return KMEANS2_ERR_CUDA; }
    do {
        cudaGraphConditionalHandle handle;
        e = cudaGraphConditionalHandleCreate(&handle, graph, 1u, cudaGraphCondAssignDefault);
        if (e != cudaSuccess) { set_last_error("cudaGraphConditionalHandleCreate", e); rc = KMEANS2_ERR_CUDA; break; }
        // cudaGraphNodeParams has no default constructor: build it zeroed in raw storage.
        alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
        std::memset(raw, 0, sizeof(raw));
        cudaGraphNodeParams* p = reinterpret_cast<cudaGraphNodeParams*>(raw);
        p->type = cudaGraphNodeTypeConditional;
        p->conditional.handle = handle;
        p->conditional.type = cudaGraphCondTypeWhile;
        p->conditional.size = 1;
        cudaGraphNode_t node;
        e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, p);
        if (e != cudaSuccess) { set_last_error("cudaGraphAddNode", e); rc = KMEANS2_ERR_CUDA; break; }
        cudaGraph_t body = p->conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { set_last_error("cudaStreamBeginCaptureToGraph", e); rc = KMEANS2_ERR_CUDA; break; }
        const long long body0 = g_launches;
        rc = launch_iteration(X, n, d, w, labels, (unsigned long long)handle, 1, s, sm_count);
        const long long body_launches = g_launches - body0;
        cudaGraph_t captured = nullptr;
        e = cudaStreamEndCapture(s, &captured);
        if (rc != KMEANS2_OK) break;
        if (e != cudaSuccess) { set_last_error("cudaStreamEndCapture", e); rc = KMEANS2_ERR_CUDA; break; }
        e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) { set_last_error("cudaGraphInstantiate", e); rc = KMEANS2_ERR_CUDA; break; }
        e = cudaGraphLaunch(exec, s);
        if (e != cudaSuccess) { set_last_error("cudaGraphLaunch", e); rc = KMEANS2_ERR_CUDA; break; }
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { set_last_error("cudaStreamSynchronize", e); rc = KMEANS2_ERR_CUDA; break; }
        int iters = 0;
        // stream-ordered read: a legacy-stream copy would wait for every other stream
        e = cudaMemcpyAsync(&iters, &w.st->iter, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { set_last_error("cudaMemcpyAsync", e); rc = KMEANS2_ERR_CUDA; break; }
        // the capture counted the body's kernels once; each further iteration reruns them
        g_launches += body_launches * (iters > 1 ? iters - 1 : 0);
    } while (0);
    if (exec) cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    return rc;
}

// Host-driven loop; with a profile, CUDA events bracket each distance-kernel launch.
int run_loop_host(const float* X, long long n, int d, Workspace& w, int* labels, int max_iter,
                  cudaStream_t s, int sm_count, kmeans2_profile* prof)
{
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (prof) {
        KM2_CUDA(cudaEventCreate(&ev0));
        KM2_CUDA(cudaEventCreate(&ev1));
    }
    int rc = KMEANS2_OK;
    for (int it = 0; it < max_iter && rc == KMEANS2_OK; ++it) {
        NvtxRange iteration_range("kmeans2 iteration");
        if (prof) {
            cudaEventRecord(ev0, s);
            rc = launch_assign(X, n, d, w, labels, s, sm_count);
            cudaEventRecord(ev1, s);
            if (rc == KMEANS2_OK)
                rc = launch_recheck(X, d, w.c, labels, w.list, w.st, w.acc, s, sm_count);
            if (rc == KMEANS2_OK)
                rc = launch_finalize(w.acc, w.c, w.st, w.traj(), w.clus, 0ull, 0, s);
        } else {
            rc = launch_iteration(X, n, d, w, labels, 0ull, 0, s, sm_count);
        }
        if (rc != KMEANS2_OK) break;
        int done = 0;
        cudaError_t e = cudaMemcpyAsync(&done, &w.st->done, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { set_last_error("stage loop", e); rc = KMEANS2_ERR_CUDA; break; }
        if (prof) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev0, ev1);
            prof->assign_launches += 1;
            prof->assign_ms += ms;
            prof->assign_flops += 2.0 * (double)n * w.c.k * d;
            prof->assign_bytes += 4.0 * (double)n * d;
        }
        if (done) break;
    }
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    return rc;
}

int map_stage_error(int err)
{
    if (err == kErrNonFinite) {
        set_last_error_text("X holds a NaN or an infinity");
        return KMEANS2_ERR_NONFINITE;
    }
    if (err == kErrTimeout) {
        set_last_error_text("a device-side wait on the tensor-core pipeline timed out");
        return KMEANS2_ERR_TIMEOUT;
    }
    if (err == kErrBounds) {
        set_last_error_text("a device-side index check failed (debug build)");
        return KMEANS2_ERR_CUDA;
    }
    set_last_error_text("max|x| >= 2^50 is outside the supported range");
    return KMEANS2_ERR_UNSUPPORTED;
}

// Run one stage on device-resident X (n x d) from the centers in w.c (FP64
// master already set).  The caller has zeroed w.st and recorded max|x| in it.
// Share of a stage's rows the single-pass FP16 form may leave undecided in its
// first iteration before an AUTO fit moves that stage to the split form.
constexpr double kFp16ProbeMaxUndecided = 0.10;

int run_stage(const float* X, long long n, int d, Workspace& w, int* labels, double tol,
              int max_iter, bool use_graph, cudaStream_t s, int sm_count, StageState& out,
              double* traj_J_host, double* traj_shift_host, kmeans2_profile* prof,
              const char* name = "kmeans2 stage", double* traj_c_host = nullptr,
              int64_t* traj_n_host = nullptr, bool probe16 = false)
{
    NvtxRange stage_range(name);
    size_t kd = (size_t)w.c.k * d;
    KM2_CUDA(cudaMemsetAsync(w.acc.s_lo, 0, kd * 8, s));
    KM2_CUDA(cudaMemsetAsync(w.acc.s_hi, 0, kd * 8, s));
    KM2_CUDA(cudaMemsetAsync(w.acc.cnt, 0, (size_t)w.c.k * 8, s));
    KM2_TRY(launch_center_prep(w.c, w.st, s));
    KM2_TRY(launch_stage_init(w.st, d, tol, max_iter, s));
    KM2_TRY(launch_qsum(X, n, d, w.st, s, sm_count));
    KM2_TRY(prepare_stage_points(X, n, d, w, *w.ws, s));
    bool finished = false;
    int remaining = max_iter;
    if (probe16 && w.form == KMEANS2_PRECISION_FP16) {
        // one FP16 iteration from the host; if its single pass left too many
        // rows undecided, the rest of the stage runs the split form (every
        // form decides each row exactly, so the switch changes no result)
        KM2_TRY(run_loop_host(X, n, d, w, labels, 1, s, sm_count, prof));
        StageState p;
        KM2_CUDA(cudaMemcpyAsync(&p, w.st, sizeof(StageState), cudaMemcpyDeviceToHost, s));
        KM2_CUDA(cudaStreamSynchronize(s));
        finished = p.done != 0 || p.error != 0;
        remaining = max_iter - 1;
        if (!finished && (double)p.undecided16_total > kFp16ProbeMaxUndecided * (double)n) {
            w.form = KMEANS2_PRECISION_BF16;
            KM2_TRY(prepare_stage_points(X, n, d, w, *w.ws, s));
        }
    }
    if (!finished) {
        if (use_graph && !prof)
            KM2_TRY(run_loop_graph(X, n, d, w, labels, s, sm_count));
        else
            KM2_TRY(run_loop_host(X, n, d, w, labels, remaining, s, sm_count, prof));
    }
    KM2_CUDA(cudaMemcpyAsync(&out, w.st, sizeof(StageState), cudaMemcpyDeviceToHost, s));
    KM2_CUDA(cudaStreamSynchronize(s));
    if (out.error) return map_stage_error(out.error);
    if (traj_J_host && out.iter > 0)
        KM2_CUDA(cudaMemcpyAsync(traj_J_host, w.traj_J, sizeof(double) * out.iter,
                                 cudaMemcpyDeviceToHost, s));
    if (traj_shift_host && out.iter > 0)
        KM2_CUDA(cudaMemcpyAsync(traj_shift_host, w.traj_shift, sizeof(double) * out.iter,
                                 cudaMemcpyDeviceToHost, s));
    if (traj_c_host && w.traj_c && out.iter > 0)
        KM2_CUDA(cudaMemcpyAsync(traj_c_host, w.traj_c,
                                 sizeof(double) * (size_t)out.iter * w.c.k * d,
                                 cudaMemcpyDeviceToHost, s));
    if (traj_n_host && w.traj_n && out.iter > 0)
        KM2_CUDA(cudaMemcpyAsync(traj_n_host, w.traj_n, sizeof(int64_t) * (size_t)out.iter * w.c.k,
                                 cudaMemcpyDeviceToHost, s));
    KM2_CUDA(cudaStreamSynchronize(s));
    return KMEANS2_OK;
}

bool valid_shape(long long n, int d, int k)
{
    return n >= 1 && d >= 1 && d <= 4096 && k >= 1 && k <= n && n < (1ll << 31) &&
           (long long)k * d <= (1ll << 24);
}

// Device-resident, 16-byte aligned view of X (staged through scratch when needed).
int device_view(const float* X, long long count, const float** out, DeviceScratch& ws,
                cudaStream_t s)
{
    bool dev = is_device_ptr(X);
    if (dev && (reinterpret_cast<uintptr_t>(X) & 15) == 0) {
        *out = X;
        return KMEANS2_OK;
    }
    float* buf = nullptr;
    KM2_TRY(ws.alloc((void**)&buf, (size_t)count * sizeof(float), s));
    KM2_CUDA(cudaMemcpyAsync(buf, X, (size_t)count * sizeof(float),
                             dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    *out = buf;
    return KMEANS2_OK;
}

Resolved resolve_options(const kmeans2_options* opt)
{
    Resolved r;
    kmeans2_default_options(&r.opt);
    if (opt) r.opt = *opt;
    r.stream = static_cast<cudaStream_t>(r.opt.stream);
    if (!r.stream) {
        int dev = 0;
        cudaGetDevice(&dev);
        r.stream = private_stream(dev);
    }
    return r;
}



// ---------------------------------------------------------------- fixed scratch
// Scratch of kmeans_step_noalloc: one file-scope device array, present on every
// GPU that loads this library until the process exits.  Its size bounds the
// shapes that entry point accepts (see kNoAlloc* below).
constexpr size_t kNoAllocBytes = 24ull << 20;           // 24 MiB per GPU
constexpr long long kNoAllocMaxN = 1ll << 22;           // points
constexpr int kNoAllocMaxK = 1024;                      // centers
constexpr int kNoAllocMaxD = 128;                       // dimensions
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {};

// Device address of g_noalloc_scratch on the current device, looked up once per
// device (in host code the symbol names a host-side stand-in, not device memory).
int noalloc_scratch(void** out)
{
    int dev = 0;
    KM2_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return KMEANS2_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        KM2_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return KMEANS2_OK;
}
}  // namespace

}  // namespace km2

using namespace km2;

extern "C" {

void kmeans2_default_options(kmeans2_options* opt)
{
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = KMEANS2_PRECISION_AUTO;
    opt->deterministic = 1;
    opt->use_graph = 1;
}

int64_t kmeans2_subset_size(int64_t n, int32_t k, double f)
{
    if (n < 1 || k < 1 || k > n || !(f > 0.0 && f <= 1.0)) return -1;
    double want = std::ceil(f * (double)n);
    int64_t m = (int64_t)want;
    if (m < k) m = k;
    if (m > n) m = n;
    return m;
}

const char* kmeans2_strerror(int status)
{
    switch (status) {
        case KMEANS2_OK: return "ok";
        case KMEANS2_PENDING: return "pending";
        case KMEANS2_ERR_INVALID: return "invalid argument";
        case KMEANS2_ERR_NOMEM: return "out of memory";
        case KMEANS2_ERR_CUDA: return "CUDA error";
        case KMEANS2_ERR_NONFINITE: return "input holds NaN or infinity";
        case KMEANS2_ERR_TIMEOUT: return "device wait timed out";
        case KMEANS2_ERR_ADMISSION: return "admission refused";
        case KMEANS2_ERR_UNSUPPORTED: return "unsupported shape or mode";
        default: return "unknown status";
    }
}

const char* kmeans2_last_error(void) { return km2::last_error(); }

uint64_t kmeans2_fit_footprint(int64_t n, int32_t d, int32_t k, double subset_fraction,
                               int32_t max_iter, int32_t precision, int32_t x_on_host,
                               int32_t labels_on_host)
{
    if (!valid_shape(n, d, k) || !(subset_fraction > 0.0 && subset_fraction <= 1.0) ||
        max_iter < 1)
        return 0;
    int form = KMEANS2_PRECISION_FP32;
    const float* aligned = reinterpret_cast<const float*>(static_cast<uintptr_t>(256));
    if (choose_form(precision, d, k, aligned, &form) != KMEANS2_OK) return 0;
    const unsigned long long m = (unsigned long long)kmeans2_subset_size(n, k, subset_fraction);
    const unsigned long long N = (unsigned long long)n, K = (unsigned long long)k,
                             D = (unsigned long long)d;
    const unsigned long long kpad = (K + 127) / 128 * 128, dpad = (D + 7) / 8 * 8;
    const unsigned long long kd = K * D;
    unsigned long long b = 0;
    int allocs = 0;
    auto add = [&](unsigned long long bytes) { b += bytes; ++allocs; };
    if (x_on_host) add(N * D * 4);
    // workspace
    add(kd * 8);
    add(kd * 4);
    add(dpad * kpad * 4);
    add(std::max(kpad, (K + 255) / 256 * 256) * 4);
    add(kd * 8);
    add(kd * 8);
    add(K * 8);
    add(sizeof(StageState));
    add(N * 4);
    add((unsigned long long)kClusSlots * K * 8);
    add(2 * (unsigned long long)max_iter * 8);
    if (tc16_form(form)) add(bf16_cb_bytes(d, k, 0));
    if (labels_on_host) add(N * 4);
    // fast stage: S_s indices, init positions, X_s, its labels
    add(m * 8);
    add(K * 8);
    add(m * D * 4);
    add(m * 4);
    // sampling scratch: two radix selects (candidate buffer ~ count / 2048 keys,
    // per-chunk counts and offsets) and the k selected positions
    for (unsigned long long cnt : {N, m}) {
        add(4096 + 2048 * 4);
        add((2 * cnt / 2048 + 4096) * 8);
        add((cnt + 4095) / 4096 * 12);
    }
    add(K * 8);
    if (tc16_form(form)) {
        // a stage's 16-bit tiles and ||x||^2, and for the single-pass form its
        // second pass's compact rows; AUTO (FP16 fast stage, then FP16 or split
        // BF16) counts the larger slow stage
        auto second = [&](long long rows) {
            const unsigned long long cap = (unsigned long long)stage_b_cap(rows);
            add(cap * D * 4);
            add(bf16_xt_bytes((long long)cap, d, 0));
            add(cap * 12);
            add(sizeof(StageState) + 8);
        };
        const bool adaptive = precision == KMEANS2_PRECISION_AUTO;
        const int single = form == KMEANS2_PRECISION_FP16 || adaptive;
        add(bf16_xt_bytes((long long)m, d, single));
        add(m * 4);
        if (single) second((long long)m);
        if (single && !adaptive) {
            add(bf16_xt_bytes(n, d, 1));
            second(n);
        } else if (!single) {
            add(bf16_xt_bytes(n, d, 0));
        } else {
            const unsigned long long b0 = b;
            const int a0 = allocs;
            add(bf16_xt_bytes(n, d, 1));
            second(n);
            const unsigned long long fp16_slow = b - b0;
            b = b0;
            allocs = a0 + 5;
            b += std::max(fp16_slow, (unsigned long long)bf16_xt_bytes(n, d, 0));
        }
        add(N * 4);
        if (single) add(bf16_cb_bytes(d, k, 0));
    }
    return b + (unsigned long long)allocs * 1024ull + (4ull << 20);
}

int32_t kmeans2_version(void) { return (1 << 16) | 0; }

int kmeans2_release_memory(void)
{
    int dev = 0;
    KM2_CUDA(cudaGetDevice(&dev));
    cudaMemPool_t pool = library_pool(dev);
    if (!pool) return KMEANS2_ERR_CUDA;
    KM2_CUDA(cudaDeviceSynchronize());
    KM2_CUDA(cudaMemPoolTrimTo(pool, 0));
    return KMEANS2_OK;
}

int kmeans2_sample(int64_t n, int32_t k, double f, uint64_t seed, int64_t* subset_out,
                   int64_t* init_pos_out, void* stream)
{
    int64_t m = kmeans2_subset_size(n, k, f);
    if (m < 0 || !subset_out || !init_pos_out || n >= (1ll << 40)) return KMEANS2_ERR_INVALID;
    kmeans2_options o;
    kmeans2_default_options(&o);
    o.stream = stream;
    Resolved r = resolve_options(&o);
    cudaStream_t s = r.stream;
    DeviceScratch ws(s);
    bool sub_dev = is_device_ptr(subset_out), pos_dev = is_device_ptr(init_pos_out);
    long long* sub = sub_dev ? (long long*)subset_out : nullptr;
    long long* pos = pos_dev ? (long long*)init_pos_out : nullptr;
    if (!sub) KM2_TRY(ws.alloc((void**)&sub, sizeof(long long) * (size_t)m, s));
    if (!pos) KM2_TRY(ws.alloc((void**)&pos, sizeof(long long) * (size_t)k, s));
    KM2_TRY(sample_device(n, k, m, seed, sub, pos, s, ws));
    if (!sub_dev)
        KM2_CUDA(cudaMemcpyAsync(subset_out, sub, sizeof(long long) * (size_t)m,
                                 cudaMemcpyDeviceToHost, s));
    if (!pos_dev)
        KM2_CUDA(cudaMemcpyAsync(init_pos_out, pos, sizeof(long long) * (size_t)k,
                                 cudaMemcpyDeviceToHost, s));
    KM2_CUDA(cudaStreamSynchronize(s));
    return KMEANS2_OK;
}

int kmeans_step(const float* X, int64_t n, int32_t d, int32_t k, const double* centers_in,
                double* centers_out, int32_t* labels_out, double* J_out, double* shift_out,
                int32_t* empty_out, const kmeans2_options* opt)
{
    if (!X || !centers_in || !centers_out || !labels_out || !valid_shape(n, d, k))
        return KMEANS2_ERR_INVALID;
    Resolved r = resolve_options(opt);
    const long long launches0 = g_launches;
    cudaStream_t s = r.stream;
    DeviceScratch ws(s);
    const float* Xd = nullptr;
    KM2_TRY(device_view(X, (long long)n * d, &Xd, ws, s));
    Workspace w;
    KM2_TRY(choose_form(r.opt.precision, d, k, Xd, &w.form));
    KM2_TRY(alloc_workspace(w, ws, n, k, d, 1, s));
    bool lab_dev = is_device_ptr(labels_out) && (reinterpret_cast<uintptr_t>(labels_out) & 3) == 0;
    int* labels = lab_dev ? labels_out : nullptr;
    if (!labels) KM2_TRY(ws.alloc((void**)&labels, sizeof(int) * (size_t)n, s));
    KM2_CUDA(cudaMemcpyAsync(w.c.c64, centers_in, sizeof(double) * (size_t)k * d,
                             is_device_ptr(centers_in) ? cudaMemcpyDeviceToDevice
                                                       : cudaMemcpyHostToDevice, s));
    KM2_CUDA(cudaMemsetAsync(w.st, 0, sizeof(StageState), s));
    KM2_TRY(launch_maxabs(Xd, n, d, w.st, s, ws.sm_count));
    StageState out;
    KM2_TRY(run_stage(Xd, n, d, w, labels, 0.0, 1, false, s, ws.sm_count, out, nullptr, nullptr,
                      r.opt.profile));
    KM2_CUDA(cudaMemcpyAsync(centers_out, w.c.c64, sizeof(double) * (size_t)k * d,
                             is_device_ptr(centers_out) ? cudaMemcpyDeviceToDevice
                                                        : cudaMemcpyDeviceToHost, s));
    if (!lab_dev)
        KM2_CUDA(cudaMemcpyAsync(labels_out, labels, sizeof(int) * (size_t)n,
                                 is_device_ptr(labels_out) ? cudaMemcpyDeviceToDevice
                                                           : cudaMemcpyDeviceToHost, s));
    KM2_CUDA(cudaStreamSynchronize(s));
    if (J_out) *J_out = out.J;
    if (shift_out) *shift_out = out.shift;
    if (empty_out) *empty_out = out.empty;
    if (r.opt.profile) r.opt.profile->kernel_launches += g_launches - launches0;
    return KMEANS2_OK;
}

int kmeans_step_noalloc(const float* X, int64_t n, int32_t d, int32_t k,
                        const double* centers_in, double* centers_out, int32_t* labels_out,
                        double* J_out, double* shift_out, int32_t* empty_out, void* stream)
{
    if (!X || !centers_in || !centers_out || !labels_out || !valid_shape(n, d, k))
        return KMEANS2_ERR_INVALID;
    if (n > kNoAllocMaxN || k > kNoAllocMaxK || d > kNoAllocMaxD) {
        char msg[200];
        std::snprintf(msg, sizeof(msg),
                      "kmeans_step_noalloc: n=%lld, k=%d, d=%d exceed the fixed scratch limits "
                      "n <= %lld, k <= %d, d <= %d", (long long)n, k, d, kNoAllocMaxN,
                      kNoAllocMaxK, kNoAllocMaxD);
        set_last_error_text(msg);
        return KMEANS2_ERR_INVALID;
    }
    if (!is_device_ptr(X) || !is_device_ptr(centers_in) || !is_device_ptr(centers_out) ||
        !is_device_ptr(labels_out) || (reinterpret_cast<uintptr_t>(X) & 15) != 0 ||
        (reinterpret_cast<uintptr_t>(labels_out) & 3) != 0) {
        set_last_error_text("kmeans_step_noalloc: X, centers and labels must be device memory "
                            "(X 16-byte aligned)");
        return KMEANS2_ERR_INVALID;
    }
    void* arena = nullptr;
    KM2_TRY(noalloc_scratch(&arena));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceScratch ws(s, arena, kNoAllocBytes);
    // The CUDA-core form: its scratch (the near-tie list, n ints, plus O(k d)
    // center copies and sums) fits the array over the whole stated range; the
    // tensor-core forms would also need a per-call copy of X (about 4 n d
    // bytes for BF16), which it cannot hold.  Every form returns the same
    // labels, centers and J.
    Workspace w;
    w.form = KMEANS2_PRECISION_FP32;
    KM2_TRY(alloc_workspace(w, ws, n, k, d, 1, s));
    KM2_CUDA(cudaMemcpyAsync(w.c.c64, centers_in, sizeof(double) * (size_t)k * d,
                             cudaMemcpyDeviceToDevice, s));
    KM2_CUDA(cudaMemsetAsync(w.st, 0, sizeof(StageState), s));
    KM2_TRY(launch_maxabs(X, n, d, w.st, s, ws.sm_count));
    StageState out;
    KM2_TRY(run_stage(X, n, d, w, labels_out, 0.0, 1, false, s, ws.sm_count, out, nullptr,
                      nullptr, nullptr));
    KM2_CUDA(cudaMemcpyAsync(centers_out, w.c.c64, sizeof(double) * (size_t)k * d,
                             cudaMemcpyDeviceToDevice, s));
    KM2_CUDA(cudaStreamSynchronize(s));
    if (J_out) *J_out = out.J;
    if (shift_out) *shift_out = out.shift;
    if (empty_out) *empty_out = out.empty;
    return KMEANS2_OK;
}

}  // extern "C"

namespace {

// Share of a fast stage's rows (per iteration) that the single-pass FP16 form
// may leave undecided for AUTO to keep it in the slow stage: its pass costs
// ~0.85 of the split form's, and its second pass re-runs the undecided rows
// through the split kernel.
constexpr double kFp16MaxUndecided = 0.05;

// The two-stage fit on Xd, n*d FP32 points the device can read (its own
// memory or page-locked host memory), 16-byte aligned; arguments checked.
int fit_on(const float* Xd, int64_t n, int32_t d, int32_t k, double subset_fraction,
           uint64_t seed, double tol, int32_t max_iter, double* centers_out, int32_t* labels_out,
           kmeans2_result* res, const Resolved& r, DeviceScratch& ws,
           std::chrono::steady_clock::time_point t0, long long launches0)
{
    NvtxRange fit_range("kmeans2 fit");
    const kmeans2_options& o = r.opt;
    const double tol_fast = (o.tol_fast > 0.0) ? o.tol_fast : tol;
    const bool use_graph = o.use_graph != 0;
    cudaStream_t s = r.stream;
    const long long m = kmeans2_subset_size(n, k, subset_fraction);
    Workspace w;
    KM2_TRY(choose_form(o.precision, d, k, Xd, &w.form));
    // AUTO on a 16-bit tensor-core shape: the fast stage runs the single-pass
    // FP16 form and the slow stage keeps it only if that left few rows
    // undecided there (on tie-heavy data its second pass and the FP64 recheck
    // would cost more than the split form saves; measured)
    const bool adaptive = o.precision == KMEANS2_PRECISION_AUTO &&
                          w.form == KMEANS2_PRECISION_BF16 && o.start_stage == 0;
    if (adaptive) w.form = KMEANS2_PRECISION_FP16;
    KM2_TRY(alloc_workspace(w, ws, n, k, d, max_iter, s));
    if (o.traj_centers_fast || o.traj_centers_slow)
        KM2_TRY(ws.alloc((void**)&w.traj_c, sizeof(double) * (size_t)max_iter * k * d, s));
    if (o.traj_counts_fast || o.traj_counts_slow)
        KM2_TRY(ws.alloc((void**)&w.traj_n, sizeof(long long) * (size_t)max_iter * k, s));
    bool lab_dev = is_device_ptr(labels_out) && (reinterpret_cast<uintptr_t>(labels_out) & 3) == 0;
    int* labels = lab_dev ? labels_out : nullptr;
    if (!labels) KM2_TRY(ws.alloc((void**)&labels, sizeof(int) * (size_t)n, s));

    kmeans2_result rr;
    std::memset(&rr, 0, sizeof(rr));
    rr.precision_used = w.form;
    rr.subset_size = m;
    StageState fs;
    std::memset(&fs, 0, sizeof(fs));

    if (o.init_centers) {
        KM2_CUDA(cudaMemcpyAsync(w.c.c64, o.init_centers, sizeof(double) * (size_t)k * d,
                                 is_device_ptr(o.init_centers) ? cudaMemcpyDeviceToDevice
                                                               : cudaMemcpyHostToDevice, s));
    }
    if (o.start_stage == 0) {
        // fast stage on S_s (Algorithm: a per% subset, initial centers drawn from it)
        long long* subset = nullptr;
        long long* pos = nullptr;
        float* Xs = nullptr;
        int* labels_s = nullptr;
        KM2_TRY(ws.alloc((void**)&subset, sizeof(long long) * (size_t)m, s));
        KM2_TRY(ws.alloc((void**)&pos, sizeof(long long) * (size_t)k, s));
        KM2_TRY(ws.alloc((void**)&Xs, sizeof(float) * (size_t)m * d, s));
        KM2_TRY(ws.alloc((void**)&labels_s, sizeof(int) * (size_t)m, s));
        KM2_TRY(sample_device(n, k, m, seed, subset, pos, s, ws));
        KM2_CUDA(cudaMemsetAsync(w.st, 0, sizeof(StageState), s));
        KM2_TRY(launch_gather(Xd, d, subset, m, Xs, w.st, s, ws.sm_count));
        if (!o.init_centers) KM2_TRY(launch_init_centers(Xs, d, pos, k, w.c.c64, s));
        KM2_TRY(run_stage(Xs, m, d, w, labels_s, tol_fast, max_iter, use_graph, s, ws.sm_count,
                          fs, o.traj_J_fast, o.traj_shift_fast, o.profile, "kmeans2 fast stage",
                          o.traj_centers_fast, o.traj_counts_fast, adaptive));
        rr.iters_fast = fs.iter;
        rr.converged_fast = fs.converged;
        rr.shift_fast = fs.shift;
        rr.rechecked_points += fs.rechecked_total;
        rr.undecided_fast = fs.undecided16_total;
        if (adaptive && w.form == KMEANS2_PRECISION_FP16) {
            const double undecided = fs.iter > 0 && m > 0
                                         ? (double)fs.undecided16_total / ((double)fs.iter * (double)m)
                                         : 1.0;
            if (undecided > kFp16MaxUndecided) w.form = KMEANS2_PRECISION_BF16;
        }
    }
    // slow stage on S_n from the fast stage's final centers (Section 2; Section 5)
    KM2_CUDA(cudaMemsetAsync(w.st, 0, sizeof(StageState), s));
    KM2_TRY(launch_maxabs(Xd, n, d, w.st, s, ws.sm_count));
    StageState ss;
    KM2_TRY(run_stage(Xd, n, d, w, labels, tol, max_iter, use_graph, s, ws.sm_count, ss,
                      o.traj_J_slow, o.traj_shift_slow, o.profile, "kmeans2 slow stage",
                      o.traj_centers_slow, o.traj_counts_slow));
    rr.precision_used = w.form;
    rr.iters_slow = ss.iter;
    rr.converged_slow = ss.converged;
    rr.shift_slow = ss.shift;
    rr.J = ss.J;
    rr.empty_clusters = ss.empty;
    rr.rechecked_points += ss.rechecked_total;
    rr.undecided_slow = ss.undecided16_total;
    rr.distance_evals = (int64_t)rr.iters_fast * m * k + (int64_t)rr.iters_slow * n * k;

    KM2_CUDA(cudaMemcpyAsync(centers_out, w.c.c64, sizeof(double) * (size_t)k * d,
                             is_device_ptr(centers_out) ? cudaMemcpyDeviceToDevice
                                                        : cudaMemcpyDeviceToHost, s));
    if (!lab_dev)
        KM2_CUDA(cudaMemcpyAsync(labels_out, labels, sizeof(int) * (size_t)n,
                                 is_device_ptr(labels_out) ? cudaMemcpyDeviceToDevice
                                                           : cudaMemcpyDeviceToHost, s));
    KM2_CUDA(cudaStreamSynchronize(s));
    rr.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (res) *res = rr;
    if (o.profile) o.profile->kernel_launches += g_launches - launches0;
    return KMEANS2_OK;
}

}  // namespace

extern "C" {

int kmeans2_fit(const float* X, int64_t n, int32_t d, int32_t k, double subset_fraction,
                uint64_t seed, double tol, int32_t max_iter, double* centers_out,
                int32_t* labels_out, kmeans2_result* res, const kmeans2_options* opt)
{
    auto t0 = std::chrono::steady_clock::now();
    const long long launches0 = g_launches;
    if (!X || !centers_out || !labels_out || !valid_shape(n, d, k) ||
        !(subset_fraction > 0.0 && subset_fraction <= 1.0) || !(tol >= 0.0) || max_iter < 1)
        return KMEANS2_ERR_INVALID;
    Resolved r = resolve_options(opt);
    if (r.opt.start_stage != 0 && r.opt.start_stage != 1) return KMEANS2_ERR_INVALID;
    if (r.opt.start_stage == 1 && !r.opt.init_centers) return KMEANS2_ERR_INVALID;
    DeviceScratch ws(r.stream);
    const float* Xd = nullptr;
    KM2_TRY(device_view(X, (long long)n * d, &Xd, ws, r.stream));
    return fit_on(Xd, n, d, k, subset_fraction, seed, tol, max_iter, centers_out, labels_out, res,
                  r, ws, t0, launches0);
}

}  // extern "C"

namespace {

constexpr long long kDefaultChunkPoints = 1ll << 26;

// Host-resident X streamed through two device chunk buffers: copies run on a
// stream of their own and overlap the kernels of the previous chunk.
struct ChunkStreamer {
    const float* X = nullptr;
    long long n = 0, chunk = 0, nchunks = 0;
    int d = 0;
    float* buf[2] = {nullptr, nullptr};
    cudaStream_t copy = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr}, used[2] = {nullptr, nullptr};

    long long rows(long long c) const { return c + 1 < nchunks ? chunk : n - c * chunk; }

    int init(const float* X_, long long n_, int d_, long long chunk_, cudaStream_t s,
             DeviceScratch& ws)
    {
        X = X_;
        n = n_;
        d = d_;
        chunk = chunk_ < n_ ? chunk_ : n_;
        nchunks = (n + chunk - 1) / chunk;
        for (int b = 0; b < 2; ++b)
            KM2_TRY(ws.alloc((void**)&buf[b], (size_t)chunk * d * sizeof(float), s));
        KM2_CUDA(cudaStreamCreateWithFlags(&copy, cudaStreamNonBlocking));
        for (int b = 0; b < 2; ++b) {
            KM2_CUDA(cudaEventCreateWithFlags(&copied[b], cudaEventDisableTiming));
            KM2_CUDA(cudaEventCreateWithFlags(&used[b], cudaEventDisableTiming));
            KM2_CUDA(cudaEventRecord(used[b], s));      // both buffers start free
        }
        return KMEANS2_OK;
    }
    // Copy chunk c into buffer c % 2 once the kernels that read it last are done.
    int fetch(long long c)
    {
        const int b = (int)(c & 1);
        KM2_CUDA(cudaStreamWaitEvent(copy, used[b], 0));
        KM2_CUDA(cudaMemcpyAsync(buf[b], X + (size_t)(c * chunk) * d, (size_t)rows(c) * d * sizeof(float),
                                 cudaMemcpyHostToDevice, copy));
        KM2_CUDA(cudaEventRecord(copied[b], copy));
        return KMEANS2_OK;
    }
    ~ChunkStreamer()
    {
        if (copy) cudaStreamSynchronize(copy);
        for (int b = 0; b < 2; ++b) {
            if (copied[b]) cudaEventDestroy(copied[b]);
            if (used[b]) cudaEventDestroy(used[b]);
        }
        if (copy) cudaStreamDestroy(copy);
    }
};

// One pass over all chunks: before(c) gets each chunk once it is resident in
// buffer c % 2 (on stream s), then the buffer is released for the next copy.
template <class Fn>
int stream_pass(ChunkStreamer& cs, cudaStream_t s, Fn&& on_chunk)
{
    KM2_TRY(cs.fetch(0));
    for (long long c = 0; c < cs.nchunks; ++c) {
        if (c + 1 < cs.nchunks) KM2_TRY(cs.fetch(c + 1));
        const int b = (int)(c & 1);
        KM2_CUDA(cudaStreamWaitEvent(s, cs.copied[b], 0));
        KM2_TRY(on_chunk(c, cs.buf[b], cs.rows(c)));
        KM2_CUDA(cudaEventRecord(cs.used[b], s));
    }
    return KMEANS2_OK;
}

}  // namespace

extern "C" {

int kmeans2_fit_streamed(const float* X, int64_t n, int32_t d, int32_t k, double subset_fraction,
                         uint64_t seed, double tol, int32_t max_iter, int64_t chunk_points,
                         double* centers_out, int32_t* labels_out, kmeans2_result* res,
                         const kmeans2_options* opt)
{
    auto t0 = std::chrono::steady_clock::now();
    const long long launches0 = g_launches;
    if (!X || !centers_out || !labels_out || !valid_shape(n, d, k) ||
        !(subset_fraction > 0.0 && subset_fraction <= 1.0) || !(tol >= 0.0) || max_iter < 1)
        return KMEANS2_ERR_INVALID;
    if (is_device_ptr(X)) {
        set_last_error_text("kmeans2_fit_streamed: X must be host memory (use kmeans2_fit)");
        return KMEANS2_ERR_INVALID;
    }
    Resolved r = resolve_options(opt);
    const kmeans2_options& o = r.opt;
    if (o.start_stage != 0 && o.start_stage != 1) return KMEANS2_ERR_INVALID;
    if (o.start_stage == 1 && !o.init_centers) return KMEANS2_ERR_INVALID;
    if (o.precision != KMEANS2_PRECISION_FP32 && o.precision != KMEANS2_PRECISION_AUTO) {
        set_last_error_text("kmeans2_fit_streamed runs the CUDA-core FP32 form only");
        return KMEANS2_ERR_UNSUPPORTED;
    }
    if (chunk_points < 0) {
        // page-locked X: the kernels read it where it is, over the CPU-GPU
        // link, with no staging copies
        cudaPointerAttributes pa;
        const void* dp = nullptr;
        if (cudaPointerGetAttributes(&pa, X) == cudaSuccess && pa.type == cudaMemoryTypeHost)
            dp = pa.devicePointer;
        cudaGetLastError();
        if (dp && (reinterpret_cast<uintptr_t>(dp) & 15) == 0) {
            Resolved rd = r;
            rd.opt.precision = KMEANS2_PRECISION_FP32;
            DeviceScratch ws(rd.stream);
            return fit_on(static_cast<const float*>(dp), n, d, k, subset_fraction, seed, tol,
                          max_iter, centers_out, labels_out, res, rd, ws, t0, launches0);
        }
        chunk_points = 0;                     // pageable memory: staged chunks
    }
    if (chunk_points == 0) chunk_points = kDefaultChunkPoints;
    const double tol_fast = (o.tol_fast > 0.0) ? o.tol_fast : tol;
    cudaStream_t s = r.stream;
    DeviceScratch ws(s);
    const long long m = kmeans2_subset_size(n, k, subset_fraction);
    const long long chunk = chunk_points < n ? chunk_points : n;

    Workspace w;
    w.form = KMEANS2_PRECISION_FP32;
    KM2_TRY(alloc_workspace(w, ws, std::max(m, chunk), k, d, max_iter, s));
    bool lab_dev = is_device_ptr(labels_out) && (reinterpret_cast<uintptr_t>(labels_out) & 3) == 0;
    int* labels = lab_dev ? labels_out : nullptr;
    if (!labels) KM2_TRY(ws.alloc((void**)&labels, sizeof(int) * (size_t)n, s));

    kmeans2_result rr;
    std::memset(&rr, 0, sizeof(rr));
    rr.precision_used = KMEANS2_PRECISION_FP32;
    rr.subset_size = m;
    if (o.init_centers)
        KM2_CUDA(cudaMemcpyAsync(w.c.c64, o.init_centers, sizeof(double) * (size_t)k * d,
                                 is_device_ptr(o.init_centers) ? cudaMemcpyDeviceToDevice
                                                               : cudaMemcpyHostToDevice, s));
    if (o.start_stage == 0) {
        // fast stage: S_s gathered on the host, copied once, run resident
        long long* subset = nullptr;
        long long* pos = nullptr;
        float* Xs = nullptr;
        int* labels_s = nullptr;
        KM2_TRY(ws.alloc((void**)&subset, sizeof(long long) * (size_t)m, s));
        KM2_TRY(ws.alloc((void**)&pos, sizeof(long long) * (size_t)k, s));
        KM2_TRY(ws.alloc((void**)&Xs, sizeof(float) * (size_t)m * d, s));
        KM2_TRY(ws.alloc((void**)&labels_s, sizeof(int) * (size_t)m, s));
        KM2_TRY(sample_device(n, k, m, seed, subset, pos, s, ws));
        std::vector<long long> idx((size_t)m);
        KM2_CUDA(cudaMemcpyAsync(idx.data(), subset, sizeof(long long) * (size_t)m,
                                 cudaMemcpyDeviceToHost, s));
        KM2_CUDA(cudaStreamSynchronize(s));
        float* hs = nullptr;
        KM2_CUDA(cudaMallocHost((void**)&hs, sizeof(float) * (size_t)m * d));
        for (long long i = 0; i < m; ++i)
            std::memcpy(hs + (size_t)i * d, X + (size_t)idx[(size_t)i] * d, sizeof(float) * (size_t)d);
        cudaError_t e = cudaMemcpyAsync(Xs, hs, sizeof(float) * (size_t)m * d, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFreeHost(hs);
        if (e != cudaSuccess) { set_last_error("kmeans2_fit_streamed: S_s copy", e); return KMEANS2_ERR_CUDA; }
        KM2_CUDA(cudaMemsetAsync(w.st, 0, sizeof(StageState), s));
        KM2_TRY(launch_maxabs(Xs, m, d, w.st, s, ws.sm_count));
        if (!o.init_centers) KM2_TRY(launch_init_centers(Xs, d, pos, k, w.c.c64, s));
        StageState fs;
        KM2_TRY(run_stage(Xs, m, d, w, labels_s, tol_fast, max_iter, o.use_graph != 0, s, ws.sm_count,
                          fs, o.traj_J_fast, o.traj_shift_fast, nullptr));
        rr.iters_fast = fs.iter;
        rr.converged_fast = fs.converged;
        rr.shift_fast = fs.shift;
        rr.rechecked_points += fs.rechecked_total;
    }

    // slow stage on S_n from the fast stage's final centers, X streamed per pass
    ChunkStreamer cs;
    KM2_TRY(cs.init(X, n, d, chunk, s, ws));
    const size_t kd = (size_t)k * d;
    KM2_CUDA(cudaMemsetAsync(w.st, 0, sizeof(StageState), s));
    KM2_TRY(stream_pass(cs, s, [&](long long, const float* Xc, long long rows) {
        return launch_maxabs(Xc, rows, d, w.st, s, ws.sm_count);
    }));
    KM2_CUDA(cudaMemsetAsync(w.acc.s_lo, 0, kd * 8, s));
    KM2_CUDA(cudaMemsetAsync(w.acc.s_hi, 0, kd * 8, s));
    KM2_CUDA(cudaMemsetAsync(w.acc.cnt, 0, (size_t)k * 8, s));
    KM2_TRY(launch_center_prep(w.c, w.st, s));
    KM2_TRY(launch_stage_init(w.st, d, tol, max_iter, s));
    StageState ss;
    std::memset(&ss, 0, sizeof(ss));
    for (int it = 0; it < max_iter; ++it) {
        NvtxRange iteration_range("kmeans2 streamed iteration");
        KM2_TRY(stream_pass(cs, s, [&](long long c, const float* Xc, long long rows) {
            int* lab = labels + c * chunk;
            if (it == 0) KM2_TRY(launch_qsum(Xc, rows, d, w.st, s, ws.sm_count));
            KM2_TRY(launch_assign(Xc, rows, d, w, lab, s, ws.sm_count));
            KM2_TRY(launch_recheck(Xc, d, w.c, lab, w.list, w.st, w.acc, s, ws.sm_count));
            return launch_recheck_reset(w.st, s);
        }));
        KM2_TRY(launch_finalize(w.acc, w.c, w.st, w.traj(), w.clus, 0ull, 0, s));
        KM2_CUDA(cudaMemcpyAsync(&ss, w.st, sizeof(StageState), cudaMemcpyDeviceToHost, s));
        KM2_CUDA(cudaStreamSynchronize(s));
        if (ss.error) return map_stage_error(ss.error);
        if (ss.done) break;
    }
    if (o.traj_J_slow && ss.iter > 0)
        KM2_CUDA(cudaMemcpyAsync(o.traj_J_slow, w.traj_J, sizeof(double) * ss.iter,
                                 cudaMemcpyDeviceToHost, s));
    if (o.traj_shift_slow && ss.iter > 0)
        KM2_CUDA(cudaMemcpyAsync(o.traj_shift_slow, w.traj_shift, sizeof(double) * ss.iter,
                                 cudaMemcpyDeviceToHost, s));
    rr.iters_slow = ss.iter;
    rr.converged_slow = ss.converged;
    rr.shift_slow = ss.shift;
    rr.J = ss.J;
    rr.empty_clusters = ss.empty;
    rr.rechecked_points += ss.rechecked_total;
    rr.distance_evals = (int64_t)rr.iters_fast * m * k + (int64_t)rr.iters_slow * n * k;
    KM2_CUDA(cudaMemcpyAsync(centers_out, w.c.c64, sizeof(double) * kd,
                             is_device_ptr(centers_out) ? cudaMemcpyDeviceToDevice
                                                        : cudaMemcpyDeviceToHost, s));
    if (!lab_dev)
        KM2_CUDA(cudaMemcpyAsync(labels_out, labels, sizeof(int) * (size_t)n,
                                 is_device_ptr(labels_out) ? cudaMemcpyDeviceToDevice
                                                           : cudaMemcpyDeviceToHost, s));
    KM2_CUDA(cudaStreamSynchronize(s));
    rr.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (res) *res = rr;
    if (o.profile) o.profile->kernel_launches += g_launches - launches0;
    return KMEANS2_OK;
}

}  // extern "C"
