// server.cu -- the serving form: a request loop of independent two-stage fits
// with continuous batching.
//
// The server owns W worker threads, each bound to the server's device and to
// one non-blocking stream of its own.  Jobs wait in arrival order.  A free
// worker admits, under the FIFO policy, the first waiting job whose device
// footprint fits into the HBM budget next to the jobs already running (a job
// passed over kMaxBypass times blocks everything behind it, so large jobs are
// not starved), or under the SHORTEST policy the fitting job with the least
// work per iteration (n k d) unless some job has waited longer than the aging
// limit; it runs kmeans2_fit on it, the job's data, labels and centers
// resident from admission to result.  Stage loops run as graphs with
// device-side while conditions or, the default with several slots, from the
// worker thread: on GB300 one job's while-graph holds back another job's
// while-graph until it ends (a short job arriving beside a long one waited
// for all of it), while host-driven loops interleave (measured on the serving
// trace: p50 0.14 s instead of 0.34-0.44 s).
// Different jobs' kernels therefore overlap on the GPU, and a job that arrives
// while others run starts as soon as a worker and memory are free -- no batch
// boundary to wait for.  Every job runs exactly the kernels of a lone
// kmeans2_fit call (exact fixed-point cluster sums, so sharing the GPU changes
// no bit of the result).
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "api_internal.h"

namespace km2 {
namespace {

constexpr int kMaxSlots = 64;
constexpr int kMaxBypass = 8;

enum class JobState { Queued, Running, Done };

struct Ticket {
    kmeans2_job job{};
    kmeans2_materialize_fn materialize = nullptr;   // lazy input (NULL: job.X given)
    kmeans2_consume_fn consume = nullptr;
    void* user = nullptr;
    uint64_t footprint = 0;
    double work = 0.0;          // n k d: the cost of one iteration
    JobState state = JobState::Queued;
    int status = KMEANS2_PENDING;
    int bypassed = 0;
    kmeans2_result res{};
    kmeans2_ticket_times times{};
};

bool on_device(const void* p, uintptr_t align)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) &&
           (reinterpret_cast<uintptr_t>(p) & (align - 1)) == 0;
}

}  // namespace
}  // namespace km2

struct kmeans2_server {
    int device = 0;
    uint64_t budget = 0;
    int slots = 0;
    kmeans2_options opt{};
    std::chrono::steady_clock::time_point t0;

    std::mutex mu;
    std::condition_variable cv_work;   // workers: a job arrived, memory was freed, or stop
    std::condition_variable cv_done;   // waiters: a job finished
    std::deque<uint64_t> queue;        // waiting tickets, arrival order
    std::deque<uint64_t> finished;     // finished tickets not yet handed out by wait_any
    std::unordered_map<uint64_t, km2::Ticket> tickets;
    uint64_t next_ticket = 1;
    uint64_t in_use = 0, peak = 0;
    int running = 0;
    int64_t submitted = 0, admitted = 0, completed = 0, failed = 0, rejected = 0, launches = 0;
    bool stop = false;
    int policy = KMEANS2_POLICY_FIFO;
    double aging_s = 0.0;

    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }

    // Under mu: the ticket a free worker should start, or 0.
    uint64_t pick()
    {
        if (policy == KMEANS2_POLICY_SHORTEST) return pick_shortest();
        for (size_t i = 0; i < queue.size(); ++i) {
            km2::Ticket& t = tickets[queue[i]];
            if (in_use + t.footprint <= budget) {
                const uint64_t id = queue[i];
                for (size_t j = 0; j < i; ++j) tickets[queue[j]].bypassed += 1;
                queue.erase(queue.begin() + (long)i);
                return id;
            }
            if (t.bypassed >= km2::kMaxBypass) break;   // nothing may pass it any more
        }
        return 0;
    }

    // Under mu: a job that has waited aging_s or longer goes first (oldest
    // first; while it does not fit nothing else is admitted); otherwise the
    // waiting job with the least work per iteration that fits.
    uint64_t pick_shortest()
    {
        if (queue.empty()) return 0;
        const double t = now();
        const uint64_t head = queue.front();
        km2::Ticket& h = tickets[head];
        if (t - h.times.t_submit >= aging_s) {
            if (in_use + h.footprint > budget) return 0;
            queue.pop_front();
            return head;
        }
        size_t best = queue.size();
        for (size_t i = 0; i < queue.size(); ++i) {
            const km2::Ticket& c = tickets[queue[i]];
            if (in_use + c.footprint > budget) continue;
            if (best == queue.size() || c.work < tickets[queue[best]].work) best = i;
        }
        if (best == queue.size()) return 0;
        const uint64_t id = queue[best];
        queue.erase(queue.begin() + (long)best);
        return id;
    }

    void work(int slot)
    {
        cudaSetDevice(device);
        for (;;) {
            uint64_t id = 0;
            kmeans2_job job{};
            kmeans2_materialize_fn materialize = nullptr;
            kmeans2_consume_fn consume = nullptr;
            void* user = nullptr;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] {
                    if (stop) return true;
                    id = pick();
                    return id != 0;
                });
                if (stop) {
                    if (id) {   // picked in the same wake-up as the stop: give it back as cancelled
                        km2::Ticket& t = tickets[id];
                        t.state = km2::JobState::Done;
                        t.status = KMEANS2_ERR_ADMISSION;
                        t.times.t_done = now();
                        ++failed;
                        finished.push_back(id);
                        cv_done.notify_all();
                    }
                    return;
                }
                km2::Ticket& t = tickets[id];
                t.state = km2::JobState::Running;
                t.times.t_admit = now();
                in_use += t.footprint;
                if (in_use > peak) peak = in_use;
                ++running;
                ++admitted;
                job = t.job;
                materialize = t.materialize;
                consume = t.consume;
                user = t.user;
            }
            kmeans2_options o = opt;
            o.stream = streams[slot];
            kmeans2_result r;
            std::memset(&r, 0, sizeof(r));
            const long long l0 = km2::g_launches;
            int rc = KMEANS2_OK;
            if (materialize)
                rc = run_lazy(job, materialize, consume, user, o, &r);
            else
                rc = kmeans2_fit(job.X, job.n, job.d, job.k, job.subset_fraction, job.seed,
                                 job.tol, job.max_iter, job.centers_out, job.labels_out, &r, &o);
            const long long dl = km2::g_launches - l0;
            {
                std::lock_guard<std::mutex> lk(mu);
                km2::Ticket& t = tickets[id];
                t.state = km2::JobState::Done;
                t.status = rc;
                t.res = r;
                t.times.t_done = now();
                in_use -= t.footprint;
                --running;
                if (rc == KMEANS2_OK) ++completed; else ++failed;
                launches += dl;
                finished.push_back(id);
            }
            cv_work.notify_all();
            cv_done.notify_all();
        }
    }

    // A lazy job: device buffers for X, centers and labels on the worker's
    // stream, the caller's materialize, the fit, the caller's consume.
    int run_lazy(const kmeans2_job& job, kmeans2_materialize_fn materialize,
                 kmeans2_consume_fn consume, void* user, const kmeans2_options& o,
                 kmeans2_result* r)
    {
        cudaStream_t s = static_cast<cudaStream_t>(o.stream);
        float* X = nullptr;
        double* cen = nullptr;
        int* lab = nullptr;
        int rc = KMEANS2_OK;
        const size_t xb = (size_t)job.n * (size_t)job.d * 4;
        if (km2::pool_malloc_async((void**)&X, xb, s) != cudaSuccess ||
            km2::pool_malloc_async((void**)&cen, (size_t)job.k * job.d * 8, s) != cudaSuccess ||
            km2::pool_malloc_async((void**)&lab, (size_t)job.n * 4, s) != cudaSuccess) {
            cudaGetLastError();
            km2::set_last_error_text("server: no device memory for a lazy job");
            rc = KMEANS2_ERR_NOMEM;
        }
        if (rc == KMEANS2_OK && materialize(user, X, o.stream) != 0) {
            km2::set_last_error_text("server: the job's materialize callback failed");
            rc = KMEANS2_ERR_INVALID;
        }
        if (rc == KMEANS2_OK)
            rc = kmeans2_fit(X, job.n, job.d, job.k, job.subset_fraction, job.seed, job.tol,
                             job.max_iter, cen, lab, r, &o);
        if (rc == KMEANS2_OK && consume) consume(user, cen, lab, o.stream);
        if (lab) cudaFreeAsync(lab, s);
        if (cen) cudaFreeAsync(cen, s);
        if (X) cudaFreeAsync(X, s);
        cudaStreamSynchronize(s);
        return rc;
    }

    // Under mu: the status of a finished ticket (and release it), or PENDING.
    int take(uint64_t id, kmeans2_result* res, kmeans2_ticket_times* times)
    {
        auto it = tickets.find(id);
        if (it == tickets.end()) return KMEANS2_ERR_INVALID;
        if (it->second.state != km2::JobState::Done) return KMEANS2_PENDING;
        const int st = it->second.status;
        if (res) *res = it->second.res;
        if (times) *times = it->second.times;
        tickets.erase(it);
        return st;
    }
};

extern "C" {

kmeans2_server* kmeans2_server_create(uint64_t hbm_budget, int32_t max_slots,
                                      const kmeans2_options* opt)
{
    if (max_slots < 1 || max_slots > km2::kMaxSlots) return nullptr;
    kmeans2_options o;
    kmeans2_default_options(&o);
    if (opt) o = *opt;
    // with several slots and no options, host-driven stage loops: another
    // job's while-graph would not start while one runs (measured)
    if (!opt && max_slots > 1) o.use_graph = 0;
    if (o.stream || o.init_centers || o.start_stage != 0 || o.profile || o.traj_J_fast ||
        o.traj_shift_fast || o.traj_J_slow || o.traj_shift_slow)
        return nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    if (hbm_budget == 0) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return nullptr;
        hbm_budget = (uint64_t)((double)free_b * 0.9);
    }
    auto* s = new kmeans2_server();
    s->device = dev;
    s->budget = hbm_budget;
    s->slots = max_slots;
    s->opt = o;
    s->t0 = std::chrono::steady_clock::now();
    for (int i = 0; i < max_slots; ++i) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            delete s;
            return nullptr;
        }
        s->streams.push_back(st);
    }
    for (int i = 0; i < max_slots; ++i) s->workers.emplace_back([s, i] { s->work(i); });
    return s;
}

namespace {

int submit_common(kmeans2_server* srv, const kmeans2_job* job, kmeans2_materialize_fn materialize,
                  kmeans2_consume_fn consume, void* user, uint64_t* ticket)
{
    if (!srv || !job || !ticket) return KMEANS2_ERR_INVALID;
    const kmeans2_job& J = *job;
    const bool lazy = materialize != nullptr;
    if ((!lazy && (!J.X || !J.centers_out || !J.labels_out)) || J.reserved != 0 || J.n < 1 ||
        J.d < 1 || J.k < 1 || J.k > J.n || !(J.subset_fraction > 0.0 && J.subset_fraction <= 1.0) ||
        !(J.tol >= 0.0) || J.max_iter < 1) {
        km2::set_last_error_text("kmeans2_server_submit: job out of range");
        return KMEANS2_ERR_INVALID;
    }
    const bool x_dev = lazy || km2::on_device(J.X, 16);
    const bool lab_dev = lazy || km2::on_device(J.labels_out, 4);
    uint64_t fp = kmeans2_fit_footprint(J.n, J.d, J.k, J.subset_fraction, J.max_iter,
                                        srv->opt.precision, x_dev ? 0 : 1, lab_dev ? 0 : 1);
    if (fp == 0) {
        km2::set_last_error_text("kmeans2_server_submit: shape or precision not supported");
        return KMEANS2_ERR_INVALID;
    }
    if (x_dev) fp += (uint64_t)J.n * (uint64_t)J.d * 4;   // resident data counts against the budget
    if (lazy) fp += (uint64_t)J.k * (uint64_t)J.d * 8 + (uint64_t)J.n * 4;   // server-owned outputs
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stop) return KMEANS2_ERR_ADMISSION;
    if (fp > srv->budget) {
        ++srv->rejected;
        km2::set_last_error_text("kmeans2_server_submit: job footprint exceeds the HBM budget");
        return KMEANS2_ERR_ADMISSION;
    }
    const uint64_t id = srv->next_ticket++;
    km2::Ticket& t = srv->tickets[id];
    t.job = J;
    t.materialize = materialize;
    t.consume = consume;
    t.user = user;
    t.footprint = fp;
    t.work = (double)J.n * (double)J.k * (double)J.d;
    t.times.t_submit = srv->now();
    srv->queue.push_back(id);
    ++srv->submitted;
    *ticket = id;
    srv->cv_work.notify_all();
    return KMEANS2_OK;
}

}  // namespace

int kmeans2_server_submit(kmeans2_server* srv, const kmeans2_job* job, uint64_t* ticket)
{
    return submit_common(srv, job, nullptr, nullptr, nullptr, ticket);
}

int kmeans2_server_submit_lazy(kmeans2_server* srv, const kmeans2_job* job,
                               kmeans2_materialize_fn materialize, kmeans2_consume_fn consume,
                               void* user, uint64_t* ticket)
{
    if (!materialize) return KMEANS2_ERR_INVALID;
    return submit_common(srv, job, materialize, consume, user, ticket);
}

int kmeans2_server_poll(kmeans2_server* srv, uint64_t ticket, kmeans2_result* res,
                        kmeans2_ticket_times* times)
{
    if (!srv) return KMEANS2_ERR_INVALID;
    std::lock_guard<std::mutex> lk(srv->mu);
    return srv->take(ticket, res, times);
}

int kmeans2_server_wait(kmeans2_server* srv, uint64_t ticket, double timeout_s,
                        kmeans2_result* res, kmeans2_ticket_times* times)
{
    if (!srv) return KMEANS2_ERR_INVALID;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto ready = [&] {
        auto it = srv->tickets.find(ticket);
        return it == srv->tickets.end() || it->second.state == km2::JobState::Done;
    };
    if (timeout_s < 0)
        srv->cv_done.wait(lk, ready);
    else
        srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready);
    return srv->take(ticket, res, times);
}

int kmeans2_server_stats_get(kmeans2_server* srv, kmeans2_server_stats* out)
{
    if (!srv || !out) return KMEANS2_ERR_INVALID;
    std::lock_guard<std::mutex> lk(srv->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = srv->submitted;
    out->admitted = srv->admitted;
    out->completed = srv->completed;
    out->failed = srv->failed;
    out->rejected = srv->rejected;
    out->kernel_launches = srv->launches;
    out->queued = (int32_t)srv->queue.size();
    out->running = srv->running;
    out->slots = srv->slots;
    out->hbm_budget = srv->budget;
    out->hbm_in_use = srv->in_use;
    out->hbm_peak = srv->peak;
    return KMEANS2_OK;
}

double kmeans2_server_now(kmeans2_server* srv) { return srv ? srv->now() : 0.0; }

int kmeans2_server_wait_any(kmeans2_server* srv, double timeout_s, uint64_t* ticket)
{
    if (!srv || !ticket) return KMEANS2_ERR_INVALID;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto ready = [&] {
        // skip tickets already collected by poll / wait
        while (!srv->finished.empty() && srv->tickets.find(srv->finished.front()) == srv->tickets.end())
            srv->finished.pop_front();
        return !srv->finished.empty();
    };
    if (timeout_s < 0)
        srv->cv_done.wait(lk, ready);
    else
        srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready);
    if (!ready()) return KMEANS2_PENDING;
    *ticket = srv->finished.front();
    srv->finished.pop_front();
    return KMEANS2_OK;
}

int kmeans2_server_set_policy(kmeans2_server* srv, int32_t policy, double aging_s)
{
    if (!srv || (policy != KMEANS2_POLICY_FIFO && policy != KMEANS2_POLICY_SHORTEST) ||
        !(aging_s >= 0.0))
        return KMEANS2_ERR_INVALID;
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->policy = policy;
    srv->aging_s = aging_s;
    srv->cv_work.notify_all();
    return KMEANS2_OK;
}

void kmeans2_server_destroy(kmeans2_server* srv)
{
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        for (uint64_t id : srv->queue) {
            km2::Ticket& t = srv->tickets[id];
            t.state = km2::JobState::Done;
            t.status = KMEANS2_ERR_ADMISSION;
            t.times.t_done = srv->now();
            ++srv->failed;
        }
        srv->queue.clear();
    }
    srv->cv_work.notify_all();
    srv->cv_done.notify_all();
    for (std::thread& w : srv->workers) w.join();
    for (cudaStream_t s : srv->streams) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    delete srv;
}

}  // extern "C"
