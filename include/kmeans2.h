/*
 * kmeans2.h -- C ABI of libkmeans2, a GB300 (sm_103a) implementation of the
 * two-stage k-means of Salman et al., "Fast k-means algorithm clustering"
 * (arXiv 1108.1351).
 *
 * The method (Section 2, Algorithm): draw a random subset S_s (per% of the
 * data S_n) and k random initial centers from it; run Lloyd iterations on S_s
 * until the centers stop moving (fast stage); then run Lloyd iterations on the
 * whole S_n starting from those centers (slow stage).  One Lloyd iteration
 * (Section 4.1, Lloyd's method) is: squared distance of every point to every
 * center (Eq. 1 without the root, the Algorithm's "modified distance"),
 * nearest-center label, the objective J (Eq. 3), new centers = cluster means,
 * and the stop test on the largest center movement (Sections 5-6).
 *
 * Conventions shared by every entry point
 *  - X is row-major FP32, n rows of d values.  Centers are row-major FP64,
 *    k rows of d values.  Labels are int32 in [0, k).
 *  - Every pointer may be a device pointer (cudaMalloc, torch tensors) or a
 *    host pointer (pageable or pinned); the library checks each with
 *    cudaPointerGetAttributes and stages host buffers through device memory.
 *    Host staging copies are part of the call.  Device pointers must belong to
 *    the current device (the one the call runs on): the kernels address them
 *    directly, and another GPU's memory is not supported.
 *  - The caller owns every buffer it passes.  The library allocates only
 *    scratch (stream-ordered, from the device's default memory pool) and
 *    frees it before returning.
 *  - All calls are synchronous with respect to the host: outputs are ready
 *    when the call returns.  Work is issued on options->stream (NULL: the
 *    legacy default stream).  Calls on different streams may run concurrently;
 *    calls sharing output buffers must not.
 *  - Return value: KMEANS2_OK (0) or a negative status; kmeans2_strerror()
 *    names it.  On error no output is guaranteed to be written.  Reaching
 *    max_iter without convergence is NOT an error (see kmeans2_result).
 *  - Limits: 1 <= d <= 4096, 1 <= k <= n < 2^31, and k*d <= 2^24.
 *
 * Numerics (the results the library guarantees)
 *  - Labels: for given FP64 centers, the label of every point equals the
 *    index of the smallest FP64 squared distance sum_t fma(x_t - c_t, ...)
 *    evaluated left to right, the lowest index winning exact ties.  The fast
 *    FP32 distance kernels decide every point whose best and second-best
 *    distances are farther apart than a rigorous rounding-error bound; the
 *    other points are re-evaluated in exactly that FP64 form.
 *  - Cluster sums are exact integer (fixed-point) sums of the FP32 inputs at a
 *    per-stage scale 2^F, F = min(120, 46 - E) with E the smallest integer
 *    such that max|x| < 2^E (so a center is off the exact mean by at most
 *    2^-(F+1) per coordinate, plus the FP64 rounding of the division), which
 *    makes every mode deterministic: results do not depend on thread
 *    scheduling.  The cap keeps 2^F a finite FP32 scale: data with max|x| <
 *    2^-74 keep the absolute grid 2^-120 and so fewer than 46 bits.
 *  - J (Eq. 3) is formed on the same fixed-point values, without cancellation:
 *    J = W + M with W = (sum_i ||s_i||^2 - sum_j ||s_j||^2 / N_j) 2^-2F, where s
 *    are the integer coordinates and s_j their exact cluster sums (exact
 *    256-bit integer arithmetic, one final rounding), and M = sum_j N_j
 *    ||c_j - mu_j||^2 with each displacement from the exact mean mu_j formed in
 *    double-word arithmetic.  J therefore equals sum_i ||x_i - c_label(i)||^2
 *    to a few FP64 ulps relative; only coordinates with |x| < 2^(E-23), which
 *    lie off the 2^-F grid, can add more (at most 2^(2E-46) each).
 */
#ifndef KMEANS2_H
#define KMEANS2_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define KMEANS2_API __attribute__((visibility("default")))
#else
#define KMEANS2_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define KMEANS2_OK 0
#define KMEANS2_ERR_INVALID (-1)      /* an argument is out of range or NULL */
#define KMEANS2_ERR_NOMEM (-2)        /* device or pinned-host allocation failed */
#define KMEANS2_ERR_CUDA (-3)         /* a CUDA runtime call failed */
#define KMEANS2_ERR_NONFINITE (-4)    /* X holds a NaN or an infinity */
#define KMEANS2_ERR_TIMEOUT (-5)      /* a bounded device-side wait gave up */
#define KMEANS2_ERR_ADMISSION (-6)    /* a server refused a job (HBM budget) */
#define KMEANS2_ERR_UNSUPPORTED (-7)  /* shape or mode not supported */

/* ---------------------------------------------------------------- options */
/* Forms of the distance kernel.  Every form returns the same labels (near
   ties are re-decided in FP64); they differ in speed and in how many points
   need that recheck. */
#define KMEANS2_PRECISION_FP32 0      /* FP32 FMA chains on the CUDA cores (plain form) */
#define KMEANS2_PRECISION_BF16 1      /* cross term on the tensor cores in BF16 (operands
                                         split in two BF16 parts, three products, FP32
                                         accumulation); d a multiple of 16 in [16, 128] */
#define KMEANS2_PRECISION_AUTO 2      /* fastest form measured for the shape (default):
                                         for d in {64, 80, ..., 128} and k >= 512,
                                         kmeans2_fit starts the fast stage in FP16 and
                                         moves to BF16 if its first iteration leaves
                                         more than 10 % of the rows undecided; the slow
                                         stage runs FP16 if the fast stage left at most
                                         5 % per iteration, else BF16 (the other entry
                                         points take BF16 there); FP32 otherwise */
#define KMEANS2_PRECISION_TF32X3 3    /* cross term on the tensor cores as three TF32
                                         products of the exact hi/lo split of the FP32
                                         operands; d in {4, 8, 16, 32}, k <= 256 */
#define KMEANS2_PRECISION_FP16 4      /* cross term on the tensor cores in one FP16 pass
                                         (operands scaled by powers of two into the FP16
                                         range, one product, FP32 accumulation); rows
                                         inside its bound are re-run in the split-BF16
                                         form before the FP64 recheck; same shapes as BF16 */

/* Optional per-call measurement, filled by the library when options->profile
   is set.  A profiled call runs each stage loop from the host (no graph) and
   brackets every launch of the fused distance kernel with CUDA events on the
   call's stream. */
typedef struct kmeans2_profile {
    int64_t kernel_launches;    /* kernels of this library launched by the call */
    int64_t assign_launches;    /* launches of the fused distance kernel */
    double assign_ms;           /* their summed CUDA-event time */
    double assign_flops;        /* algorithmic 2*N*k*d summed over those launches */
    double assign_bytes;        /* algorithmic 4*N*d (one read of X) summed */
} kmeans2_profile;

typedef struct kmeans2_options {
    int32_t precision;          /* KMEANS2_PRECISION_*; default AUTO */
    int32_t deterministic;      /* accepted for interface stability; every mode is
                                   deterministic (exact integer cluster sums) */
    double tol_fast;            /* stop tolerance of the fast stage; <= 0: use tol.
                                   Section 5 uses 1e-3 fast / 1e-6 slow. */
    const double* init_centers; /* k*d FP64 starting centers (host or device), or
                                   NULL for the random draw of the Algorithm */
    int32_t start_stage;        /* with init_centers: 0 = run both stages from them,
                                   1 = skip the fast stage (resume a slow stage) */
    int32_t use_graph;          /* 1 (default when options are NULL): run each stage
                                   loop as one CUDA graph with a device-side while
                                   loop; 0: one host round trip per iteration.
                                   Fits meant to run side by side on several
                                   streams should use 0: on GB300 a second
                                   while-graph waits for a running one to end */
    void* stream;               /* cudaStream_t, NULL = legacy default stream */
    /* Optional HOST arrays of capacity max_iter receiving one value per
       iteration (Figs. 4-11 and Table 1 track exactly these trajectories). */
    double* traj_J_fast;
    double* traj_shift_fast;
    double* traj_J_slow;
    double* traj_shift_slow;
    kmeans2_profile* profile;   /* optional HOST struct, see kmeans2_profile */
    /* kmeans2_fit only: optional HOST arrays receiving, per iteration, the
       updated centers (capacity max_iter*k*d FP64, iteration-major) and the
       cluster sizes of that iteration's assignment (max_iter*k int64): the
       center movements of Figs. 4-9 and the point / center distribution of
       Table 1. */
    double* traj_centers_fast;
    double* traj_centers_slow;
    int64_t* traj_counts_fast;
    int64_t* traj_counts_slow;
} kmeans2_options;

/* Fill *opt with the defaults (AUTO form, tol_fast = tol, random init, graph loop). */
KMEANS2_API void kmeans2_default_options(kmeans2_options* opt);

typedef struct kmeans2_result {
    double J;                   /* objective of the returned labels against the
                                   centers they were assigned to (Eq. 3) */
    int32_t iters_fast;         /* Q_f: fast-stage iterations, the detecting one counted */
    int32_t iters_slow;         /* Q_s: slow-stage iterations */
    int32_t converged_fast;     /* 1 if the fast stage met its tolerance */
    int32_t converged_slow;     /* 1 if the slow stage met tol */
    int32_t empty_clusters;     /* clusters left without points in the last iteration */
    int32_t precision_used;     /* the form of the slow stage: KMEANS2_PRECISION_FP32,
                                   _BF16, _FP16 or _TF32X3 */
    int64_t subset_size;        /* m = |S_s| */
    int64_t rechecked_points;   /* points re-evaluated in FP64, summed over iterations */
    int64_t distance_evals;     /* K Q_f m + K Q_s n (Section 3 cost model) */
    double shift_fast;          /* last fast-stage max center movement */
    double shift_slow;          /* last slow-stage max center movement */
    double seconds;             /* wall time of the call */
    int64_t undecided_fast;     /* FP16 form: rows its single pass left undecided
                                   (second pass), summed over the fast stage's
                                   iterations; 0 for the other forms */
    int64_t undecided_slow;     /* the same over the slow stage */
} kmeans2_result;

/* ---------------------------------------------------------------- entry points */

/*
 * kmeans2_fit -- the whole two-stage method (Section 2, Algorithm).
 *
 *  X             n*d FP32 points S_n (host or device).
 *  subset_fraction  per, in (0, 1]; m = min(n, max(k, ceil(per*n))) points form S_s.
 *  seed          drives both random draws (see kmeans2_sample).
 *  tol           slow-stage stop tolerance on max_j ||c_j' - c_j||_2 (absolute);
 *                the fast stage uses options->tol_fast when > 0.
 *  max_iter      per-stage iteration cap (>= 1).
 *  centers_out   k*d FP64 (host or device): the slow stage's last updated centers.
 *  labels_out    n int32 (host or device): the last slow-stage assignment,
 *                made against the centers before that last update.
 *  res           host struct, may be NULL.
 *  opt           may be NULL (defaults).
 * Errors: KMEANS2_ERR_INVALID (n < 1, d < 1, k < 1, k > n, per outside (0, 1],
 * tol < 0 or NaN, max_iter < 1, NULL X/centers_out/labels_out, limits above),
 * KMEANS2_ERR_UNSUPPORTED (a precision form the shape cannot run),
 * KMEANS2_ERR_NONFINITE, KMEANS2_ERR_NOMEM, KMEANS2_ERR_CUDA,
 * KMEANS2_ERR_TIMEOUT (a bounded wait inside a tensor-core kernel gave up).
 */
KMEANS2_API int kmeans2_fit(const float* X, int64_t n, int32_t d, int32_t k, double subset_fraction,
                uint64_t seed, double tol, int32_t max_iter, double* centers_out,
                int32_t* labels_out, kmeans2_result* res, const kmeans2_options* opt);

/*
 * kmeans2_fit_streamed -- kmeans2_fit for data that stays in HOST memory (for
 * instance larger than the GPU's HBM; Abstract and Section 6: the method is
 * aimed at very large data sets).  Same method, arguments and results as
 * kmeans2_fit, and the same results bit for bit: S_s is gathered on the host
 * and copied to the device once (the fast stage runs resident); every
 * iteration of the slow stage streams X through the device in chunks of
 * chunk_points rows (two device buffers, copies on a second stream
 * overlapping the distance kernel of the previous chunk), with the near-tie
 * recheck of each chunk done while it is resident and the exact integer
 * cluster sums accumulated across chunks.  The device holds the labels (n
 * int32, unless labels_out is device memory), two chunks, S_s and the
 * workspace.  Pinned host memory (cudaHostRegister / cudaMallocHost) makes
 * the copies asynchronous; pageable memory works, synchronously.
 *
 *  X             n*d FP32 points in host memory.
 *  chunk_points  rows per chunk; 0 = 2^26 rows; < 0 = in place: if X is
 *                page-locked and 16-byte aligned the kernels read it where it
 *                is, over the CPU-GPU link (NVLink-C2C on GB300), with no
 *                staging copies and no chunk loop (same results; on GB300 the
 *                staged chunks measured faster), otherwise 2^26-row chunks.
 *  opt           precision must be FP32 or AUTO (the CUDA-core form);
 *                use_graph is ignored (the slow stage is host-driven).
 * Errors as kmeans2_fit; KMEANS2_ERR_INVALID if X is device memory,
 * KMEANS2_ERR_UNSUPPORTED for a tensor-core precision.
 */
KMEANS2_API int kmeans2_fit_streamed(const float* X, int64_t n, int32_t d, int32_t k,
                                     double subset_fraction, uint64_t seed, double tol,
                                     int32_t max_iter, int64_t chunk_points, double* centers_out,
                                     int32_t* labels_out, kmeans2_result* res,
                                     const kmeans2_options* opt);

/* ---------------------------------------------------------------- data-parallel shards
 *
 * The method split over the rows of S_n the way a group of GPUs runs it (one
 * rank per GPU): each rank keeps its rows, their labels, its exact integer
 * cluster sums and near-tie list, and a replicated copy of the centers.  Per
 * Lloyd iteration (Section 4.1) the ranks all-reduce the integer partials of
 * the centroid update -- sum_i x_i split into two int64 words, N_j and, in a
 * stage's first iteration, the exact sum of the squared fixed-point
 * coordinates (four int64 words) -- and every rank runs the same
 * finalize on the totals.  Integer sums do not depend on the order of the
 * reduction, so labels, centers, J and iteration counts equal those of
 * kmeans2_fit on the whole of X, bit for bit, for any number of ranks and any
 * split.  S_s needs no exchange (its keys depend only on global positions);
 * the initial centers and each stage's max |x| are one small all-reduce each.
 *
 * The caller owns the exchange: kmeans2_shard_advance runs the rank's kernels
 * up to the next exchange point and says what to all-reduce, in place, in the
 * caller's exchange buffer (NCCL or any collective library; every rank gets
 * the same descriptor at the same step).  Then it is called again.
 */
typedef struct kmeans2_shard kmeans2_shard;

#define KMEANS2_XCHG_SUM_I64 0   /* int64 sum (two's complement wrap-around) */
#define KMEANS2_XCHG_MAX_I64 1   /* int64 maximum */
#define KMEANS2_XCHG_SUM_F64 2   /* FP64 sum; exact in any order for this use */

typedef struct kmeans2_exchange {
    int32_t op;          /* KMEANS2_XCHG_* */
    int32_t reserved;
    int64_t count;       /* 8-byte elements of the exchange buffer to reduce, from element 0 */
} kmeans2_exchange;

/* 8-byte elements the exchange buffer must hold for (d, k): 2 k d + k + 7;
 * -1 for d < 1 or k < 1. */
KMEANS2_API int64_t kmeans2_shard_exchange_elems(int32_t d, int32_t k);

/*
 * kmeans2_shard_create -- one rank's session of a data-parallel fit.
 *
 *  X_local       n_local*d FP32 rows of S_n (host or device; copied to the
 *                device when host or misaligned), global rows
 *                [row0, row0 + n_local).  n_local may be 0 (X_local NULL).
 *  n_total       n of the whole data set; the ranks' row ranges must
 *                partition [0, n_total).
 *  subset_fraction, seed, tol, max_iter, opt   as kmeans2_fit, identical on
 *                every rank (opt->stream, trajectories and profile are per rank).
 *  exchange_buf  device memory, 8-byte aligned, kmeans2_shard_exchange_elems
 *                elements; owned by the caller, alive until destroy.
 *  out           receives the session; destroy it with kmeans2_shard_destroy.
 * Draws S_s (all n_total keys) and gathers this rank's part of it.
 * Errors: KMEANS2_ERR_INVALID (arguments as kmeans2_fit, row range outside
 * [0, n_total), exchange buffer not device memory), KMEANS2_ERR_NOMEM,
 * KMEANS2_ERR_UNSUPPORTED, KMEANS2_ERR_CUDA.
 */
KMEANS2_API int kmeans2_shard_create(const float* X_local, int64_t n_local, int64_t row0,
                                     int64_t n_total, int32_t d, int32_t k,
                                     double subset_fraction, uint64_t seed, double tol,
                                     int32_t max_iter, void* exchange_buf,
                                     const kmeans2_options* opt, kmeans2_shard** out);

/*
 * kmeans2_shard_advance -- run this rank to its next exchange point.
 * Returns KMEANS2_PENDING with *next set: the first next->count elements of
 * the exchange buffer are ready (the rank's stream is synchronised) and must
 * be all-reduced across ranks with next->op, in place, before the next call.
 * Returns KMEANS2_OK once the fit has finished (every rank at the same call),
 * or a negative status (the same on every rank for data errors such as
 * KMEANS2_ERR_NONFINITE; a device-side timeout on one rank reaches the others
 * through the next exchange).  After an error the session only reports it.
 */
KMEANS2_API int kmeans2_shard_advance(kmeans2_shard* sh, kmeans2_exchange* next);

/* Results of a finished session: centers (k*d FP64, host or device; the same
 * on every rank), this rank's n_local labels (host or device), and res (J,
 * iteration counts and distance_evals are global; rechecked_points counts
 * this rank's points).  Any output may be NULL.  KMEANS2_ERR_INVALID before
 * the fit has finished; the session's error after a failure. */
KMEANS2_API int kmeans2_shard_result(kmeans2_shard* sh, double* centers_out, int32_t* labels_out,
                                     kmeans2_result* res);

/* Waits for the rank's stream and frees the session (NULL is a no-op). */
KMEANS2_API void kmeans2_shard_destroy(kmeans2_shard* sh);

/*
 * kmeans2_fit_sharded -- kmeans2_fit run as `shards` ranks on this one GPU:
 * the rows of X are split into contiguous blocks (boundaries on multiples of
 * 4 rows), one session per block, and each exchange is reduced in rank order
 * by a kernel over the sessions' buffers.  Results equal kmeans2_fit bit for
 * bit; a rank whose centers differ from rank 0's at the end is reported as
 * KMEANS2_ERR_CUDA ("shard replicas diverged").  res->rechecked_points sums
 * the ranks.  Arguments as kmeans2_fit; 1 <= shards <= 64.
 */
KMEANS2_API int kmeans2_fit_sharded(const float* X, int64_t n, int32_t d, int32_t k,
                                    double subset_fraction, uint64_t seed, double tol,
                                    int32_t max_iter, int32_t shards, double* centers_out,
                                    int32_t* labels_out, kmeans2_result* res,
                                    const kmeans2_options* opt);

/* One independent clustering problem: an entry of a batch (kmeans2_fit_batched)
   or a request to a server (kmeans2_server_submit).  The limits in brackets
   are the batched form's; a server job takes any shape kmeans2_fit takes. */
typedef struct kmeans2_job {
    const float* X;             /* n*d FP32 points [DEVICE memory, 16-byte aligned];
                                   server: host or device */
    int64_t n;
    int32_t d;                  /* [1 <= d <= 64] */
    int32_t k;                  /* [1 <= k <= min(n, 256)] */
    double subset_fraction;     /* per, in (0, 1] */
    uint64_t seed;
    double tol;                 /* slow-stage tolerance; options->tol_fast, when > 0,
                                   is every job's fast-stage tolerance */
    int32_t max_iter;           /* per stage, >= 1 */
    int32_t reserved;           /* must be 0 */
    double* centers_out;        /* k*d FP64 (host or device) */
    int32_t* labels_out;        /* n int32 (host or device) */
} kmeans2_job;

/*
 * kmeans2_fit_batched -- the two-stage method of kmeans2_fit applied to `count`
 * independent jobs at once (batched form).  All jobs advance together: every
 * phase of an iteration (distances, recheck, update) is one launch over all
 * jobs still running, each job carries its own stage (fast, slow, done) and
 * convergence flag on the device, and the whole loop runs as one CUDA graph
 * with a device-side while condition.  Jobs are grouped by dimension class
 * (d rounded up to 2, 4, 8, 16, 32 or 64); per class a built-in autotuner picks
 * the distance kernel's tile shape (point slots per lane, lanes sharing a
 * point) and the 1024-point tiles per work item, timed on the first call for
 * that class and then cached for the process.  Each job's result equals
 * kmeans2_fit on that job alone.
 *
 *  jobs      count descriptors (host array).
 *  results   count results (host array), may be NULL.
 *  opt       may be NULL; precision must be FP32 or AUTO (the batched kernels
 *            are the CUDA-core FP32 form).
 * Errors: KMEANS2_ERR_INVALID (a job out of range; nothing is run),
 * KMEANS2_ERR_NONFINITE (some job holds NaN / inf: the other jobs complete),
 * KMEANS2_ERR_NOMEM, KMEANS2_ERR_CUDA.
 */
KMEANS2_API int kmeans2_fit_batched(int32_t count, const kmeans2_job* jobs,
                                    kmeans2_result* results, const kmeans2_options* opt);

/*
 * kmeans2_batched_tile_shape -- the choice the batched form's autotuner made in
 * this process for the dimension class of d: point slots per lane
 * (*points), lanes that share each point (*lanes; 1 = whole points per
 * thread) and 1024-point tiles per work item (*tiles).  Output pointers are
 * host memory and must not be NULL.  Returns KMEANS2_OK, or
 * KMEANS2_ERR_INVALID when d is outside [1, 64] or no kmeans2_fit_batched call
 * of this process has tuned that class yet (outputs untouched).
 */
KMEANS2_API int kmeans2_batched_tile_shape(int32_t d, int32_t* points, int32_t* lanes,
                                           int32_t* tiles);

/*
 * Serving: continuous batching of independent two-stage fits.  (The paper has
 * no counterpart; this is the library's request loop around kmeans2_fit.)
 *
 * A server owns `max_slots` worker threads, each with its own non-blocking
 * CUDA stream on the device that was current at creation.  Submitted jobs wait
 * in arrival order; a free worker admits the first waiting job whose device
 * footprint (kmeans2_fit_footprint) fits into the HBM budget beside the jobs
 * already running, and runs kmeans2_fit on it (graph-captured stage loops), so
 * the work of different jobs overlaps on the GPU.  A job may be passed over
 * by later, smaller jobs at most 8 times; after that nothing behind it is
 * admitted before it.  A job's data, centers and labels stay on the device
 * from admission until its result is written.  Each result equals kmeans2_fit
 * on that job alone (same kernels, exact cluster sums).
 */
typedef struct kmeans2_server kmeans2_server;

#define KMEANS2_PENDING 1             /* kmeans2_server_poll: not finished yet */

typedef struct {
    int64_t submitted, admitted, completed, failed, rejected;
    int64_t kernel_launches;          /* kernels launched by the workers */
    int32_t queued, running, slots, pad_;
    uint64_t hbm_budget, hbm_in_use, hbm_peak;   /* bytes, by footprint */
} kmeans2_server_stats;

typedef struct {
    double t_submit, t_admit, t_done; /* seconds on the server's clock */
} kmeans2_ticket_times;

/*
 * kmeans2_fit_footprint -- upper estimate of the device bytes kmeans2_fit
 * allocates for one problem: the workspace, S_s and its labels, the sampling
 * scratch, the BF16 copies when that form is chosen, the labels when the
 * caller's are not on the device, and a staged copy of X when x_on_host.
 * precision: as kmeans2_options.precision (AUTO resolves as kmeans2_fit does
 * for 16-byte aligned device X).  Returns 0 for invalid arguments.
 */
KMEANS2_API uint64_t kmeans2_fit_footprint(int64_t n, int32_t d, int32_t k,
                                           double subset_fraction, int32_t max_iter,
                                           int32_t precision, int32_t x_on_host,
                                           int32_t labels_on_host);

/*
 * kmeans2_server_create -- start a server on the current device.
 *  hbm_budget  bytes of device memory the running jobs may hold together
 *              (their footprints, with device-resident X counted too);
 *              0 = 90% of the device memory free at creation.
 *  max_slots   jobs running at once, 1..64.
 *  opt         may be NULL; precision, tol_fast, deterministic and use_graph
 *              apply to every job (stream, init_centers, start_stage,
 *              trajectories and profile must be unset).  use_graph = 1 runs
 *              each job's stage loops as graphs with a device-side while
 *              condition, 0 drives them from the worker threads; with NULL
 *              options a server of several slots uses 0.  Measured on GB300:
 *              while one job's while-graph runs, another job's while-graph
 *              does not start, whereas host-driven loops interleave with it,
 *              so short jobs progress beside long ones only with 0.
 * Returns NULL on invalid arguments or if the device cannot be used.
 */
KMEANS2_API kmeans2_server* kmeans2_server_create(uint64_t hbm_budget, int32_t max_slots,
                                                  const kmeans2_options* opt);

/*
 * kmeans2_server_submit -- queue one job; returns at once with its ticket.
 * The caller keeps job->X, centers_out and labels_out valid and untouched
 * until the job is reported finished.  Errors: KMEANS2_ERR_INVALID (argument
 * out of range), KMEANS2_ERR_ADMISSION (footprint above the whole budget; the
 * job is not queued).
 */
KMEANS2_API int kmeans2_server_submit(kmeans2_server* srv, const kmeans2_job* job,
                                      uint64_t* ticket);

/*
 * kmeans2_server_poll -- KMEANS2_PENDING while the job waits or runs; once it
 * has finished, its kmeans2_fit status (0 or a negative code), with *res and
 * *times (each may be NULL) filled in, and the ticket is released.
 * KMEANS2_ERR_INVALID for an unknown or released ticket.
 */
KMEANS2_API int kmeans2_server_poll(kmeans2_server* srv, uint64_t ticket, kmeans2_result* res,
                                    kmeans2_ticket_times* times);

/* kmeans2_server_poll after waiting up to timeout_s seconds (< 0: no limit)
   for the job to finish; KMEANS2_PENDING if it has not. */
KMEANS2_API int kmeans2_server_wait(kmeans2_server* srv, uint64_t ticket, double timeout_s,
                                    kmeans2_result* res, kmeans2_ticket_times* times);

/*
 * Lazy input: a job whose points are produced only when it is admitted, so
 * that waiting jobs hold no device memory (a request queue under overload).
 *
 *  materialize(user, X, stream)  called on the worker thread, with the server's
 *      device current, once the job is admitted: it must enqueue on `stream`
 *      (a cudaStream_t) the writing of the job's n*d FP32 points to X (device
 *      memory owned by the server, 16-byte aligned, valid until the job is
 *      done) and return 0, or return nonzero to fail the job
 *      (KMEANS2_ERR_INVALID).
 *  consume(user, centers, labels, stream)  may be NULL: called after the fit
 *      with its device centers (k*d FP64) and labels (n int32), which the
 *      server frees when consume returns; copies must be enqueued on `stream`.
 *  job->X, centers_out and labels_out are ignored (NULL); the job's footprint
 *  counts the n*d*4 bytes of X.  Otherwise as kmeans2_server_submit.
 */
typedef int (*kmeans2_materialize_fn)(void* user, float* X, void* stream);
typedef void (*kmeans2_consume_fn)(void* user, const double* centers, const int32_t* labels,
                                   void* stream);
KMEANS2_API int kmeans2_server_submit_lazy(kmeans2_server* srv, const kmeans2_job* job,
                                           kmeans2_materialize_fn materialize,
                                           kmeans2_consume_fn consume, void* user,
                                           uint64_t* ticket);

/* Waits up to timeout_s seconds (< 0: no limit) for some job to finish that
   no earlier call returned, and writes its ticket: KMEANS2_OK, or
   KMEANS2_PENDING on timeout.  The ticket is then collected with
   kmeans2_server_poll. */
KMEANS2_API int kmeans2_server_wait_any(kmeans2_server* srv, double timeout_s, uint64_t* ticket);

/* Counters of the server; returns KMEANS2_ERR_INVALID for NULL arguments. */
KMEANS2_API int kmeans2_server_stats_get(kmeans2_server* srv, kmeans2_server_stats* out);

/*
 * kmeans2_server_set_policy -- which waiting job a free worker admits.
 *  KMEANS2_POLICY_FIFO (default): the first job in arrival order that fits the
 *      budget; a job passed over 8 times blocks everything behind it.
 *  KMEANS2_POLICY_SHORTEST: the fitting job with the least work per iteration
 *      (n * k * d), except that the oldest job goes first once it has waited
 *      aging_s seconds (and nothing else is admitted until it fits).
 * Errors: KMEANS2_ERR_INVALID (NULL server, unknown policy, aging_s < 0).
 */
#define KMEANS2_POLICY_FIFO 0
#define KMEANS2_POLICY_SHORTEST 1
KMEANS2_API int kmeans2_server_set_policy(kmeans2_server* srv, int32_t policy, double aging_s);

/* Seconds since the server was created (its clock for kmeans2_ticket_times). */
KMEANS2_API double kmeans2_server_now(kmeans2_server* srv);

/* Stop a server: jobs still waiting finish with KMEANS2_ERR_ADMISSION without
   running, running jobs complete, the workers exit.  Tickets not yet polled
   are released. */
KMEANS2_API void kmeans2_server_destroy(kmeans2_server* srv);

/*
 * kmeans_step -- one Lloyd iteration (Section 4.1; the loop body of the
 * Algorithm) from given centers.
 *
 *  centers_in    k*d FP64 (host or device), the centers the points are assigned to.
 *  centers_out   k*d FP64 (host or device): cluster means; an empty cluster
 *                keeps its center.  May equal centers_in.
 *  labels_out    n int32 (host or device).
 *  J_out         host, may be NULL: J of this assignment against centers_in (Eq. 3).
 *  shift_out     host, may be NULL: max_j ||c_j' - c_j||_2.
 *  empty_out     host, may be NULL: number of empty clusters.
 * Errors as kmeans2_fit.
 */
KMEANS2_API int kmeans_step(const float* X, int64_t n, int32_t d, int32_t k, const double* centers_in,
                double* centers_out, int32_t* labels_out, double* J_out, double* shift_out,
                int32_t* empty_out, const kmeans2_options* opt);

/*
 * kmeans_step_noalloc -- kmeans_step for callers that cannot allocate device
 * memory during the call.  (The paper has no counterpart: this is an
 * integration variant of the library.)
 *
 * Some callers cannot call cudaMalloc once they are running: a service whose
 * device memory is entirely owned by its own caching allocator or memory pool,
 * where a stray allocation could fail or fragment that pool, or a latency-
 * critical loop that must not wait on the allocator.  This entry point runs
 * kmeans_step's CUDA-core FP32 form (the form whose scratch fits the array for
 * every shape within the limits below; the tensor-core forms would need a copy
 * of X) and takes its scratch from one fixed device array of 24 MiB compiled
 * into the library, which every GPU that loads the library holds until the
 * process exits.  It calls no cudaMalloc, cudaFree or other allocating
 * routine.  Its labels, centers and J equal kmeans_step's in any form.
 *
 *  X, centers_in, centers_out, labels_out: DEVICE memory on the current device
 *                (X 16-byte aligned); the caller still owns and passes them.
 *  Limits: n <= 4,194,304, k <= 1024, d <= 128 (plus the limits of kmeans_step).
 *          Larger shapes are rejected with KMEANS2_ERR_INVALID and a message in
 *          kmeans2_last_error(); host pointers are rejected the same way.
 *  stream: cudaStream_t (NULL = legacy default stream).
 *  Other arguments and results as kmeans_step.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.  Every call on a device
 * shares the one array and overwrites it (each call clears what must start at
 * zero): calls that overlap on the GPU -- concurrent streams or threads --
 * race and must be serialised by the caller.
 */
KMEANS2_API int kmeans_step_noalloc(const float* X, int64_t n, int32_t d, int32_t k,
                                    const double* centers_in, double* centers_out,
                                    int32_t* labels_out, double* J_out, double* shift_out,
                                    int32_t* empty_out, void* stream);

/*
 * kmeans2_subset_size -- m = min(n, max(k, ceil(per*n))), the size of S_s
 * (the Algorithm's per% share of the data; at least k points so that k distinct
 * initial centers exist).  Host only; returns -1 on invalid arguments.
 */
KMEANS2_API int64_t kmeans2_subset_size(int64_t n, int32_t k, double subset_fraction);

/*
 * kmeans2_sample -- the Algorithm's two random draws (the fast-stage subset
 * S_s, a per% share of S_n, and the initial centers picked at random from
 * it), computed on the GPU.
 *
 * SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) is used as a counter-based
 * generator: key_i = mix64(seed + (i+1) * 0x9E3779B97F4A7C15).  S_s is the set
 * of the m indices i in [0, n) with the smallest key_i, written ascending to
 * subset_out (m int64).  The initial centers are the k positions p in [0, m)
 * with the smallest key_{n+p}, written in increasing key order to
 * init_pos_out (k int64): center j is X[subset_out[init_pos_out[j]]].
 * Both outputs may be host or device pointers.
 */
KMEANS2_API int kmeans2_sample(int64_t n, int32_t k, double subset_fraction, uint64_t seed,
                   int64_t* subset_out, int64_t* init_pos_out, void* stream);

/* Human-readable name of a status code (static storage). */
KMEANS2_API const char* kmeans2_strerror(int status);

/* Detail of the last failure on the calling thread (the failing CUDA call and
   its error string), or "" if none.  Thread-local storage, valid until the
   thread's next failing call. */
KMEANS2_API const char* kmeans2_last_error(void);

/* Library version, (major << 16) | minor. */
KMEANS2_API int32_t kmeans2_version(void);

/* Device scratch of every call comes from a library-owned stream-ordered pool
 * per GPU that keeps freed memory mapped, so repeated calls (a serving loop,
 * the stage loops of many fits) reuse it without mapping it again.  This call
 * waits for the current device and returns the pool's unused memory to the
 * driver.  Returns KMEANS2_OK or KMEANS2_ERR_CUDA. */
KMEANS2_API int kmeans2_release_memory(void);

#ifdef __cplusplus
}
#endif

#endif /* KMEANS2_H */
