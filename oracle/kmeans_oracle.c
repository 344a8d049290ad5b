/*
 * kmeans_oracle.c -- plain, slow, FP64 CPU restatement of the two-stage k-means
 * of Salman et al., "Fast k-means algorithm clustering" (arXiv 1108.1351).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  It shares no code, header,
 * table or helper with the CUDA library; neither side includes the other.
 *
 * What it computes, and where the paper says so:
 *   - sampling of the fast-stage subset S_s and of the initial centers
 *     (Section 2 and the Algorithm: a per% share of S_n, centers drawn at
 *     random from the data);
 *   - the "modified distance" (Eq. 1 without the square root, Algorithm),
 *     the nearest-center assignment with the lowest index winning ties;
 *   - the objective J (Eq. 3; WCSS of Eqs. 6-7 read with squared norms);
 *   - the center update as the mean of each cluster (Lloyd's method,
 *     Section 4.1), an empty cluster keeping its center;
 *   - the stopping test on the largest center movement (Section 5, Section 6:
 *     mu is the accuracy asked for, measured as center movement);
 *   - the fast stage on S_s, then the slow stage on S_n started from the fast
 *     stage's final centers (Algorithm; Section 2; Section 5).
 *
 * Readings where the paper is silent or garbled (each also listed in the
 * design notes):
 *   - The Algorithm prints the mean step only after the fast loop; Lloyd's
 *     method (Section 4.1) updates the centers in every iteration, so each
 *     iteration here is: assign, J, update, stop test.
 *   - The loop condition on J and mu is read as: stop once
 *     max_j ||c_j' - c_j||_2 <= tol; the iteration that detects convergence
 *     is counted (Table 1 shows old = new centers in the last counted
 *     iteration of each stage).
 *   - Subset size m = min(n, max(k, ceil(f*n))), ceil taken of the double
 *     product f*n.
 *   - Random choice: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) used as a
 *     counter-based generator, key_i = mix64(seed + (i+1)*GAMMA).  S_s is the
 *     set of the m indices with the smallest keys, listed ascending; the k
 *     initial centers are the k positions p in [0, m) with the smallest keys
 *     key_{n+p}, taken in increasing key order (a uniformly random ordered
 *     k-subset of S_s).  mix64 is a bijection, so keys never tie.
 *   - Empty cluster: keeps its previous center (counted in `empty`).
 *
 * Arithmetic (FP64 unless stated):
 *   delta_ij = sum_t fma(x_t - c_jt, x_t - c_jt, acc), acc = 0, t ascending,
 *   x_t the FP32 value widened exactly.  Label = first j reaching the minimum.
 *   Sums for the means and for J: Neumaier-compensated, in index order.
 *   shift = max_j sqrt(sum_t (c'_jt - c_jt)^2).
 *
 * Threads: the assignment loop may run on several OpenMP threads; each point
 * is independent, so no arithmetic is reordered.  Every sum runs on one thread
 * in index order.  Results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL -1
#define OR_ENOMEM -2

/* ---------------------------------------------------------------- SplitMix64 */

#define SM64_GAMMA 0x9E3779B97F4A7C15ULL

/* Finalizer of SplitMix64 (Steele, Lea & Flood 2014; constants of Stafford's
 * "Mix13" variant used by the published SplitMix64). */
static uint64_t sm64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Output number i (0-based) of the SplitMix64 stream seeded with `seed`. */
uint64_t oracle_splitmix64_at(uint64_t seed, uint64_t i)
{
    return sm64_mix(seed + (i + 1) * SM64_GAMMA);
}

/* ---------------------------------------------------------------- sampling */

int64_t oracle_subset_size(int64_t n, int32_t k, double f)
{
    double want = ceil(f * (double)n);
    int64_t m = (int64_t)want;
    if (m < k) m = k;
    if (m > n) m = n;
    return m;
}

typedef struct { uint64_t key; int64_t idx; } key_idx;

static int cmp_key(const void* a, const void* b)
{
    const key_idx* x = (const key_idx*)a;
    const key_idx* y = (const key_idx*)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->idx < y->idx) ? -1 : (x->idx > y->idx);
}

static int cmp_i64(const void* a, const void* b)
{
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x < y) ? -1 : (x > y);
}

/* S_s (m indices, ascending) and the k initial-center positions within S_s. */
int oracle_sample(int64_t n, int32_t k, double f, uint64_t seed,
                  int64_t* subset_out, int64_t* init_pos_out)
{
    if (n < 1 || k < 1 || k > n || !(f > 0.0 && f <= 1.0)) return OR_EINVAL;
    int64_t m = oracle_subset_size(n, k, f);

    key_idx* all = (key_idx*)malloc((size_t)n * sizeof(key_idx));
    if (!all) return OR_ENOMEM;
    for (int64_t i = 0; i < n; ++i) {
        all[i].key = oracle_splitmix64_at(seed, (uint64_t)i);
        all[i].idx = i;
    }
    qsort(all, (size_t)n, sizeof(key_idx), cmp_key);
    for (int64_t i = 0; i < m; ++i) subset_out[i] = all[i].idx;
    qsort(subset_out, (size_t)m, sizeof(int64_t), cmp_i64);
    free(all);

    key_idx* pos = (key_idx*)malloc((size_t)m * sizeof(key_idx));
    if (!pos) return OR_ENOMEM;
    for (int64_t p = 0; p < m; ++p) {
        pos[p].key = oracle_splitmix64_at(seed, (uint64_t)(n + p));
        pos[p].idx = p;
    }
    qsort(pos, (size_t)m, sizeof(key_idx), cmp_key);
    for (int32_t j = 0; j < k; ++j) init_pos_out[j] = pos[j].idx;
    free(pos);
    return OR_OK;
}

/* ---------------------------------------------------------------- Lloyd step */

/* Neumaier's compensated summation: running sum s, running correction c. */
static void neumaier_add(double* s, double* c, double v)
{
    double t = *s + v;
    if (fabs(*s) >= fabs(v))
        *c += (*s - t) + v;
    else
        *c += (v - t) + *s;
    *s = t;
}

/* Squared Euclidean distance of the Algorithm's "modified distance". */
static double sq_dist(const float* x, const double* c, int32_t d)
{
    double acc = 0.0;
    for (int32_t t = 0; t < d; ++t) {
        double a = (double)x[t] - c[t];
        acc = fma(a, a, acc);
    }
    return acc;
}

/* Assignment: label_i = argmin_j delta_ij (first j on ties), dmin_i = that delta. */
int oracle_assign(const float* X, int64_t n, int32_t d, int32_t k,
                  const double* C, int32_t* labels, double* dmin, int32_t nthreads)
{
    if (n < 0 || d < 1 || k < 1) return OR_EINVAL;
    if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
    for (int64_t i = 0; i < n; ++i) {
        const float* x = X + (size_t)i * (size_t)d;
        double best = sq_dist(x, C, d);
        int32_t arg = 0;
        for (int32_t j = 1; j < k; ++j) {
            double v = sq_dist(x, C + (size_t)j * (size_t)d, d);
            if (v < best) { best = v; arg = j; }
        }
        labels[i] = arg;
        if (dmin) dmin[i] = best;
    }
    return OR_OK;
}

/* One Lloyd iteration: assign against C_in, J of that assignment (Eq. 3),
 * new centers = cluster means (empty cluster keeps its center), shift. */
int oracle_lloyd_step(const float* X, int64_t n, int32_t d, int32_t k,
                      const double* C_in, double* C_out, int32_t* labels,
                      double* J_out, double* shift_out, int32_t* empty_out,
                      int32_t nthreads)
{
    if (n < 1 || d < 1 || k < 1) return OR_EINVAL;
    double* dmin = (double*)malloc((size_t)n * sizeof(double));
    double* sum = (double*)calloc((size_t)k * (size_t)d, sizeof(double));
    double* cmp = (double*)calloc((size_t)k * (size_t)d, sizeof(double));
    int64_t* cnt = (int64_t*)calloc((size_t)k, sizeof(int64_t));
    if (!dmin || !sum || !cmp || !cnt) {
        free(dmin); free(sum); free(cmp); free(cnt);
        return OR_ENOMEM;
    }
    oracle_assign(X, n, d, k, C_in, labels, dmin, nthreads);

    double js = 0.0, jc = 0.0;
    for (int64_t i = 0; i < n; ++i) neumaier_add(&js, &jc, dmin[i]);
    if (J_out) *J_out = js + jc;

    for (int64_t i = 0; i < n; ++i) {
        int32_t j = labels[i];
        const float* x = X + (size_t)i * (size_t)d;
        cnt[j] += 1;
        for (int32_t t = 0; t < d; ++t)
            neumaier_add(&sum[(size_t)j * d + t], &cmp[(size_t)j * d + t], (double)x[t]);
    }

    int32_t empty = 0;
    double shift = 0.0;
    for (int32_t j = 0; j < k; ++j) {
        const double* c = C_in + (size_t)j * d;
        double* cn = C_out + (size_t)j * d;
        if (cnt[j] == 0) {
            ++empty;
            for (int32_t t = 0; t < d; ++t) cn[t] = c[t];
        } else {
            for (int32_t t = 0; t < d; ++t)
                cn[t] = (sum[(size_t)j * d + t] + cmp[(size_t)j * d + t]) / (double)cnt[j];
        }
        double mv = 0.0;
        for (int32_t t = 0; t < d; ++t) {
            double e = cn[t] - c[t];
            mv += e * e;
        }
        mv = sqrt(mv);
        if (mv > shift) shift = mv;
    }
    if (shift_out) *shift_out = shift;
    if (empty_out) *empty_out = empty;
    free(dmin); free(sum); free(cmp); free(cnt);
    return OR_OK;
}

/* ---------------------------------------------------------------- stage loop */

/* Lloyd loop until shift <= tol or max_iter iterations (both counted).
 * C (k*d) holds the starting centers on entry and the final c' on exit.
 * labels/J are those of the last assignment.  traj_J / traj_shift, when not
 * NULL, receive one value per iteration (capacity max_iter). */
int oracle_lloyd_stage(const float* X, int64_t n, int32_t d, int32_t k,
                       double* C, double tol, int32_t max_iter,
                       int32_t* labels, double* J_out, int32_t* iters_out,
                       int32_t* converged_out, int32_t* empty_out,
                       double* traj_J, double* traj_shift, int32_t nthreads)
{
    if (n < 1 || d < 1 || k < 1 || k > n || max_iter < 1 || !(tol >= 0.0)) return OR_EINVAL;
    double* nxt = (double*)malloc((size_t)k * (size_t)d * sizeof(double));
    if (!nxt) return OR_ENOMEM;
    int32_t it = 0, conv = 0, empty = 0;
    double J = 0.0, shift = 0.0;
    while (it < max_iter) {
        int rc = oracle_lloyd_step(X, n, d, k, C, nxt, labels, &J, &shift, &empty, nthreads);
        if (rc != OR_OK) { free(nxt); return rc; }
        if (traj_J) traj_J[it] = J;
        if (traj_shift) traj_shift[it] = shift;
        ++it;
        memcpy(C, nxt, (size_t)k * (size_t)d * sizeof(double));
        if (shift <= tol) { conv = 1; break; }
    }
    free(nxt);
    if (J_out) *J_out = J;
    if (iters_out) *iters_out = it;
    if (converged_out) *converged_out = conv;
    if (empty_out) *empty_out = empty;
    return OR_OK;
}

/* ---------------------------------------------------------------- two-stage fit */

typedef struct {
    double J;
    int32_t iters_fast, iters_slow;
    int32_t converged_fast, converged_slow;
    int32_t empty_clusters;
    int32_t pad_;
    int64_t subset_size;
    int64_t distance_evals;
} oracle_result;

/* Two-stage fit (Algorithm).  fast_centers_out (k*d), when not NULL, receives
 * the fast stage's final centers, i.e. the slow stage's starting centers. */
int oracle_fit(const float* X, int64_t n, int32_t d, int32_t k, double f,
               uint64_t seed, double tol_fast, double tol, int32_t max_iter,
               double* centers_out, int32_t* labels_out, double* fast_centers_out,
               double* traj_J_fast, double* traj_shift_fast,
               double* traj_J_slow, double* traj_shift_slow,
               oracle_result* res, int32_t nthreads)
{
    if (n < 1 || d < 1 || k < 1 || k > n || !(f > 0.0 && f <= 1.0) ||
        max_iter < 1 || !(tol >= 0.0))
        return OR_EINVAL;
    if (!(tol_fast > 0.0)) tol_fast = tol;
    int64_t m = oracle_subset_size(n, k, f);
    int64_t* subset = (int64_t*)malloc((size_t)m * sizeof(int64_t));
    int64_t* pos = (int64_t*)malloc((size_t)k * sizeof(int64_t));
    float* Xs = (float*)malloc((size_t)m * (size_t)d * sizeof(float));
    int32_t* ls = (int32_t*)malloc((size_t)m * sizeof(int32_t));
    if (!subset || !pos || !Xs || !ls) {
        free(subset); free(pos); free(Xs); free(ls);
        return OR_ENOMEM;
    }
    int rc = oracle_sample(n, k, f, seed, subset, pos);
    if (rc != OR_OK) goto done;
    for (int64_t p = 0; p < m; ++p)
        memcpy(Xs + (size_t)p * d, X + (size_t)subset[p] * d, (size_t)d * sizeof(float));
    for (int32_t j = 0; j < k; ++j)
        for (int32_t t = 0; t < d; ++t)
            centers_out[(size_t)j * d + t] = (double)Xs[(size_t)pos[j] * d + t];

    oracle_result r;
    memset(&r, 0, sizeof(r));
    double Jf = 0.0;
    int32_t ef = 0;
    rc = oracle_lloyd_stage(Xs, m, d, k, centers_out, tol_fast, max_iter, ls, &Jf,
                            &r.iters_fast, &r.converged_fast, &ef,
                            traj_J_fast, traj_shift_fast, nthreads);
    if (rc != OR_OK) goto done;
    if (fast_centers_out)
        memcpy(fast_centers_out, centers_out, (size_t)k * (size_t)d * sizeof(double));
    rc = oracle_lloyd_stage(X, n, d, k, centers_out, tol, max_iter, labels_out, &r.J,
                            &r.iters_slow, &r.converged_slow, &r.empty_clusters,
                            traj_J_slow, traj_shift_slow, nthreads);
    if (rc != OR_OK) goto done;
    r.subset_size = m;
    /* Section 3: cost O(K Q_f N_f) + O(K Q_s N) distance evaluations. */
    r.distance_evals = (int64_t)r.iters_fast * m * k + (int64_t)r.iters_slow * n * k;
    if (res) *res = r;
done:
    free(subset); free(pos); free(Xs); free(ls);
    return rc;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
