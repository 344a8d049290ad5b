"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer (CPU).

The oracle's C source is compiled together with a small driver into one
executable instrumented with -fsanitize=address,undefined (no recovery: any
finding aborts with a non-zero exit).  The driver runs every entry point on
small synthetic inputs and on the degenerate shapes (k = n, n = 1, f = 1,
exact duplicates, an empty cluster), so out-of-bounds accesses, leaks, signed
overflow or misaligned loads anywhere on those paths fail the test."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "kmeans_oracle.c")

DRIVER = r"""
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double J;
    int32_t iters_fast, iters_slow, converged_fast, converged_slow, empty_clusters, pad_;
    int64_t subset_size, distance_evals;
} oracle_result;

int64_t oracle_subset_size(int64_t n, int32_t k, double f);
int oracle_sample(int64_t n, int32_t k, double f, uint64_t seed, int64_t* subset_out,
                  int64_t* init_pos_out);
int oracle_assign(const float* X, int64_t n, int32_t d, int32_t k, const double* C,
                  int32_t* labels, double* dmin, int32_t nthreads);
int oracle_lloyd_step(const float* X, int64_t n, int32_t d, int32_t k, const double* C_in,
                      double* C_out, int32_t* labels, double* J_out, double* shift_out,
                      int32_t* empty_out, int32_t nthreads);
int oracle_fit(const float* X, int64_t n, int32_t d, int32_t k, double f, uint64_t seed,
               double tol_fast, double tol, int32_t max_iter, double* centers_out,
               int32_t* labels_out, double* fast_centers_out, double* traj_J_fast,
               double* traj_shift_fast, double* traj_J_slow, double* traj_shift_slow,
               oracle_result* res, int32_t nthreads);

static uint64_t s = 0x9E3779B97F4A7C15ull;
static double unif(void)
{
    s ^= s << 13; s ^= s >> 7; s ^= s << 17;
    return (double)(s >> 11) * (1.0 / 9007199254740992.0);
}

static int run(int64_t n, int32_t d, int32_t k, double f, int dup)
{
    float* X = malloc(sizeof(float) * (size_t)(n * d));
    for (int64_t i = 0; i < n * d; ++i) X[i] = (float)(20.0 * unif() - 10.0);
    if (dup)
        for (int64_t i = 1; i < n; ++i) memcpy(X + i * d, X, sizeof(float) * (size_t)d);
    const int maxit = 30;
    double* C = malloc(sizeof(double) * (size_t)(k * d));
    double* Cf = malloc(sizeof(double) * (size_t)(k * d));
    double* C2 = malloc(sizeof(double) * (size_t)(k * d));
    int32_t* lab = malloc(sizeof(int32_t) * (size_t)n);
    double* dm = malloc(sizeof(double) * (size_t)n);
    double *t1 = malloc(sizeof(double) * maxit), *t2 = malloc(sizeof(double) * maxit);
    double *t3 = malloc(sizeof(double) * maxit), *t4 = malloc(sizeof(double) * maxit);
    oracle_result r;
    int rc = oracle_fit(X, n, d, k, f, 7, 0.0, 1e-6, maxit, C, lab, Cf, t1, t2, t3, t4, &r, 2);
    if (rc == 0) rc = oracle_assign(X, n, d, k, C, lab, dm, 2);
    double J, sh;
    int32_t em;
    if (rc == 0) rc = oracle_lloyd_step(X, n, d, k, C, C2, lab, &J, &sh, &em, 1);
    int64_t m = oracle_subset_size(n, k, f);
    int64_t* sub = malloc(sizeof(int64_t) * (size_t)m);
    int64_t* pos = malloc(sizeof(int64_t) * (size_t)k);
    if (rc == 0) rc = oracle_sample(n, k, f, 3, sub, pos);
    free(X); free(C); free(Cf); free(C2); free(lab); free(dm);
    free(t1); free(t2); free(t3); free(t4); free(sub); free(pos);
    return rc;
}

int main(void)
{
    int rc = 0;
    rc |= run(2000, 3, 7, 0.1, 0);
    rc |= run(500, 16, 40, 0.3, 0);
    rc |= run(50, 4, 50, 1.0, 0);     /* k = n, f = 1 */
    rc |= run(1, 2, 1, 1.0, 0);       /* n = 1 */
    rc |= run(300, 5, 6, 0.5, 1);     /* all points equal: ties and empty clusters */
    if (rc != 0) { printf("status %d\n", rc); return 2; }
    printf("ok\n");
    return 0;
}
"""


def test_oracle_under_address_and_undefined_behavior_sanitizers(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    drv = tmp_path / "driver.c"
    drv.write_text(DRIVER)
    exe = tmp_path / "oracle_sanitized"
    cmd = ["gcc", "-O1", "-g", "-std=c11", "-fno-omit-frame-pointer",
           "-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-ffp-contract=off",
           SRC, str(drv), "-lm", "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in (r.stderr or ""):
        pytest.skip("sanitizer runtime not available: " + r.stderr.strip()[:200])
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300, env=env)
    assert run.returncode == 0, run.stdout + run.stderr
    assert run.stdout.strip() == "ok"
