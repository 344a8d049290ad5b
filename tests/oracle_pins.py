"""Pins for the FP64 oracle: checks against what the paper and the mathematics
fix, never against the oracle itself.

Each ``pin_*`` function takes an oracle object (the default build, or a
variant with a planted mistake) and raises ``AssertionError`` when the pin does
not hold.  ``test_oracle_pins.py`` runs them on the real oracle;
``test_oracle_mutations.py`` shows that every planted mistake trips one.

Sources of truth used here:
* brute force over all k^n labelings / all partitions (tiny n);
* numpy library routines (mean, plain sums) for the closed forms;
* Lloyd's invariants (Section 4.1 cites Lloyd's method): J never increases,
  a fixed point has each center at the mean of its points and no point closer
  to another center; at exact means one step suffices (Section 7);
* the Theorem of Section 4.1: with the whole set as the subset, the slow stage
  starts at a fixed point;
* the stage hand-off (Section 5: the slow stage starts from the fast stage's
  last centers);
* Section 3's cost model O(K Q_f N_f) + O(K Q_s N);
* SplitMix64's published outputs (tests/golden/splitmix64.txt).
"""
from __future__ import annotations

import itertools
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
M64 = (1 << 64) - 1


def _py_splitmix64_at(seed: int, i: int) -> int:
    """Independent Python restatement of SplitMix64 output i (big-int arithmetic)."""
    z = (seed + (i + 1) * 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def _np_cost(X, C, labels):
    """sum_i ||x_i - c_{l_i}||^2 with numpy (float64)."""
    X = np.asarray(X, dtype=np.float64)
    diff = X - np.asarray(C, dtype=np.float64)[labels]
    return float(np.sum(diff * diff))


def _np_sqdist(X, C):
    X = np.asarray(X, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    return ((X[:, None, :] - C[None, :, :]) ** 2).sum(-1)


def _rel(a, b):
    return abs(a - b) / max(abs(a), abs(b), 1e-300)


# --------------------------------------------------------------------- sampling

def pin_splitmix64_golden(o):
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as fh:
        rows = [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]
    assert rows
    for seed, idx, val in rows:
        assert o.splitmix64_at(int(seed), int(idx)) == int(val), (seed, idx)


def pin_subset_size_rule(o):
    # m = min(n, max(k, ceil(f n)))
    assert o.subset_size(20000, 4, 0.1) == 2000
    assert o.subset_size(1000, 256, 0.1) == 256
    assert o.subset_size(10, 3, 1.0) == 10
    assert o.subset_size(7, 2, 0.5) == 4
    assert o.subset_size(500_000_000, 32, 0.01) == 5_000_000


def pin_sample_brute_force(o):
    """S_s = the m smallest keys (ascending indices); init = k smallest keys of
    stream positions n..n+m-1, in key order.  Recomputed here in pure Python."""
    for (n, k, f, seed) in [(50, 3, 0.2, 0), (200, 7, 0.1, 12345), (31, 31, 0.5, 9),
                            (1000, 5, 0.013, 2**63 + 5)]:
        sub, pos = o.sample(n, k, f, seed)
        m = o.subset_size(n, k, f)
        keys = [_py_splitmix64_at(seed, i) for i in range(n)]
        want = sorted(sorted(range(n), key=lambda i: keys[i])[:m])
        assert list(sub) == want, (n, k, f, seed)
        pk = [_py_splitmix64_at(seed, n + p) for p in range(m)]
        want_pos = sorted(range(m), key=lambda p: pk[p])[:k]
        assert list(pos) == want_pos
        assert len(set(pos.tolist())) == k and all(0 <= p < m for p in pos)


def pin_sample_uniform(o):
    """Each index is in S_s with probability m/n (chi-square over many seeds)."""
    n, k, f, trials = 20, 2, 0.25, 4000
    m = o.subset_size(n, k, f)
    hits = np.zeros(n)
    first = np.zeros(m)
    for s in range(trials):
        sub, pos = o.sample(n, k, f, s)
        hits[sub] += 1
        first[pos[0]] += 1
    exp = trials * m / n
    chi2 = float(((hits - exp) ** 2 / exp).sum())
    assert chi2 < 60.0, chi2           # 19 dof: P(chi2 > 60) < 1e-5
    exp2 = trials / m
    chi2b = float(((first - exp2) ** 2 / exp2).sum())
    assert chi2b < 30.0, chi2b         # 4 dof


# ------------------------------------------------------------------ assignment

def pin_assign_brute_force(o):
    """The labeling minimises J over all k^n labelings (Eq. 3 for fixed centers)."""
    rng = np.random.default_rng(1)
    for trial in range(12):
        n = int(rng.integers(2, 8))
        d = int(rng.integers(1, 4))
        k = int(rng.integers(2, 4))
        X = rng.normal(size=(n, d)).astype(np.float32)
        C = rng.normal(size=(k, d))
        lab, dm = o.assign(X, C)
        best = min(_np_cost(X, C, np.array(L)) for L in itertools.product(range(k), repeat=n))
        got = _np_cost(X, C, lab)
        assert _rel(got, best) < 1e-12, (trial, got, best)
        assert np.allclose(dm, _np_sqdist(X, C)[np.arange(n), lab], rtol=1e-13, atol=0)


def pin_assign_ties_lowest_index(o):
    X = np.array([[0.0], [3.0], [5.0]], dtype=np.float32)
    for C, want in [([[-1.0], [1.0]], [0, 1, 1]), ([[1.0], [-1.0]], [0, 0, 0]),
                    ([[2.0], [4.0], [4.0]], [0, 0, 1]), ([[5.0], [5.0]], [0, 0, 0]),
                    ([[4.0], [6.0], [2.0]], [2, 0, 0])]:
        lab, _ = o.assign(X, np.array(C))
        assert lab.tolist() == want, (C, lab.tolist(), want)


def pin_assign_matches_numpy_argmin(o):
    rng = np.random.default_rng(2)
    X = rng.normal(size=(300, 5)).astype(np.float32) * 3
    C = rng.normal(size=(9, 5)) * 3
    lab, dm = o.assign(X, C)
    D = _np_sqdist(X, C)
    assert np.array_equal(lab, D.argmin(1))
    assert np.allclose(dm, D.min(1), rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------------- update

def _random_instance(seed, n=400, d=4, k=6, spread=5.0):
    rng = np.random.default_rng(seed)
    X = (rng.normal(size=(n, d)) + spread * rng.normal(size=(k, d))[rng.integers(0, k, n)])
    return X.astype(np.float32), (spread * rng.normal(size=(k, d)))


def pin_update_is_mean(o):
    X, C = _random_instance(3)
    Cn, lab, J, shift, empty = o.lloyd_step(X, C)
    X64 = X.astype(np.float64)
    for j in range(C.shape[0]):
        mem = X64[lab == j]
        if len(mem):
            assert np.allclose(Cn[j], mem.mean(0), rtol=1e-13, atol=1e-13), j
        else:
            assert np.array_equal(Cn[j], C[j])
    assert _rel(J, _np_cost(X, C, lab)) < 1e-12
    assert _rel(shift, float(np.linalg.norm(Cn - C, axis=1).max())) < 1e-12


def pin_mean_minimises(o):
    """Closed form: the mean is the unique minimiser of sum ||x - c||^2."""
    X, C = _random_instance(4, n=120, d=3, k=3)
    Cn, lab, _, _, _ = o.lloyd_step(X, C)
    rng = np.random.default_rng(5)
    for j in range(3):
        mem = X[lab == j].astype(np.float64)
        if not len(mem):
            continue
        base = float(((mem - Cn[j]) ** 2).sum())
        for _ in range(20):
            e = rng.normal(size=3) * 1e-3
            assert float(((mem - (Cn[j] + e)) ** 2).sum()) > base


def pin_empty_cluster_keeps_center(o):
    X = np.array([[0.0, 0.0], [1.0, 0.0], [10.0, 10.0], [11.0, 10.0]], dtype=np.float32)
    C = np.array([[0.0, 0.0], [10.0, 10.0], [1e6, -1e6]])
    Cn, lab, J, shift, empty = o.lloyd_step(X, C)
    assert empty == 1
    assert lab.tolist() == [0, 0, 1, 1]
    assert np.array_equal(Cn[2], C[2])
    assert np.array_equal(Cn[0], [0.5, 0.0]) and np.array_equal(Cn[1], [10.5, 10.0])
    assert J == 2.0 and shift == 0.5


def pin_step_large_offsets(o):
    """Data far from the origin: the FP64 sums must not lose the spread."""
    rng = np.random.default_rng(6)
    X = (1e4 + rng.normal(size=(500, 3))).astype(np.float32)
    C = X[:4].astype(np.float64)
    Cn, lab, J, shift, _ = o.lloyd_step(X, C)
    X64 = X.astype(np.float64)
    for j in range(4):
        assert np.allclose(Cn[j], X64[lab == j].mean(0), rtol=1e-15, atol=1e-11)
    assert _rel(J, _np_cost(X, C, lab)) < 1e-11


# ----------------------------------------------------------------- stage loop

def pin_J_non_increasing(o):
    for s in range(6):
        X, C = _random_instance(10 + s, n=600, d=3, k=7)
        r = o.lloyd_stage(X, C, tol=0.0, max_iter=60)
        tj = r["traj_J"]
        assert len(tj) >= 2
        assert np.all(np.diff(tj) <= 1e-12 * tj[:-1]), tj


def pin_fixed_point(o):
    """At convergence with shift 0: each center is the mean of its points and
    no point is strictly closer to another center."""
    X, C = _random_instance(20, n=500, d=2, k=5)
    r = o.lloyd_stage(X, C, tol=0.0, max_iter=200)
    assert r["converged"] and r["traj_shift"][-1] == 0.0
    Cf, lab = r["centers"], r["labels"]
    X64 = X.astype(np.float64)
    for j in range(5):
        mem = X64[lab == j]
        if len(mem):
            assert np.allclose(Cf[j], mem.mean(0), rtol=1e-13, atol=1e-13)
    D = _np_sqdist(X, Cf)
    assert np.all(D[np.arange(len(X)), lab] <= D.min(1) * (1 + 1e-12) + 1e-12)


def pin_one_step_at_exact_means(o):
    """Section 7: centers already at the means need a single Lloyd step."""
    X = np.array([[0, 0], [2, 0], [0, 2], [2, 2], [20, 20], [22, 20], [20, 22], [22, 22]],
                 dtype=np.float32)
    C = np.array([[1.0, 1.0], [21.0, 21.0]])
    r = o.lloyd_stage(X, C, tol=0.0, max_iter=50)
    assert r["iters"] == 1 and r["converged"]
    assert np.array_equal(r["centers"], C) and r["J"] == 16.0


def pin_stop_rule_and_count(o):
    """Stop when shift <= tol; the detecting iteration is counted (Table 1)."""
    X = np.array([[0.0], [4.0], [10.0]], dtype=np.float32)
    C = np.array([[0.0], [10.0]])
    r = o.lloyd_stage(X, C, tol=2.0, max_iter=10)          # shift of step 1 is exactly 2
    assert r["iters"] == 1 and r["converged"], r
    r = o.lloyd_stage(X, C, tol=1.999, max_iter=10)
    assert r["iters"] == 2 and r["converged"] and r["traj_shift"].tolist() == [2.0, 0.0], r
    r = o.lloyd_stage(X, C, tol=1.0, max_iter=1)
    assert r["iters"] == 1 and not r["converged"]
    assert r["labels"].tolist() == [0, 0, 1] and r["centers"].ravel().tolist() == [2.0, 10.0]


def pin_returned_labels_are_last_assignment(o):
    """The returned labels are those of the last assignment, made against the
    centers before that iteration's update (here the point at 4.8 would move
    to the other cluster if re-assigned against the updated centers)."""
    X = np.array([[-10.0], [4.8], [10.0]], dtype=np.float32)
    C = np.array([[0.0], [10.0]])
    r = o.lloyd_stage(X, C, tol=0.0, max_iter=1)
    assert r["labels"].tolist() == [0, 0, 1], r["labels"]
    assert _rel(r["J"], _np_cost(X, C, np.array([0, 0, 1]))) < 1e-15
    assert np.allclose(r["centers"].ravel(), [(-10.0 + np.float32(4.8)) / 2, 10.0])


def _partition_cost(X64, L, k):
    """Sum over clusters of squared distances to the cluster mean (direct form)."""
    cost = 0.0
    for j in range(k):
        mem = X64[L == j]
        if len(mem):
            cost += float(((mem - mem.mean(0)) ** 2).sum())
    return cost


def pin_global_optimum(o):
    """Converged J >= the optimum over all k^n labelings (n = 10, k = 3);
    equal when the components are separated.  The labelings are scored in one
    vectorised pass (sum of squares minus |sum|^2 / count per cluster) and the
    best one is rescored in the direct mean-centred form."""
    rng = np.random.default_rng(7)
    n, k = 10, 3
    labelings = np.array(list(itertools.product(range(k), repeat=n)), dtype=np.int8)
    for trial in range(5):
        sep = 40.0 if trial < 3 else 1.0
        means = rng.uniform(-1, 1, size=(k, 2)) * sep
        X = (means[np.arange(n) % k] + rng.normal(size=(n, 2))).astype(np.float32)
        X64 = X.astype(np.float64)
        sq = (X64 ** 2).sum(1)
        total = np.zeros(len(labelings))
        for j in range(k):
            m = (labelings == j).astype(np.float64)
            cnt = m.sum(1)
            s = m @ X64
            total += m @ sq - np.where(cnt > 0, (s ** 2).sum(1) / np.maximum(cnt, 1), 0.0)
        order = np.argsort(total)[:64]                     # rescore the best few exactly
        best = min(_partition_cost(X64, labelings[i], k) for i in order)
        brute = _partition_cost(X64, np.arange(n) % k, k)   # the planted labeling is a candidate
        assert best <= brute * (1 + 1e-12) + 1e-12
        C0 = X64[[0, 1, 2]]                               # one point of each component
        r = o.lloyd_stage(X, C0, tol=0.0, max_iter=100)
        assert r["J"] >= best * (1 - 1e-12) - 1e-12
        if sep > 10:
            assert _rel(r["J"], best) < 1e-10, (r["J"], best)


# ------------------------------------------------------------------ two stages

def pin_planted_recovery(o):
    """Well separated planted Gaussians are recovered exactly (up to a
    permutation) when the random init draws one point per component."""
    rng = np.random.default_rng(8)
    found = 0
    for seed in range(40):
        k, d, n = 4, 3, 2000
        means = np.array([[0, 0, 0], [30, 0, 0], [0, 30, 0], [0, 0, 30]], dtype=np.float64)
        comp = rng.integers(0, k, n)
        X = (means[comp] + 0.5 * rng.normal(size=(n, d))).astype(np.float32)
        sub, pos = o.sample(n, k, 0.1, seed)
        if len(set(comp[sub[pos]].tolist())) < k:
            continue
        r = o.fit(X, k, 0.1, seed, tol=1e-9, max_iter=100)
        perm = {}
        for c, lab in zip(comp, r["labels"]):
            perm.setdefault(int(lab), int(c))
            assert perm[int(lab)] == int(c)
        for lab, c in perm.items():
            assert np.linalg.norm(r["centers"][lab] - means[c]) < 0.2
        found += 1
        if found == 3:
            break
    assert found == 3


def pin_theorem_full_subset(o):
    """Section 4.1 Theorem: with f = 100% the fast stage is normal k-means, so
    the slow stage starts at its fixed point: one iteration, no movement."""
    X, _ = _random_instance(30, n=800, d=2, k=4)
    r = o.fit(X, 4, 1.0, 11, tol=0.0, max_iter=300)
    assert r["subset_size"] == 800 and r["converged_fast"]
    assert r["iters_slow"] == 1 and r["traj_shift_slow"].tolist() == [0.0]
    assert np.array_equal(r["centers"], r["fast_centers"])


def pin_stage_handoff(o):
    """Section 5: the slow stage's first centers are the fast stage's last."""
    X, _ = _random_instance(31, n=3000, d=3, k=5)
    r = o.fit(X, 5, 0.1, 3, tol=1e-8, max_iter=100, tol_fast=1e-3)
    D = _np_sqdist(X, r["fast_centers"])
    assert _rel(r["traj_J_slow"][0], float(D.min(1).sum())) < 1e-11
    sub, pos = o.sample(3000, 5, 0.1, 3)
    init = X[sub[pos]].astype(np.float64)
    Dsub = _np_sqdist(X[sub], init)
    assert _rel(r["traj_J_fast"][0], float(Dsub.min(1).sum())) < 1e-11


def pin_cost_model(o):
    """Section 3: distance evaluations = K Q_f N_f + K Q_s N."""
    X, _ = _random_instance(32, n=1000, d=2, k=4)
    r = o.fit(X, 4, 0.1, 5, tol=1e-6, max_iter=100)
    assert r["distance_evals"] == 4 * (r["iters_fast"] * 100 + r["iters_slow"] * 1000)


def pin_final_outputs_consistent(o):
    """Returned labels are the last assignment (against the pre-update
    centers) and J is that assignment's cost."""
    X, _ = _random_instance(33, n=900, d=2, k=3)
    r = o.fit(X, 3, 0.2, 9, tol=1e-4, max_iter=4)
    assert _rel(r["J"], r["traj_J_slow"][-1]) == 0.0
    lab = r["labels"]
    for j in range(3):
        mem = X[lab == j].astype(np.float64)
        assert np.allclose(r["centers"][j], mem.mean(0), rtol=1e-13, atol=1e-13)


ALL_PINS = [v for k_, v in sorted(globals().items()) if k_.startswith("pin_")]
