"""Plant a mistake in a copy of the oracle and check that a pin catches it.

This shows the pins have teeth: a dropped term, a wrong sign or index, an
off-by-one in the stop rule or in the sampling stream each fail at least one
pin.  The mutated copies are compiled to temporary files; the real oracle
source is never modified."""
import pytest

import oracle
from tests import oracle_pins

MUTATIONS = [
    ("tie_rule", "if (v < best) { best = v; arg = j; }", "if (v <= best) { best = v; arg = j; }"),
    ("dropped_accumulation", "acc = fma(a, a, acc);", "acc = fma(a, a, 0.0);"),
    ("wrong_sign", "double a = (double)x[t] - c[t];", "double a = (double)x[t] + c[t];"),
    ("empty_goes_to_origin", "for (int32_t t = 0; t < d; ++t) cn[t] = c[t];",
     "for (int32_t t = 0; t < d; ++t) cn[t] = 0.0;"),
    ("mean_off_by_one", "/ (double)cnt[j];", "/ (double)(cnt[j] + 1);"),
    ("transposed_sum_index", "cn[t] = (sum[(size_t)j * d + t] + cmp[(size_t)j * d + t])",
     "cn[t] = (sum[(size_t)t * d + j] + cmp[(size_t)t * d + j])"),
    ("strict_stop", "if (shift <= tol) { conv = 1; break; }", "if (shift < tol) { conv = 1; break; }"),
    ("shift_summed", "if (mv > shift) shift = mv;", "shift += mv;"),
    ("stream_offset", "return sm64_mix(seed + (i + 1) * SM64_GAMMA);",
     "return sm64_mix(seed + i * SM64_GAMMA);"),
    ("mix_shift", "z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;",
     "z = (z ^ (z >> 29)) * 0x94D049BB133111EBULL;"),
    ("subset_floor", "double want = ceil(f * (double)n);", "double want = floor(f * (double)n);"),
    ("init_from_full_set", "pos[p].key = oracle_splitmix64_at(seed, (uint64_t)(n + p));",
     "pos[p].key = oracle_splitmix64_at(seed, (uint64_t)p);"),
    ("J_not_compensated_dropped", "for (int64_t i = 0; i < n; ++i) neumaier_add(&js, &jc, dmin[i]);",
     "for (int64_t i = 1; i < n; ++i) neumaier_add(&js, &jc, dmin[i]);"),
    ("slow_stage_restarts_from_init", "if (fast_centers_out)\n        memcpy(fast_centers_out,",
     "for (int32_t j = 0; j < k; ++j)\n        for (int32_t t = 0; t < d; ++t)\n"
     "            centers_out[(size_t)j * d + t] = (double)Xs[(size_t)pos[j] * d + t];\n"
     "    if (fast_centers_out)\n        memcpy(fast_centers_out,"),
    ("shift_without_root", "        mv = sqrt(mv);\n", "\n"),
    ("subset_unsorted", "    qsort(subset_out, (size_t)m, sizeof(int64_t), cmp_i64);\n", "\n"),
    ("empty_not_counted", "            ++empty;\n", "\n"),
    ("labels_after_update", "memcpy(C, nxt, (size_t)k * (size_t)d * sizeof(double));\n        if (shift <= tol)",
     "memcpy(C, nxt, (size_t)k * (size_t)d * sizeof(double));\n"
     "        oracle_assign(X, n, d, k, C, labels, NULL, nthreads);\n        if (shift <= tol)"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(name, old, new):
    src = oracle.source_text()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    variant = oracle.build_variant(src.replace(old, new), name)
    failed = []
    for pin in oracle_pins.ALL_PINS:
        try:
            pin(variant)
        except (AssertionError, ValueError):
            failed.append(pin.__name__)
    assert failed, f"no pin caught the planted mistake {name}"
