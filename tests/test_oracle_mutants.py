"""Plant plausible mistakes in copies of the oracle and check the pins catch them.

Each mutant is oracle.c with one textual change (a dropped byte, a wrong index,
an off-by-one range check, a dropped rank or run start in the three-phase
statement, a reversed tie order,
a shortened key, a neighbouring dimension row, a reversed join order), compiled
into a temporary library and swapped in; at least one pin must then fail.
"""
import ctypes
import os
import subprocess

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    "dropped_byte": ("memcpy(dst + i * rec, src + (uint64_t)rids[i] * rec, rec);",
                     "memcpy(dst + i * rec, src + (uint64_t)rids[i] * rec, rec - (rec > 1));"),
    "reversed_index": ("memcpy(dst + i * rec, src + (uint64_t)rids[i] * rec, rec);",
                       "memcpy(dst + i * rec, src + (uint64_t)rids[n - 1 - i] * rec, rec);"),
    "range_off_by_one": ("if (rids[i] < 0 || (uint64_t)rids[i] >= n_src) return OR_ERANGE;\n  for (uint64_t i = 0; i < n; ++i)\n    memcpy",
                         "if (rids[i] < 0 || (uint64_t)rids[i] > n_src) return OR_ERANGE;\n  for (uint64_t i = 0; i < n; ++i)\n    memcpy"),
    "gather_rank_dropped": ("      if ((uint64_t)rids[m] / L == j) rank++;", "      ;"),
    "probe_wrong_entry": ("memcpy(internal + k * rec, src + (uint64_t)rid_runs[k] * rec, rec);",
                          "memcpy(internal + k * rec, src + (uint64_t)rid_runs[n - 1 - k] * rec, rec);"),
    "run_start_off_by_one": ("for (uint64_t m = 0; m < j; ++m) start += run_sizes[m];",
                             "for (uint64_t m = 0; m + 1 < j; ++m) start += run_sizes[m];"),
    "tie_order_reversed": ("return (ra > rb) - (ra < rb);", "return (ra < rb) - (ra > rb);"),
    "short_key": ("int c = memcmp(a, b, g_key_bytes);", "int c = memcmp(a, b, g_key_bytes - 1);"),
    "neighbour_dim_row": ("memcpy(out + i * w + fact_bytes, dim + (uint64_t)fk * dim_bytes, dim_bytes);",
                          "memcpy(out + i * w + fact_bytes, dim + (uint64_t)(fk > 0 ? fk - 1 : 0) * dim_bytes, dim_bytes);"),
    "order_ties_reversed": ("for (uint64_t i = 0; i < n_fact; ++i) order[",
                            "for (uint64_t i = n_fact; i-- > 0;) order["),
    "join_order_reversed": ("if (x->fk != y->fk) return (x->fk > y->fk) - (x->fk < y->fk);",
                            "if (x->fk != y->fk) return (x->fk < y->fk) - (x->fk > y->fk);"),
}

PIN_CALLS = [
    lambda: pins.test_retrieve_all_permutations_small(1),
    lambda: pins.test_retrieve_random_permutation_by_scatter(100),
    lambda: pins.test_retrieve_duplicates_decode(100),
    lambda: pins.test_retrieve_permutation_multiset_and_exactly_once(),
    lambda: pins.test_retrieve_out_of_range_writes_nothing(50),
    lambda: pins.test_worked_example_section_2_2(),
    lambda: pins.test_three_phases_equal_definition(4),
    lambda: pins.test_sort_keyptr_sorted_permutation(100),
    lambda: pins.test_sort_keyptr_matches_selection_sort(),
    lambda: pins.test_sort_keyptr_every_key_byte_counts(),
    lambda: pins.test_sort_records_sorted_file(),
    lambda: pins.test_fk_join_move_equals_nested(50, 400),
    lambda: pins.test_fk_join_sorted_order(50, 400),
    lambda: pins.test_fk_join_order_is_the_sorted_join(50, 400),
]


def _failures():
    failed = 0
    for call in PIN_CALLS:
        try:
            call()
        except (AssertionError, oracle.OracleRangeError, ValueError, pytest.fail.Exception):
            failed += 1
    return failed


def test_pins_pass_on_the_real_oracle():
    assert _failures() == 0


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) >= 1, f"mutation site for {name} not found"
    path = tmp_path / f"{name}.c"
    path.write_text(text.replace(old, new, 1))
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", str(path), "-o", str(so)],
                   check=True, capture_output=True)
    prev = oracle.use_library(oracle.configure(ctypes.CDLL(str(so))))
    try:
        assert _failures() >= 1, f"no pin caught mutant {name}"
    finally:
        oracle.use_library(prev)
