"""Plant one mistake at a time in a copy of the oracle's C source and check
that the pins catch every one (no GPU).

Each mutant is compiled into a temporary library and checked in a child
process, so that a mutant which corrupts memory cannot take the test run down
with it.
"""
import multiprocessing as mp
import os
import sys

import pytest

import oracle

# (name, original text, planted text): each a mistake someone could make.
MUTANTS = [
    ("bit_order_in_word", "bitmap[x / 32u] | (1u << (x % 32u))",
     "bitmap[x / 32u] | (1u << (31u - x % 32u))"),
    ("emit_bit_reversed", "out[k] = (uint32_t)(w * 32u + b);",
     "out[k] = (uint32_t)(w * 32u + (31u - b));"),
    ("emit_drops_bit_31", "for (unsigned b = 0; b < 32u; ++b)", "for (unsigned b = 0; b < 31u; ++b)"),
    ("range_bound_in_32_bits", "uint64_t M = (uint64_t)max_value + 1u;",
     "uint64_t M = (uint32_t)(max_value + 1u);"),
    ("range_check_strict", "if (x > max_value) { out_of_range = 1; continue; }",
     "if (x >= max_value) { out_of_range = 1; continue; }"),
    ("duplicate_test_wrong", "if (k < n) return ORACLE_DUPLICATE;", "if (k > n) return ORACLE_DUPLICATE;"),
    ("word_index_shift", "out[k] = (uint32_t)(w * 32u + b);", "out[k] = (uint32_t)(w * 31u + b);"),
    ("and_instead_of_or", "bitmap[x / 32u] | (1u << (x % 32u))", "bitmap[x / 32u] & (1u << (x % 32u))"),
    ("paper_ones_first", "if (a[i] & (1u << k)) { ones[n1] = a[i]; ++n1; }",
     "if (!(a[i] & (1u << k))) { ones[n1] = a[i]; ++n1; }"),
    ("paper_one_pass_short", "for (int k = 0; k < nbits; ++k) {", "for (int k = 0; k + 1 < nbits; ++k) {"),
    ("paper_not_stable", "for (uint64_t i = 0; i < n1; ++i) a[n0 + i] = ones[i];",
     "for (uint64_t i = 0; i < n1; ++i) a[n0 + i] = ones[n1 - 1 - i];"),
    ("paper_negatives_last", "for (uint64_t i = 0; i < nm; ++i) a[i] = (int32_t)neg[i];\n        for (uint64_t i = 0; i < np; ++i) a[nm + i] = (int32_t)pos[i];",
     "for (uint64_t i = 0; i < np; ++i) a[i] = (int32_t)pos[i];\n        for (uint64_t i = 0; i < nm; ++i) a[np + i] = (int32_t)neg[i];"),
    ("bitmap_words_floor", "uint64_t words = (M + 31u) / 32u;", "uint64_t words = M / 32u;"),
    ("status_precedence_swapped", "if (out_of_range) return ORACLE_KEY_RANGE;\n    if (k < n) return ORACLE_DUPLICATE;",
     "if (k < n) return ORACLE_DUPLICATE;\n    if (out_of_range) return ORACLE_KEY_RANGE;"),
    ("paper_split_msb_first", "if (a[i] & (1u << k)) { ones[n1] = a[i]; ++n1; }",
     "if (a[i] & (1u << (nbits - 1 - k))) { ones[n1] = a[i]; ++n1; }"),
    ("i32_shift_back_dropped", "out[i] = (int32_t)((int64_t)((uint32_t *)out)[i] + (int64_t)min_value);",
     "out[i] = (int32_t)((int64_t)((uint32_t *)out)[i]);"),
    ("i32_below_clamped_into_range", "d = (int64_t)max_value - (int64_t)min_value + 1; }", "d = 0; }"),
    ("i32_offset_wraps_32_bits", "int64_t d = (int64_t)keys[i] - (int64_t)min_value;",
     "int64_t d = (int64_t)(int32_t)((uint32_t)keys[i] - (uint32_t)min_value);"),
    ("u64_emit_truncated", "out[k] = w * 32u + b;", "out[k] = (uint32_t)(w * 32u + b);"),
    ("u64_range_check_32_bits", "uint64_t x = keys[i];", "uint64_t x = (uint32_t)keys[i];"),
    ("bin_repl_lsb_first", "out[15 - d] = ((bits >> d) & 1u) ? '1' : '0';",
     "out[d] = ((bits >> d) & 1u) ? '1' : '0';"),
]


def _run_pins(lib_path, q):
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import oracle as _oracle
    import oracle_pins
    o = _oracle.Oracle(_oracle.bind(lib_path))
    failed = []
    for check in oracle_pins.ALL_CHECKS:
        try:
            check(o)
        except AssertionError:
            failed.append(check.__name__)
        except Exception as e:  # a crash-free error also counts as detection
            failed.append(f"{check.__name__}:{type(e).__name__}")
    q.put(failed)


@pytest.mark.parametrize("name,orig,planted", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, name, orig, planted):
    src = open(oracle.SOURCE).read()
    assert src.count(orig) >= 1, f"mutation anchor for {name} not found in oracle.c"
    mutant = src.replace(orig, planted)
    path = tmp_path / f"{name}.c"
    path.write_text(mutant)
    lib = oracle.compile_library(str(path), str(tmp_path / f"lib{name}.so"))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_run_pins, args=(lib, q))
    p.start()
    p.join(300)
    if p.is_alive():
        p.kill()
        p.join()
        return  # a hang is detection too
    if p.exitcode != 0:
        return  # crashed: detected
    failed = q.get(timeout=10)
    assert failed, f"no pin caught the planted mistake {name}"
