"""Mutation check of the oracle pins: each case compiles a copy of sf_oracle.c with one
plausible mistake planted (a dropped term, a wrong comparison, index or operand) and asserts
that at least one pin of tests/test_oracle_pins.py fails on it.  CPU only."""
import os
import subprocess

import pytest

import oracle
import tests.test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "sf_oracle.c")
W_MAX_PIN = pins.W_MAX

# (name, exact text in sf_oracle.c, replacement)
MUTATIONS = [
    ("insert-condition-le", "if (m < Bmin) {", "if (m <= Bmin) {"),
    ("insert-one-row-only", "if (*a == m) *a = m + 1u;", "if (*a == m) { *a = m + 1u; break; }"),
    ("insert-all-rows", "if (*a == m) *a = m + 1u;", "*a = *a + 1u;"),
    ("bmin-before-increment", "*c += 1u;\n            }\n            for (uint32_t i = 0; i < d; i++) {\n                uint32_t v = *fat_at(B, w, z, i, ht[i], ft[i]);\n                if (v < Bmin) Bmin = v;",
     "(void)c;\n            }\n            for (uint32_t i = 0; i < d; i++) {\n                uint32_t v = *fat_at(B, w, z, i, ht[i], ft[i]);\n                *fat_at(B, w, z, i, ht[i], ft[i]) = v + 1u; v += 0u; if (v < Bmin) Bmin = v;"),
    ("delete-sets-unconditionally", "if (after != before && *a > after) *a = after;", "if (after != before) *a = after;"),
    ("delete-clamp-to-slot", "uint32_t mx = bucket_max(B, w, z, i, ht[i]);", "uint32_t mx = *fat_at(B, w, z, i, ht[i], ft[i]);"),
    ("chunk-drops-count", "uint64_t mc = (uint64_t)m + c_e;", "uint64_t mc = (uint64_t)m + 1u;"),
    ("chunk-m-from-live-slim", "uint32_t a0 = *slim_at(A0, w, i, h[t * d + i]);", "uint32_t a0 = *slim_at(A, w, i, h[t * d + i]) + (c_e > 1u);"),
    ("chunk-F-is-max", "if (b1 < F) F = b1;", "if (F == UINT32_MAX || b1 > F) F = b1;"),
    ("chunk-clamp-uses-min", "M[(t - c0) * d + i] = bucket_max(B, w, z, i, h[t * d + i]);",
     "M[(t - c0) * d + i] = *fat_at(B, w, z, i, h[t * d + i], f[t * d + i]);"),
    ("hash-h-from-low-bits", "*h = (uint32_t)((hi * (uint64_t)w) >> 32);", "*h = (uint32_t)((lo * (uint64_t)w) >> 32);"),
    ("hash-drops-second-word", "H = osf_mix64(H ^ x1);", "H = osf_mix64(H);"),
    ("hash-reduce-mod", "*h = (uint32_t)((hi * (uint64_t)w) >> 32);", "*h = (uint32_t)(hi % w);"),
    ("hash-f-reduce-mod", "*f = (uint32_t)((lo * (uint64_t)z) >> 32);", "*f = (uint32_t)(lo % z);"),
    ("hash-swaps-words", "H = osf_mix64(H ^ x1);", "H = osf_mix64(osf_mix64(x1 ^ row_seed) ^ x0);"),
    ("hash-tail-big-endian", "uint64_t x1 = load_le(key + 8, key_bytes - 8);",
     "uint64_t x1 = 0; for (uint32_t b = 8; b < key_bytes; b++) x1 = (x1 << 8) | key[b];"),
    ("hash-seed-added-not-xored", "uint64_t H = osf_mix64(x0 ^ row_seed);", "uint64_t H = osf_mix64(x0 + row_seed);"),
    ("mix-wrong-shift", "z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;", "z = (z ^ (z >> 28)) * 0x94D049BB133111EBULL;"),
    ("query-max", "if (v < m) m = v;\n        }\n        out[t] = m;", "if (m == UINT32_MAX || v > m) m = v;\n        }\n        out[t] = m;"),
    ("fat-transposed-index", "return &B[((uint64_t)i * w + j) * z + k];", "return &B[((uint64_t)i * z + k) * w + j];"),
    ("sf4-decrement-at-equality", "if ((uint64_t)*a > bucket_sum(B, w, z, i, ht[i])) *a -= 1u;",
     "if ((uint64_t)*a >= bucket_sum(B, w, z, i, ht[i])) *a -= 1u;"),
    ("sf4-bound-is-max", "if ((uint64_t)*a > bucket_sum(B, w, z, i, ht[i])) *a -= 1u;",
     "if (*a > bucket_max(B, w, z, i, ht[i])) *a -= 1u;"),
    ("sf4-sum-drops-a-slot", "for (uint32_t k = 0; k < z; k++) s += *fat_at(B, w, z, i, j, k);",
     "for (uint32_t k = 1; k < z; k++) s += *fat_at(B, w, z, i, j, k);"),
    ("sf4-chunk-bound-is-max", "uint64_t sb = bucket_sum(B, w, z, i, h[t * d + i]);",
     "uint64_t sb = bucket_max(B, w, z, i, h[t * d + i]);"),
    ("sf4-chunk-clamps-to-zero", "if (*a > mb) *a -= 1u;", "if (*a > mb) *a = 0u;"),
]


def _pins_pass() -> bool:
    checks = [
        pins.test_splitmix64_published_vectors,
        pins.test_mix64_inverts_with_the_published_constants,
        lambda: pins.test_power_of_two_reduction_takes_the_top_bits(4096, 16),
        pins.test_13_byte_keys_use_all_bytes,
        lambda: pins.test_multiply_shift_partitions_the_32_bit_range_in_order(1000),
        lambda: pins.test_multiply_shift_partitions_the_32_bit_range_in_order(W_MAX_PIN),
        lambda: pins.test_short_keys_hash_as_one_mix_of_the_key_xor_the_row_seed(4),
        lambda: pins.test_long_keys_fold_the_second_word_in_after_the_first_mix(13),
        lambda: pins.test_worked_example_sec32("seq"),
        lambda: pins.test_worked_example_sec32("chunk1"),
        lambda: pins.test_brute_force_tiny_streams_against_literal_transcription(
            ([[0, 0], [0, 1], [1, 1]], [[0, 1], [1, 0], [0, 0]])),
        lambda: pins.test_chunk_size_one_is_sequential(0),
        lambda: pins.test_no_underestimation_and_slim_below_bucket_max(64),
        lambda: pins.test_fat_is_the_cm_histogram_and_rows_sum_to_the_net_count(13),
        lambda: pins.test_theorem_slim_counter_is_max_frequency_with_error_free_fat(31),
        lambda: pins.test_exact_counts_without_collisions(64),
        lambda: pins.test_chunk_equals_its_order_free_closed_form(0),
        pins.test_zero_length_and_edge_shapes,
        pins.test_chunk_hand_derived_single_counter,
        pins.test_sf4_hand_derived_bucket,
        lambda: pins.test_sf4_chunk_size_one_is_sequential(0),
        lambda: pins.test_sf4_slim_below_bucket_sum_and_no_underestimation(7),
        lambda: pins.test_sf4_decrement_is_a_clamp_to_the_bucket_sum(13),
    ]
    for c in checks:
        try:
            c()
        except (AssertionError, ValueError, IndexError):
            return False
    return True


def test_unmutated_oracle_passes_the_pin_subset():
    assert _pins_pass()


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(name, old, new, tmp_path):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mutant = src.replace(old, new)
    c = tmp_path / "mutant.c"
    so = tmp_path / "libmutant.so"
    c.write_text(mutant)
    subprocess.check_call(["gcc", "-O1", "-std=c99", "-shared", "-fPIC", "-o", str(so), str(c)])
    with oracle.use_library(str(so)):
        caught = not _pins_pass()
    assert caught, f"no pin catches the planted mistake '{name}'"
