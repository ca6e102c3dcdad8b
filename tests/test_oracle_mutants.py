"""Planted mistakes in the oracle, on the CPU.

Each mutant is the oracle's C source with one plausible error -- an
off-by-one, a wrong comparison, an inverted bit, a dropped term -- compiled
into a scratch directory and loaded as a separate copy of the oracle module.
The pin named beside it must reject the mutant.  This shows that the pins, and
not only the oracle's agreement with itself, fix each part of the
computation.  (The hash functions' values are readings the paper leaves open
and are not pinned here; the independent CUDA path checks them.)
"""
from __future__ import annotations

import importlib.util
import os
from fractions import Fraction

import pytest

import test_oracle_build as build_pins
import test_oracle_pins as pins
import test_oracle_rf as rf_pins

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_DIR = os.path.join(ROOT, "oracle")

# (what the mistake is, text in shk_oracle.c, replacement, the pin that must fail)
MUTANTS = [
    ("mixer: last xor-shift by 32",
     "return z ^ (z >> 31);", "return z ^ (z >> 32);",
     lambda o: pins.test_mixer_matches_published_splitmix64(o)),
    ("bucket: scaled by B - 1",
     "((u128)hi * B) >> 64", "((u128)hi * (B - 1)) >> 64",
     lambda o: build_pins.test_bucket_occupancy_chi_square(o)),
    ("in-bucket order: lo compared before hi",
     "  if (x[1] != y[1]) return x[1] < y[1] ? -1 : 1; /* hi first */\n  if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;",
     "  if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;\n  if (x[1] != y[1]) return x[1] < y[1] ? -1 : 1;",
     lambda o: build_pins.test_format_sections_decode(o)),
    ("partition: a child's keys in reverse order",
     "    for (uint32_t i = 0; i < m; i++)\n      if (orc_split_child(lo[i], s, m, unit, fan) == j) {",
     "    for (uint32_t i = m; i-- > 0;)\n      if (orc_split_child(lo[i], s, m, unit, fan) == j) {",
     lambda o: build_pins.test_leaf_order_is_the_stable_partition(o, 24)),
    ("tree shape: one part too many",
     "*fanout = (m + n - 1) / n;", "*fanout = (m + n) / n;",
     lambda o: pins.test_tree_shape_example_n64(o)),
    ("split seed: a count one short accepted",
     "if (cnt[j] != part_size(m, unit, fan, j)) ok = 0;",
     "if (cnt[j] + 1 < part_size(m, unit, fan, j)) ok = 0;",
     lambda o: pins.test_split_seed_is_minimum(o)),
    ("leaf hash: both cells may coincide",
     "*h1 = t + (t >= u ? 1u : 0u);", "*h1 = t + (t > u ? 1u : 0u);",
     lambda o: pins.test_leaf_seed_m2_is_zero_and_hash_avoids_self_loops(o)),
    ("leaf seed: search starts one seed late",
     "for (uint64_t s = start; s < cap; s++) {", "for (uint64_t s = start + 1; s < cap; s++) {",
     lambda o: pins.test_leaf_seed_m2_is_zero_and_hash_avoids_self_loops(o)),
    ("pseudoforest: a component with as many edges as nodes rejected",
     "if (edges[v] > nodes[v]) return 0;", "if (edges[v] >= nodes[v]) return 0;",
     lambda o: pins.test_pseudoforest_equals_orientability_all_graphs(o, 4, Fraction(53, 72))),
    ("filter: the full mask one cell short",
     "uint64_t full = m == 64 ? ~0ull : ((1ull << m) - 1);",
     "uint64_t full = m == 64 ? ~0ull : ((1ull << (m - 1)) - 1);",
     lambda o: pins.test_filter_exact_coverage_count(o, 4)),
    ("orientation: the second cell tried first",
     "    fixed[i] = 0;\n    if (!bijection_exists(m, h0, h1, fixed)) fixed[i] = 1;",
     "    fixed[i] = 1;\n    if (!bijection_exists(m, h0, h1, fixed)) fixed[i] = 0;",
     lambda o: pins.test_orientation_is_lexicographic_minimum_and_count(o, 6)),
    ("Rice: unary part terminated by a one",
     "return bv_push_bit(bv, 0);", "return bv_push_bit(bv, 1);",
     lambda o: build_pins.test_format_sections_decode(o)),
    ("Rice: one leaf parameter one too large",
     "19, 19, 20, 20, 21", "19, 19, 20, 21, 21",
     lambda o: pins.test_leaf_rice_table_follows_its_closed_form(o)),
    ("Elias-Fano: low-bit width one too large",
     "return 63 - (uint32_t)__builtin_clzll(q);", "return 64 - (uint32_t)__builtin_clzll(q);",
     lambda o: build_pins.test_format_sections_decode(o)),
    ("retrieval: free columns set to one",
     "      sol[ii] = 0;\n      continue;", "      sol[ii] = 1;\n      continue;",
     lambda o: pins.test_ribbon_canonical_solution(o, 60, 3277, 128)),
    ("retrieval: band start range one slot short",
     "*start = (uint64_t)(((u128)u * (m - (w - 1))) >> 64);", "*start = (uint64_t)(((u128)u * (m - w)) >> 64);",
     lambda o: pins.test_ribbon_row_start_uniform_and_coefficients_balanced(o, 128)),
    ("retrieval: orientation bits stored inverted",
     "    uint8_t b = f[i];", "    uint8_t b = f[i] ^ 1u;",
     lambda o: build_pins.test_build_is_bijection(o, 3000, 8, 100)),
    ("Elias-Fano: low parts taken one bit too high",
     "if (!bv_push_bits(low, v[i], l)) return 0;", "if (!bv_push_bits(low, v[i] >> 1, l)) return 0;",
     lambda o: build_pins.test_format_sections_decode(o)),
    ("query: a set retrieval bit read as the first cell",
     "local = bit ? h1 : h0;", "local = bit ? h0 : h1;",
     lambda o: build_pins.test_build_is_bijection(o, 3000, 8, 100)),
    ("query: skipped subtrees not counted",
     "      offset += p;\n", "\n",
     lambda o: build_pins.test_build_is_bijection(o, 3000, 8, 100)),
    ("rotation fitting: partial-hash period 4",
     "#define RF_PARTIAL_K 8u", "#define RF_PARTIAL_K 4u",
     lambda o: rf_pins.test_candidate_cells_rotation_and_partial_seed(o, 48)),
    ("rotation fitting: value search starts one candidate late",
     "if (v < start) continue;", "if (v <= start) continue;",
     lambda o: rf_pins.test_rf_value_is_the_minimum(o, 3)),
    ("rotation fitting: first cell rotated the other way",
     "*h0 = (uint32_t)((*h0 + r) % m);", "*h0 = (uint32_t)((*h0 + m - r) % m);",
     lambda o: rf_pins.test_candidate_cells_rotation_and_partial_seed(o, 17)),
    ("SipHash: first rotation by 12",
     "v[1] = rotl64(v[1], 13)", "v[1] = rotl64(v[1], 12)",
     lambda o: pins.test_siphash_published_vector(o)),
    ("SipHash: length byte left out of the last block",
     "uint64_t b = (len & 0xFF) << 56;", "uint64_t b = 0;",
     lambda o: pins.test_siphash_published_vector(o)),
    ("SipHash: tail bytes dropped",
     "for (uint64_t t = 0; t < len - 8 * full; t++) b |=", "for (uint64_t t = 0; t < 0; t++) b |=",
     lambda o: pins.test_siphash_published_vector(o)),
    ("string fingerprint: both halves under the same key",
     "hi[i] = orc_siphash24(STR_SALT_B, STR_SALT_A, p, len);", "hi[i] = orc_siphash24(STR_SALT_A, STR_SALT_B, p, len);",
     lambda o: pins.test_string_fingerprint_is_keyed_siphash_and_sensitive(o)),
    ("retrieval row: coefficient bit 0 not forced",
     "uint64_t c0 = orc_mix64(u ^ RET_SALT2) | 1ull;", "uint64_t c0 = orc_mix64(u ^ RET_SALT2);",
     lambda o: pins.test_ribbon_row_start_uniform_and_coefficients_balanced(o, 64)),
    ("retrieval row: band start over half the range",
     "*start = (uint64_t)(((u128)u * (m - (w - 1))) >> 64);", "*start = (uint64_t)(((u128)u * (m - (w - 1))) >> 65);",
     lambda o: pins.test_ribbon_row_start_uniform_and_coefficients_balanced(o, 64)),
    ("retrieval: 128-bit rows keep only their low word",
     "uint64_t c1 = w == 128 ? orc_mix64(u ^ RET_SALT3) : 0;", "uint64_t c1 = 0;",
     lambda o: pins.test_ribbon_row_start_uniform_and_coefficients_balanced(o, 128)),
    ("retrieval: 128-bit band back substitution stops at bit 63",
     "    for (uint32_t j = 1; j < w; j++)\n      if ((rows[ii] >> j) & 1) b ^= sol[ii + j];",
     "    for (uint32_t j = 1; j < 64; j++)\n      if ((rows[ii] >> j) & 1) b ^= sol[ii + j];",
     lambda o: pins.test_ribbon_canonical_solution(o, 300, 3277, 128)),
    ("leaf hash: second cell from bits overlapping the first",
     "uint32_t t = (uint32_t)(((uint64_t)(uint32_t)w * (m - 1)) >> 32);",
     "uint32_t t = (uint32_t)(((uint64_t)(uint32_t)(w >> 8) * (m - 1)) >> 32);",
     lambda o: pins.test_leaf_hash_filter_rate_matches_exact(o, 48, 4000000)),
]


def _load_mutant(tmp_path, old: str, new: str):
    src = open(os.path.join(ORACLE_DIR, "shk_oracle.c")).read()
    assert src.count(old) == 1, old
    c_path = tmp_path / "shk_oracle.c"
    c_path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location(f"oracle_mutant_{tmp_path.name}",
                                                  os.path.join(ORACLE_DIR, "__init__.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._SRC = str(c_path)
    mod._LIB_DIR = str(tmp_path / "_build")
    mod._LIB = str(tmp_path / "_build" / "liboracle.so")
    mod._lib = None
    mod.build()
    return mod


@pytest.mark.parametrize("what,old,new,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_rejects_planted_mistake(tmp_path, orc, what, old, new, pin):
    pin(orc)  # the pin holds for the oracle itself
    mutant = _load_mutant(tmp_path, old, new)
    with pytest.raises(Exception):
        pin(mutant)
