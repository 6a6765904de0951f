"""Plant plausible mistakes in copies of the oracle (on the CPU) and check
that the pins of test_oracle_pins.py catch every one: a dropped term, a wrong
comparison or index, a wrong constant, a transposed operand."""
import os
import subprocess

import numpy as np
import pytest

from oracle import wrs_oracle as O
from tests import test_oracle_pins as P
from tests import test_oracle_psaplus as PP

SRC = os.path.join(os.path.dirname(O.__file__), "wrs_oracle.c")

MUTANTS = {
    # Alg. 2: tie goes the wrong way (pack a light bucket when w == capacity)
    "sweep_tie": ("        if (w > in.Q) { /* pack a light bucket */", "        if (w >= in.Q) { /* pack a light bucket */"),
    # Alg. 2: residual update drops the light item's weight
    "sweep_drop_term": ("            w = (w + nq(&in, i)) - in.Q;\n            i = next_light", "            w = w - in.Q + 1;\n            i = next_light"),
    # Alg. 2: light bucket takes the next heavy as alias instead of the current one
    "sweep_alias_index": ("            put(bw, al, i, nq(&in, i), j);\n            w = (w + nq(&in, i)) - in.Q;",
                          "            put(bw, al, i, nq(&in, i), next_heavy(&in, j + 1) < n ? next_heavy(&in, j + 1) : j);\n"
                          "            w = (w + nq(&in, i)) - in.Q;"),
    # classification: light iff n*q < Q (strict)
    "light_strict": ("static int is_light(const wo_in *in, uint64_t k) { return nq(in, k) <= in->Q; }",
                     "static int is_light(const wo_in *in, uint64_t k) { return nq(in, k) < in->Q; }"),
    # Alg. 3 split: strict comparison picks the smaller j
    "split_strict": ("    return (u128)s->in->n * sigma <= (u128)np * s->in->Q;", "    return (u128)s->in->n * sigma < (u128)np * s->in->Q;"),
    # Alg. 3 split: spill uses the wrong heavy (h[j-1])
    "split_spill_index": ("ld128(s->in->q + 2 * (uint64_t)s->h[j]))", "ld128(s->in->q + 2 * (uint64_t)s->h[j > 0 ? j - 1 : 0]))"),
    # normalisation: beta ignores the trailing zeros of the mantissa
    "beta_no_ctz": ("            if (m && e + ctz32(m) < beta) beta = e + ctz32(m);", "            if (m && e < beta) beta = e;"),
    # Alg. 1: drops b[i].w in the cancellation-avoiding update
    "vose_drop_term": ("(ld128(bw + 2 * (uint64_t)j) + ld128(bw + 2 * (uint64_t)i)) - in.Q", "ld128(bw + 2 * (uint64_t)j) - in.Q"),
    # Philox: wrong Weyl constant
    "philox_weyl": ("k0 += 0x9E3779B9u;", "k0 += 0x9E3779B8u;"),
    # Philox: words 1 and 3 swapped in the round
    "philox_swap": ("n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;", "n0 = (uint32_t)(p1 >> 32) ^ c3 ^ k0;"),
    # query: heads on <= (coin comparison off by one)
    "query_le": ("        heads = (uint64_t)(((u128)v * Qp) >> 64) < thr[r];", "        heads = (uint64_t)(((u128)v * Qp) >> 64) <= thr[r];"),
    # query: bucket from the high word (operands transposed)
    "query_words": ("        r = (uint64_t)(((u128)u * n) >> 64);\n        heads", "        r = (uint64_t)(((u128)v * n) >> 64);\n        heads"),
    # encoding: thresholds not shifted like the denominator
    "encode_shift": ("    for (b = 0; b < n; ++b) thr[b] = (uint64_t)(ld128(bw + 2 * b) >> s);", "    for (b = 0; b < n; ++b) thr[b] = (uint64_t)(ld128(bw + 2 * b) >> (s ? s - 1 : 0));"),
}

PINS = [
    P.test_philox_known_answers,
    P.test_quantize_f32_matches_exact_rationals,
    P.test_hand_examples,
    P.test_exhaustive_small_sweep_psa_vose_are_alias_tables,
    P.test_exact_query_distribution_equals_definition,
    P.test_random_tables_invariants_and_psa_identity,
    P.test_psa_splits_satisfy_paper_condition,
    P.test_one_heavy_among_equal_lights_closed_form,
    P.test_sampler_n1_and_full_buckets_reduce_to_multiply_shift,
    P.test_sampler_tails_take_the_alias,
    P.test_sampler_coin_with_small_denominator,
]


# PSA+ (Sec. 4.2 "Performance Optimization in Practice"), caught by the PSA+ pins
PP_MUTANTS = {
    # the heavy item current at the stop is handed on whole instead of with its residual
    "pp_residual_dropped": ("            st128(lv + 2 * m, k == cur ? w : nq(&in, k));",
                            "            st128(lv + 2 * m, nq(&in, k));"),
    # a heavy item at or under capacity with no next heavy in the tile is finished in place
    "pp_finish_in_place": ("                    if (jn >= t1) break;\n                    put(bw, al, j, w, jn);",
                           "                    if (jn >= t1) { put(bw, al, j, w, j); done[j - t0] = 1; break; }\n"
                           "                    put(bw, al, j, w, jn);"),
    # a packed heavy item's overflow goes to itself instead of the next heavy item
    "pp_heavy_alias_self": ("                    put(bw, al, j, w, jn);\n                    done[j - t0] = 1;",
                            "                    put(bw, al, j, w, j);\n                    done[j - t0] = 1;"),
}


def _pp_alias_tables():
    for name, w in PP.INPUTS[:4]:
        for T in (3, 64):
            PP.test_every_tile_size_gives_an_alias_table(name, w, T)


PP_PINS = [PP.test_hand_examples, PP.test_exhaustive_small, _pp_alias_tables]


def _run_mutant(old, new, pins, tmp_path):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation site not found exactly once"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    so = str(tmp_path / "libmutant.so")
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", so, str(mutated), "-lm"])
    caught = []
    with O.use_library(so):
        for pin in pins:
            try:
                pin()
            except Exception:  # a failed assertion or an oracle error both count as caught
                caught.append(pin.__name__)
    return caught


@pytest.mark.parametrize("name", sorted(PP_MUTANTS))
def test_every_planted_psa_plus_mistake_is_caught(name, tmp_path):
    old, new = PP_MUTANTS[name]
    assert _run_mutant(old, new, PP_PINS, tmp_path), f"mutant {name} passed every PSA+ pin"


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_every_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    so = str(tmp_path / "libmutant.so")
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", so, str(mutated)])
    caught = []
    with O.use_library(so):
        for pin in PINS:
            try:
                pin()
            except Exception:  # a failed assertion or an oracle error both count as caught
                caught.append(pin.__name__)
    assert caught, f"mutant {name} passed every pin"
