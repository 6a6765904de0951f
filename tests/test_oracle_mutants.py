"""Plant plausible mistakes in copies of the oracle (on the CPU) and check
that the pins of test_oracle_pins.py catch every one: a dropped term, a wrong
comparison or index, a wrong constant, a transposed operand."""
import os
import subprocess

import numpy as np
import pytest

from oracle import wrs_oracle as O
from tests import test_oracle_2lvl as TL
from tests import test_oracle_osnd as OS
from tests import test_oracle_pins as P
from tests import test_oracle_psaplus as PP
from tests import test_oracle_sample_at as SA

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
    # Alg. 3 boundaries: floor(n k / p) instead of ceil(n k / p)
    "psa_boundary_floor": ("        snp[k] = (uint64_t)(((u128)n * k + p - 1) / p); /* ceil(n*k/p) */",
                           "        snp[k] = (uint64_t)(((u128)n * k) / p); /* ceil(n*k/p) */"),
    # Alg. 3 pack: a light bucket names itself instead of the current heavy item
    "psa_pack_light_self": ("                put(bw, al, s.l[i], nq(&in, s.l[i]), j < s.nh ? s.h[j] : s.l[i]);",
                            "                put(bw, al, s.l[i], nq(&in, s.l[i]), s.l[i]);"),
    # Alg. 3 split: spill uses the wrong heavy (h[j-1])
    "split_spill_index": ("ld128(s->in->q + 2 * (uint64_t)s->h[j]))", "ld128(s->in->q + 2 * (uint64_t)s->h[j > 0 ? j - 1 : 0]))"),
    # normalisation: beta ignores the trailing zeros of the mantissa
    "beta_no_ctz": ("            if (m && e + ctz32(m) < beta) beta = e + ctz32(m);", "            if (m && e < beta) beta = e;"),
    # Alg. 1: drops b[i].w in the cancellation-avoiding update
    "vose_drop_term": ("(ld128(bw + 2 * (uint64_t)j) + ld128(bw + 2 * (uint64_t)i)) - in.Q", "ld128(bw + 2 * (uint64_t)j) - in.Q"),
    # Alg. 1: a light bucket names itself instead of the heavy item that fills it
    "vose_alias_self": ("            i = ls[--nl];\n            al[i] = j; set[i] = 1;",
                        "            i = ls[--nl];\n            al[i] = i; set[i] = 1;"),
    # Alg. 1 in binary64: capacity W / (n + 1) instead of W / n
    "vose_f64_capacity": ("    cap = W / (double)n;", "    cap = W / (double)(n + 1);"),
    # Philox: wrong Weyl constant
    "philox_weyl": ("k0 += 0x9E3779B9u;", "k0 += 0x9E3779B8u;"),
    # Philox: words 1 and 3 swapped in the round
    "philox_swap": ("n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;", "n0 = (uint32_t)(p1 >> 32) ^ c3 ^ k0;"),
    # query: heads on <= (coin comparison off by one)
    "query_le": ("        heads = (uint64_t)(((u128)v * Qp) >> 64) < thr[r];", "        heads = (uint64_t)(((u128)v * Qp) >> 64) <= thr[r];"),
    # query: bucket from the high word (operands transposed)
    "query_words": ("        r = (uint64_t)(((u128)u * n) >> 64);\n        heads", "        r = (uint64_t)(((u128)v * n) >> 64);\n        heads"),
    # binary32 decoding: subnormals scaled like normals (2^-150 instead of 2^-149)
    "subnormal_scale": ("    if (ex == 0) { *m = fr; *e = -149; }", "    if (ex == 0) { *m = fr; *e = -150; }"),
    # binary32 decoding: the hidden bit of normal numbers dropped
    "hidden_bit": ("    else { *m = fr | 0x800000u; *e = (int)ex - 150; }", "    else { *m = fr; *e = (int)ex - 150; }"),
    # binary32 decoding: the sign bit ignored (negative weights accepted)
    "sign_ignored": ("    if (bits >> 31) return 1;\n", ""),
    # the running total's range check dropped
    "range_unchecked": ("            if (bitlen128(Q) > WO_Q_BITS) return WO_EOVERFLOW;\n", ""),
    # encoding: thresholds not shifted like the denominator
    "encode_shift": ("    for (b = 0; b < n; ++b) thr[b] = (uint64_t)(ld128(bw + 2 * b) >> s);", "    for (b = 0; b < n; ++b) thr[b] = (uint64_t)(ld128(bw + 2 * b) >> (s ? s - 1 : 0));"),
}

PINS = [
    P.test_philox_known_answers,
    P.test_quantize_f32_matches_exact_rationals,
    P.test_quantize_subnormals_exact,
    P._quantize_rejections,
    P.test_hand_examples,
    P.test_exhaustive_small_sweep_psa_vose_are_alias_tables,
    P.test_exact_query_distribution_equals_definition,
    P.test_random_tables_invariants_and_psa_identity,
    P.test_psa_splits_satisfy_paper_condition,
    P.test_one_heavy_among_equal_lights_closed_form,
    P.test_vose_f64_against_exact_probabilities,
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
    # the second phase skips leftovers at exactly capacity when looking for its first light item
    "pp_second_phase_full_not_light": ("    while (i < m && V(i) > Q) ++i;           /* first light */",
                                       "    while (i < m && V(i) >= Q) ++i;          /* first light */"),
    # a tile's residual drops the packed light item's weight
    "pp_residual_drops_light": ("                    w = (w + nq(&in, i)) - Q;", "                    w = w - Q;"),
    # the next item of a packed heavy is looked up among the lights
    "pp_next_heavy_is_light": ("                    while (jn < t1 && is_light(&in, jn)) ++jn;",
                               "                    while (jn < t1 && !is_light(&in, jn)) ++jn;"),
}


# The indexed queries (the checkers of the full-size sample tests), caught by
# the pins of test_oracle_sample_at.py.
SA_MUTANTS = {
    # the sample index's high word dropped from the counter
    "sample_at_counter_hi": ("        uint64_t s = s_idx[t];\n        uint32_t key[2], ctr[4], x[4];\n        uint64_t u, v, r;\n"
                             "        key[0] = (uint32_t)seed; key[1] = (uint32_t)(seed >> 32);\n"
                             "        ctr[0] = (uint32_t)s; ctr[1] = (uint32_t)(s >> 32);",
                             "        uint64_t s = s_idx[t];\n        uint32_t key[2], ctr[4], x[4];\n        uint64_t u, v, r;\n"
                             "        key[0] = (uint32_t)seed; key[1] = (uint32_t)(seed >> 32);\n"
                             "        ctr[0] = (uint32_t)s; ctr[1] = 0;"),
    # the seed's words swapped in the key
    "sample_at_key_swapped": ("        uint64_t s = s_idx[t];\n        uint32_t key[2], ctr[4], x[4];\n        uint64_t u, v, r;\n"
                              "        key[0] = (uint32_t)seed; key[1] = (uint32_t)(seed >> 32);",
                              "        uint64_t s = s_idx[t];\n        uint32_t key[2], ctr[4], x[4];\n        uint64_t u, v, r;\n"
                              "        key[0] = (uint32_t)(seed >> 32); key[1] = (uint32_t)seed;"),
    # the listed position used as the counter instead of the listed sample index
    "sample_at_position": ("        uint64_t s = s_idx[t];\n", "        uint64_t s = t;\n"),
    # the two-level walk drops the sample index's high word
    "sample_2lvl_counter_hi": ("        key[1] = (uint32_t)(seed >> 32) + (uint32_t)d * 0xBB67AE85u;\n"
                               "        ctr[0] = (uint32_t)s; ctr[1] = (uint32_t)(s >> 32);",
                               "        key[1] = (uint32_t)(seed >> 32) + (uint32_t)d * 0xBB67AE85u;\n"
                               "        ctr[0] = (uint32_t)s; ctr[1] = 0;"),
    # the indexed two-level queries walk sample t instead of the listed index
    "sample_2lvl_at_position": ("out[t] = sample_2lvl_one(L, sizes, G, thr, al, qp, seed, stream, s_idx[t]);",
                                "out[t] = sample_2lvl_one(L, sizes, G, thr, al, qp, seed, stream, t);"),
}

SA_PINS = [SA.test_sample_at_equals_sequential_queries, SA.test_sample_at_high_counter_words_against_published_philox,
           SA.test_sample_2lvl_at_equals_sequential_walk, SA.test_sample_2lvl_at_bottom_level_against_published_philox]


def _pp_alias_tables():
    for name, w in PP.INPUTS[:4]:
        for T in (3, 64):
            PP.test_every_tile_size_gives_an_alias_table(name, w, T)


PP_PINS = [PP.test_hand_examples, PP.test_exhaustive_small, _pp_alias_tables]


# Two-level tables (Sec. 6, Alg. 2 per group), caught by the two-level pins.
# Every mutant keeps each index inside its level, so a mutated oracle cannot
# read out of bounds.
TL_MUTANTS = {
    # a group's aliases stay local to the group instead of level-wide indices
    "tl_alias_local": ("            for (m = 0; m < ng; ++m) al[off + b0 + m] += (uint32_t)b0;\n", ""),
    # the next level's weight of a group is its first member's instead of the group total
    "tl_next_weight": ("st128(next + 2 * g, S);", "st128(next + 2 * g, ld128(w + 2 * b0));"),
    # every level draws with the same key, so the levels' picks are correlated
    "tl_same_key_each_level": ("        key[0] = (uint32_t)seed + (uint32_t)d * 0x9E3779B9u;\n"
                               "        key[1] = (uint32_t)(seed >> 32) + (uint32_t)d * 0xBB67AE85u;",
                               "        key[0] = (uint32_t)seed;\n        key[1] = (uint32_t)(seed >> 32);"),
    # the coin of every group uses the denominator of the level's first group
    "tl_coin_group0": ("g = ((uint64_t)(((u128)v * qp[goffs[lv] + g]) >> 64) < thr[b]) ? base + r : al[b];",
                       "g = ((uint64_t)(((u128)v * qp[goffs[lv]]) >> 64) < thr[b]) ? base + r : al[b];"),
}


def _tl_pins():
    for n, G, seed in TL.GROUP_CASES:
        TL.test_every_group_is_an_alias_table(n, G, seed)


def _tl_probabilities():
    for n, G, seed in TL.PROB_CASES:
        TL.test_item_probabilities_are_the_weights(n, G, seed)


TL_PINS = [TL.test_hand_examples, _tl_pins, _tl_probabilities, TL.test_samples_follow_the_weights]


# OS-ND (Sec. 5 output-sensitive sampling, Sec. 10 base case), caught by the
# OS-ND pins.  An inversion try ends once its pmf terms underflow, so a mutant
# whose P(X = 0) is too small only makes more tries fail.
OS_MUTANTS = {
    # symmetry: the deviate drawn for 1 - p is returned as the one for p
    "os_flip_dropped": ("return flip ? n - x : x;", "return x;"),
    # the left child's weight counts the middle member too
    "os_split_mid": ("if (i < mid) wl += w;", "if (i <= mid) wl += w;"),
    # inversion: the pmf ratio drops its "- p/q" term
    "os_inversion_ratio": ("r *= (x <= 40 ? a * DET_INV[x] : a / (double)x) - s;",
                           "r *= (x <= 40 ? a * DET_INV[x] : a / (double)x);"),
    # BTRS: log(q/p) in place of log(p/q) in the acceptance test
    "os_btrs_lpq": ("lpq = det_log(p / q);", "lpq = det_log(q / p);"),
    # base case: every group's coin uses the level's first denominator
    "os_base_coin_group0": ("x->qp[x->goffs[level] + g]", "x->qp[x->goffs[level]]"),
    # log: range reduction moves the exponent the wrong way
    "log_reduction": ("if (f > 1.4142135623730951) { f = f * 0.5; e += 1; }",
                      "if (f > 1.4142135623730951) { f = f * 0.5; e -= 1; }"),
    # log(1 - p): sign of the series dropped
    "log1m_sign": ("return -p * acc;", "return p * acc;"),
    # Stirling: (k + 1/2) log z written as k log z
    "lfact_half": ("((double)k + 0.5) * det_log(z) - z", "(double)k * det_log(z) - z"),
    # Stirling: the 1/(12 z) ... correction dropped
    "lfact_corr": ("0.5 * det_log(6.283185307179586) + corr;", "0.5 * det_log(6.283185307179586);"),
    # p's conversion: ties rounded up instead of to even
    "u128_ties_up": ("if (rem > half || (rem == half && (m & 1))) {", "if (rem >= half) {"),
    # power-of-two scaling: exponent bias off by one
    "ldexp_bias": ("t.u = (uint64_t)(e + 1023) << 52;", "t.u = (uint64_t)(e + 1022) << 52;"),
    # exp: range reduction adds k ln 2 instead of subtracting it
    "exp_reduction": ("r = x - kd * 0.6931471805599453;", "r = x + kd * 0.6931471805599453;"),
    # exp: the Taylor terms' 1/j taken as 1/(j + 1)
    "exp_term_index": ("for (j = 20; j >= 1; --j) acc = acc * (r * DET_INV[j]) + 1.0;",
                       "for (j = 20; j >= 1; --j) acc = acc * (r * DET_INV[j + 1]) + 1.0;"),
}


def _os_laws():
    for n, num, den in OS.LAW_CASES:
        OS.test_binomial_law(n, num, den)


def _os_counts():
    for k in OS.COUNT_CASES:
        OS.test_osnd_counts_add_up(k)


def _os_single_weight():
    for n in (2047, 5000):
        OS.test_osnd_single_nonzero_weight(n)


OS_PINS = [OS.test_series_log_exp, OS.test_series_log1m, OS.test_series_lfact,
           OS.test_u128_to_double_rounds_to_nearest_even, OS.test_ldexp_is_exact_scaling, OS.test_binomial_edges,
           OS.test_binomial_tiny_p_huge_n, _os_laws, _os_counts, OS.test_osnd_is_multinomial,
           OS.test_osnd_small_k_follows_the_weights, _os_single_weight]


def _run_mutant(old, new, pins, tmp_path):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation site not found exactly once"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    so = str(tmp_path / "libmutant.so")
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-shared", "-fPIC", "-o", so,
                           str(mutated), "-lm"])
    caught = []
    with O.use_library(so):
        for pin in pins:
            try:
                pin()
            except (Exception, pytest.fail.Exception):  # a failed check or an oracle error: caught
                caught.append(pin.__name__)
    return caught


@pytest.mark.parametrize("name", sorted(PP_MUTANTS))
def test_every_planted_psa_plus_mistake_is_caught(name, tmp_path):
    old, new = PP_MUTANTS[name]
    assert _run_mutant(old, new, PP_PINS, tmp_path), f"mutant {name} passed every PSA+ pin"


@pytest.mark.parametrize("name", sorted(TL_MUTANTS))
def test_every_planted_two_level_mistake_is_caught(name, tmp_path):
    old, new = TL_MUTANTS[name]
    assert _run_mutant(old, new, TL_PINS, tmp_path), f"mutant {name} passed every two-level pin"


@pytest.mark.parametrize("name", sorted(OS_MUTANTS))
def test_every_planted_osnd_mistake_is_caught(name, tmp_path):
    old, new = OS_MUTANTS[name]
    assert _run_mutant(old, new, OS_PINS, tmp_path), f"mutant {name} passed every OS-ND pin"


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_every_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    assert _run_mutant(old, new, PINS, tmp_path), f"mutant {name} passed every pin"


@pytest.mark.parametrize("name", sorted(SA_MUTANTS))
def test_every_planted_indexed_query_mistake_is_caught(name, tmp_path):
    old, new = SA_MUTANTS[name]
    assert _run_mutant(old, new, SA_PINS, tmp_path), f"mutant {name} passed every indexed-query pin"
