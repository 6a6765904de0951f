"""Independent checks of alias tables against what the paper and the
mathematics fix.  Nothing here calls the oracle's construction code: the
checks start from the weights and a table (bucket masses, aliases, coin
thresholds) and verify the definition of an alias table (Sec. 2.2), the exact
distribution P[X = i] = w_i / W (problem WRS-1, Sec. 1) and closed forms.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

TWO64 = 1 << 64


def exact_units(w) -> tuple[list[int], int, int]:
    """Independent normalisation: q_i = w_i * 2^-beta with beta the lowest set
    bit over all nonzero weights (Fractions, not the oracle's decoder)."""
    arr = np.asarray(w)
    if arr.dtype == np.uint32:
        q = [int(x) for x in arr]
        return q, sum(q), 0
    fr = [Fraction(float(x)) for x in arr]
    lows = []
    for f in fr:
        if f == 0:
            continue
        num, den = f.numerator, f.denominator
        v2 = (num & -num).bit_length() - 1
        lows.append(v2 - (den.bit_length() - 1))
    beta = min(lows)
    q = [int(f / Fraction(2) ** beta) for f in fr]
    for f, qi in zip(fr, q):
        assert Fraction(qi) * Fraction(2) ** beta == f
    return q, sum(q), beta


def check_alias_table(q: list[int], Q: int, bw: list[int], alias: list[int]) -> None:
    """Sec. 2.2: n buckets of capacity W/n (here Q); bucket b holds part bw_b of
    item b and the rest of its capacity for one alias; light items (n q <= Q)
    keep their whole weight in their own bucket; the pieces of every item add
    up to its weight (here n q_i).  Also: full buckets point to themselves and
    every other alias is a heavy item."""
    n = len(q)
    assert len(bw) == n and len(alias) == n
    mass = [0] * n
    for b in range(n):
        assert 0 <= bw[b] <= Q, (b, bw[b], Q)
        a = int(alias[b])
        assert 0 <= a < n
        mass[b] += bw[b]
        if a != b:
            assert n * q[a] > Q, f"alias {a} of bucket {b} is not heavy"
            mass[a] += Q - bw[b]
        else:
            assert bw[b] == Q, f"self-alias on a bucket that is not full ({b})"
        if n * q[b] <= Q:
            assert bw[b] == n * q[b], f"light bucket {b} does not hold its weight"
        if bw[b] == Q:
            assert a == b
    for i in range(n):
        assert mass[i] == n * q[i], (i, mass[i], n * q[i])


def coin_heads(thr: int, Qp: int, bits: int = 64) -> int:
    """#{v in [0, 2^bits) : floor(v * Qp / 2^bits) < thr}."""
    if thr >= Qp:
        return 1 << bits
    return -((-thr << bits) // Qp)  # ceil(thr * 2^bits / Qp)


def bucket_count(r: int, n: int, bits: int = 64) -> int:
    """#{u in [0, 2^bits) : floor(u * n / 2^bits) = r}."""
    def first(x):  # the least u with floor(u * n / 2^bits) >= x
        return -((-x << bits) // n)
    return first(r + 1) - first(r)


def exact_query_distribution(thr, alias, Qp: int) -> list[Fraction]:
    """P[X = i] of the query rule applied to 128 uniform bits, summed over all
    outcomes in closed form (bucket from the low word, coin from the high)."""
    n = len(thr)
    p = [Fraction(0)] * n
    for r in range(n):
        cb = Fraction(bucket_count(r, n), TWO64)
        h = Fraction(coin_heads(int(thr[r]), Qp), TWO64)
        p[r] += cb * h
        p[int(alias[r])] += cb * (1 - h)
    return p


def _limb_sums(values: np.ndarray, index: np.ndarray, n: int) -> list[np.ndarray]:
    """Per-item sums of 16-bit limbs of uint64 values, each exact in float64
    (at most 2^32 terms of < 2^16 each)."""
    out = []
    for k in range(4):
        limb = ((values >> np.uint64(16 * k)) & np.uint64(0xFFFF)).astype(np.float64)
        out.append(np.bincount(index, weights=limb, minlength=n).astype(np.uint64))
    return out


def _combine_limbs(sums: list[np.ndarray]) -> tuple[np.ndarray, np.ndarray]:
    """sum_k sums[k] << 16k as (lo, hi) uint64 words."""
    words = []
    carry = np.zeros_like(sums[0])
    for k in range(8):
        cur = (sums[k] if k < len(sums) else np.zeros_like(carry)) + carry
        words.append(cur & np.uint64(0xFFFF))
        carry = cur >> np.uint64(16)
    lo = words[0] | (words[1] << np.uint64(16)) | (words[2] << np.uint64(32)) | (words[3] << np.uint64(48))
    hi = words[4] | (words[5] << np.uint64(16)) | (words[6] << np.uint64(32)) | (words[7] << np.uint64(48))
    return lo, hi


def item_mass_words(thr: np.ndarray, alias: np.ndarray, Qp: int) -> tuple[np.ndarray, np.ndarray]:
    """Per item: sum over buckets of own part thr_b plus, where item is the
    alias of another bucket, that bucket's rest Qp - thr_b; exact, as (lo, hi)
    uint64 words.  Vectorised for tables of any size."""
    n = thr.shape[0]
    thr = thr.astype(np.uint64)
    al = alias.astype(np.int64)
    own = _limb_sums(thr, np.arange(n), n)
    other = al != np.arange(n)
    rest = np.where(other, np.uint64(Qp) - thr, np.uint64(0)).astype(np.uint64)
    ali = _limb_sums(rest, al, n)
    return _combine_limbs([a + b for a, b in zip(own, ali)])


def times_n_words(q: np.ndarray, n: int) -> tuple[np.ndarray, np.ndarray]:
    """n * q for uint64 q as exact (lo, hi) words."""
    q = q.astype(np.uint64)
    limbs = [((q >> np.uint64(16 * k)) & np.uint64(0xFFFF)) * np.uint64(n) for k in range(4)]
    # each limb*n < 2^48; spread into 16-bit limbs of the product
    sums = [np.zeros_like(q) for _ in range(8)]
    for k, v in enumerate(limbs):
        for j in range(4):
            if k + j < 8:
                sums[k + j] = sums[k + j] + ((v >> np.uint64(16 * j)) & np.uint64(0xFFFF))
    return _combine_limbs(sums)
