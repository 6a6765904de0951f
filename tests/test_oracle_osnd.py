"""Pins of the oracle's OS-ND sampler (Sec. 5 output-sensitive sampling with
replacement; Sec. 10 "Optimizations", no deduplication), checked against
mathematics that does not come from its code: the library log/exp, the
exact binomial pmf (scipy), and the multinomial law of k draws."""
import math

import numpy as np
import pytest

from oracle import wrs_oracle as O
from paper_1903_00227_gb300 import workloads as WL

scipy_stats = pytest.importorskip("scipy.stats")


def test_series_log_exp():
    xs = [5e-324, 1e-300, 1e-10, 0.3, 0.5, 0.7071, 0.999999, 1.5, 2.0, 3.7, 1e5, 1e300, 1.7e308]
    for x in xs:
        assert abs(O.det_log(x) - math.log(x)) <= 4e-16 * abs(math.log(x)), x
    assert O.det_log(1.0) == 0.0
    for y in [-700.0, -50.0, -1.0, -0.1, 0.0, 0.1, 1.0, 10.0, 300.0, 700.0]:
        assert abs(O.det_exp(y) - math.exp(y)) <= 1e-13 * math.exp(y), y
    assert O.det_exp(-746.0) == 0.0


def test_series_log1m():
    for p in [1e-300, 1e-18, 1e-12, 3e-7, 1e-3, 0.1, 0.2499, 0.25, 0.3, 0.5]:
        want = math.log1p(-p)
        assert abs(O.det_log1m(p) - want) <= 4e-16 * abs(want), p


def test_series_lfact():
    """log(k!) of the BTRS acceptance test against the library's lgamma: exact
    product below 10; above, Stirling's series to the z^-7 term, whose error
    is below the first omitted term 1 / (1188 z^9), z = k + 1."""
    for k in list(range(40)) + [100, 1000, 10 ** 6, 10 ** 9, 10 ** 12, 2 ** 53]:
        want, z = math.lgamma(k + 1), k + 1.0
        bound = (1.0 / (1188.0 * z ** 9) if k >= 10 else 0.0) + 1e-15 * abs(want)
        assert abs(O.det_lfact(k) - want) <= bound, k
    assert O.det_lfact(0) == 0.0 and O.det_lfact(1) == 0.0


def test_u128_to_double_rounds_to_nearest_even():
    """The conversion that forms p = num / den: the nearest binary64 with
    ties to even, which is what Python's int -> float conversion guarantees."""
    rng = np.random.default_rng(17)
    xs = [0, 1, 2 ** 53 - 1, 2 ** 53, 2 ** 53 + 1, 2 ** 53 + 2, 2 ** 53 + 3, 2 ** 54 + 2, 2 ** 54 + 6,
          2 ** 64 - 1, 2 ** 64, 2 ** 95, 2 ** 95 + 2 ** 42, 2 ** 95 + 3 * 2 ** 42, 2 ** 128 - 1, 2 ** 127 + 2 ** 74]
    for bits in (54, 60, 64, 80, 96, 110, 128):
        for _ in range(200):
            x = int(rng.integers(0, 2 ** 62)) | (int(rng.integers(0, 2 ** 62)) << 62) | (int(rng.integers(0, 16)) << 124)
            x &= (1 << bits) - 1
            xs.append(x)
            sh = max(bits - 53, 1)
            xs.append((x >> sh << sh) | (1 << (sh - 1)))  # a tie at this width
    for x in xs:
        assert O.det_u128_to_double(x) == float(x), hex(x)


def test_ldexp_is_exact_scaling():
    """The power-of-two scaling of exp and of the u128 conversion, including
    results in the subnormal range (one rounding, ties to even)."""
    for x in (1.0, 1.5, 0.75, 1.9999999999999998, 2.0 ** 52 + 1):
        for e in (-1126, -1074, -1073, -1060, -1022, -1000, -999, -1, 0, 1, 75, 970, 1000, 1023):
            if math.frexp(x)[1] + e <= 1024:
                assert O.det_ldexp(x, e) == math.ldexp(x, e), (x, e)


def test_binomial_tiny_p_huge_n():
    """n p = 3 with n = 10^12: P(X = 0) = e^-3 to 1e-12 relative; the
    frequencies of 0 and of small values follow the Poisson limit."""
    N = 20_000
    draws = np.array([O.binomial(10 ** 12, 3, 10 ** 12, 5, node) for node in range(N)], dtype=np.int64)
    pmf = scipy_stats.binom.pmf(np.arange(12), 10 ** 12, 3e-12)
    obs = np.bincount(np.minimum(draws, 11), minlength=12)
    e = pmf * N
    e[11] = N - e[:11].sum()
    chi = float(((obs - e) ** 2 / e).sum())
    assert chi < 12 + 6 * math.sqrt(24), chi


def _chi2(draws, n, p):
    pmf = scipy_stats.binom.pmf(np.arange(n + 1), n, p) if n <= 10 ** 6 else None
    if pmf is None:  # bin the support around the mean
        mu, sd = n * p, math.sqrt(n * p * (1 - p))
        edges = np.floor(mu + sd * np.linspace(-4, 4, 33)).astype(np.int64)
        cdf = scipy_stats.binom.cdf(edges, n, p)
        probs = np.diff(np.concatenate([[0.0], cdf, [1.0]]))
        obs = np.bincount(np.searchsorted(edges, draws, side="left"), minlength=len(probs))
    else:
        probs, obs = pmf, np.bincount(draws, minlength=n + 1)
    e = probs * len(draws)
    keep = e >= 5
    chi = float(((obs[keep] - e[keep]) ** 2 / e[keep]).sum())
    rest_e, rest_o = e[~keep].sum(), obs[~keep].sum()
    if rest_e > 0:
        chi += (rest_o - rest_e) ** 2 / max(rest_e, 1.0)
    return chi, int(keep.sum())


LAW_CASES = [
    (5, 3, 10),            # inversion
    (30, 1, 5),            # inversion, n p = 6
    (200, 3, 10),          # BTRS
    (1000, 1, 2),          # BTRS at p = 1/2
    (1000, 7, 10),         # p > 1/2: symmetry
    (10 ** 6, 1, 10 ** 4), # BTRS, n p = 100
    (10 ** 9, 37, 100),    # BTRS, large n
    (10 ** 6, 3, 10 ** 6), # inversion, n p = 3
]
COUNT_CASES = [1, 7, 127, 128, 1000, 10 ** 6, 10 ** 12]


@pytest.mark.parametrize("n,num,den", LAW_CASES)
def test_binomial_law(n, num, den):
    N = 20_000
    draws = np.array([O.binomial(n, num, den, 11, node) for node in range(N)], dtype=np.int64)
    assert draws.min() >= 0 and draws.max() <= n
    p = num / den
    chi, dof = _chi2(draws, n, p)
    assert abs(chi - dof) < 6 * math.sqrt(2 * dof) + 10, (chi, dof)
    assert abs(draws.mean() - n * p) < 6 * math.sqrt(n * p * (1 - p) / N) + 1e-9


def test_binomial_edges():
    assert O.binomial(100, 0, 7, 1, 0) == 0
    assert O.binomial(100, 7, 7, 1, 0) == 100
    assert O.binomial(0, 1, 2, 1, 0) == 0


def _table(n, s, seed, zeros=()):
    w = WL.f32_zipf(n, s, seed)
    for z in zeros:
        w[z] = 0.0
    qz = O.quantize(w)
    return qz, O.build_2lvl(qz)


@pytest.mark.parametrize("k", COUNT_CASES)
def test_osnd_counts_add_up(k):
    qz, t = _table(5000, 1.2, 3, zeros=(10, 4999))
    items, counts = O.os_nd(qz, t, k, 5, 2)
    assert int(counts.sum()) == k and (counts >= 1).all()
    assert (items < qz.n).all()
    assert 10 not in set(items.tolist()) and 4999 not in set(items.tolist())
    if k < 128:
        assert len(items) == k and (counts == 1).all()  # base case: one pair per query
    again = O.os_nd(qz, t, k, 5, 2)
    assert np.array_equal(items, again[0]) and np.array_equal(counts, again[1])
    if k >= 10 ** 6:
        assert len(items) <= qz.n  # large counts: each item at most once (descent to the leaves)


@pytest.mark.parametrize("n", [1, 2047, 5000, 2048 * 2048 + 5])
def test_osnd_single_nonzero_weight(n):
    """All the weight on one item: every sample is that item, so a descent
    hands all k to it (one pair (i, k)), and where the item's group takes the
    base case (fewer than 128 samples, at least half as many items, Sec. 10)
    its k queries all land on it (k pairs (i, 1))."""
    i = n // 3
    w = np.zeros(n, np.float32)
    w[i] = 0.75
    qz = O.quantize(w)
    t = O.build_2lvl(qz)
    G = t.G
    n_group = min(G, n - i // G * G)  # members of the item's group
    for k in (1, 50, 127, 128, 10 ** 6, 10 ** 12):
        items, counts = O.os_nd(qz, t, k, 3, 1)
        if k < 128 and 2 * n_group >= k:
            assert items.tolist() == [i] * k and counts.tolist() == [1] * k, k
        else:
            assert items.tolist() == [i] and counts.tolist() == [k], k


def test_osnd_is_multinomial():
    qz, t = _table(3000, 1.0, 4)
    k = 10 ** 7
    items, counts = O.os_nd(qz, t, k, 9, 0)
    tot = np.bincount(items, weights=counts.astype(np.float64), minlength=qz.n)
    p = np.array([qz.q_int(i) for i in range(qz.n)], dtype=np.float64) / float(qz.Q)
    e = k * p
    chi = float(((tot - e) ** 2 / e).sum())
    assert abs(chi - qz.n) < 6 * math.sqrt(2 * qz.n), chi


def test_osnd_small_k_follows_the_weights():
    """Many independent small draws (base case, alias queries through every
    level): the per-item frequencies follow w_i / W."""
    qz, t = _table(9000, 0.9, 6)  # two levels
    tot = np.zeros(qz.n)
    for seed in range(4000):
        items, counts = O.os_nd(qz, t, 50, seed, 0)
        np.add.at(tot, items, counts)
    p = np.array([qz.q_int(i) for i in range(qz.n)], dtype=np.float64) / float(qz.Q)
    e = tot.sum() * p
    keep = e >= 5
    chi = float(((tot[keep] - e[keep]) ** 2 / e[keep]).sum())
    dof = int(keep.sum())
    assert abs(chi - dof) < 6 * math.sqrt(2 * dof) + 10, (chi, dof)
