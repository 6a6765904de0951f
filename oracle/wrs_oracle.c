/*
 * wrs_oracle.c -- CPU oracle for alias-table construction and sampling.
 *
 * TEST INFRASTRUCTURE.  This is a plain, slow, deliberately unoptimised
 * restatement of what the method computes, used only to check the CUDA
 * library.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no code, header, table or helper with the
 * CUDA path, and the product library never links or calls it.
 *
 * Source: L. Huebschle-Schneider and P. Sanders, "Parallel Weighted Random
 * Sampling" (arXiv 1903.00227).  Citations name the paper's sections and
 * algorithms:
 *   Sec. 2.2 "Bucket-Based Sampling"  -- alias table definition, query, Alg. 1
 *   Sec. 4.1 "Improved Sequential Alias Table Construction" -- Alg. 2 (sweep)
 *   Sec. 4.2 "Shared-Memory Parallel Alias Tables" -- Alg. 3 (PSA, split, pack)
 *   Sec. 10 "Experiments", paragraph "Optimizations" -- branchless query
 *
 * Exact units.  Every weight is turned into an exact non-negative integer
 * q_i (u32 weights: q_i = w_i; binary32 weights: q_i = w_i * 2^-beta with beta
 * the smallest exponent of a set mantissa bit, so q_i is an integer), and
 * Q = sum q_i.  Multiplying the paper's quantities by n/(2^beta) turns the
 * bucket capacity W/n into the integer Q and the weight of item i into the
 * integer n*q_i.  All construction arithmetic is then exact in 128 bits
 * (Q < 2^95 and n < 2^32 give n*Q < 2^127).
 *
 * Table encoding (the one reading of Sec. 2.2's "biased coin" this library
 * fixes): bucket b holds bw_b in [0, Q], the part of its own item, and an alias.
 * With s = max(0, bitlen(Q) - 64), Qp = Q >> s and thr_b = bw_b >> s, the coin
 * of bucket b comes up heads for a 64-bit uniform v iff floor(v*Qp / 2^64) <
 * thr_b.  A full bucket (bw = Q) gets alias = b.
 *
 * Status codes: 0 ok, 1 invalid input, 2 exact range exceeded, 3 an
 * invariant of exact arithmetic failed (never expected).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <limits.h>
#include <math.h>

typedef unsigned __int128 u128;

#define WO_OK 0
#define WO_EINVAL 1
#define WO_EOVERFLOW 2
#define WO_EINTERNAL 3

#define WO_Q_BITS 95 /* Q must stay below 2^95 */

static u128 ld128(const uint64_t *p) { return ((u128)p[1] << 64) | p[0]; }
static void st128(uint64_t *p, u128 v) { p[0] = (uint64_t)v; p[1] = (uint64_t)(v >> 64); }
static int bitlen128(u128 x) { int b = 0; while (x) { ++b; x >>= 1; } return b; }

/* ------------------------------------------------------------------------ */
/* Weight normalisation: q_i and Q = sum q_i (the "W := sum w_i" line that    */
/* opens Alg. 1, 2 and 3), in exact integer units.                            */
/* ------------------------------------------------------------------------ */

/* binary32 pattern -> value m * 2^e (m < 2^24).  Sign set, NaN, Inf: invalid. */
static int f32_decode(uint32_t bits, uint32_t *m, int *e)
{
    uint32_t ex = (bits >> 23) & 0xFFu, fr = bits & 0x7FFFFFu;
    if (bits >> 31) return 1;
    if (ex == 0xFFu) return 1;
    if (ex == 0) { *m = fr; *e = -149; }
    else { *m = fr | 0x800000u; *e = (int)ex - 150; }
    return 0;
}

static int ctz32(uint32_t x) { int c = 0; while (!(x & 1u)) { x >>= 1; ++c; } return c; }

/* dtype 0: uint32 weights; dtype 1: binary32 weights (passed as raw bits).
 * Out: q (2 words per item, lo/hi), Q (2 words), beta. */
int wo_quantize(int dtype, const uint32_t *w, uint64_t n, uint64_t *q,
                uint64_t *Qout, int32_t *beta_out)
{
    u128 Q = 0;
    uint64_t i;
    if (n == 0 || n >= ((uint64_t)1 << 32)) return WO_EINVAL;
    if (dtype == 0) {
        for (i = 0; i < n; ++i) { st128(q + 2 * i, w[i]); Q += w[i]; }
        *beta_out = 0;
    } else if (dtype == 1) {
        int beta = INT_MAX;
        for (i = 0; i < n; ++i) {
            uint32_t m; int e;
            if (f32_decode(w[i], &m, &e)) return WO_EINVAL;
            if (m && e + ctz32(m) < beta) beta = e + ctz32(m);
        }
        if (beta == INT_MAX) return WO_EINVAL; /* every weight is zero */
        for (i = 0; i < n; ++i) {
            uint32_t m; int e; u128 qi = 0;
            f32_decode(w[i], &m, &e);
            if (m) {
                int sh = e - beta;
                if (sh >= 0) {
                    if (bitlen128(m) + sh > WO_Q_BITS) return WO_EOVERFLOW;
                    qi = (u128)m << sh;
                } else {
                    qi = (u128)(m >> (-sh)); /* exact: m has >= -sh trailing zeros */
                }
            }
            st128(q + 2 * i, qi);
            Q += qi;
            if (bitlen128(Q) > WO_Q_BITS) return WO_EOVERFLOW;
        }
        *beta_out = beta;
    } else {
        return WO_EINVAL;
    }
    if (Q == 0) return WO_EINVAL;
    st128(Qout, Q);
    return WO_OK;
}

/* ------------------------------------------------------------------------ */
/* Alg. 2 (Sec. 4.1): the sweeping construction.                             */
/* i runs over light items, j over heavy items, both in index order; w is     */
/* the part of heavy item j not yet assigned.  If w exceeds the capacity, the */
/* next light bucket is packed with j as its alias; otherwise bucket j is     */
/* packed with the next heavy item as its alias.  Ties (w = capacity) pack    */
/* the heavy bucket, and items with n*q = Q are light (Sec. 2.2: w <= W/n).   */
/* ------------------------------------------------------------------------ */

typedef struct { uint64_t n; const uint64_t *q; u128 Q; } wo_in;

static u128 nq(const wo_in *in, uint64_t k) { return (u128)in->n * ld128(in->q + 2 * k); }
static int is_light(const wo_in *in, uint64_t k) { return nq(in, k) <= in->Q; }

static uint64_t next_light(const wo_in *in, uint64_t k)
{
    while (k < in->n && !is_light(in, k)) ++k;
    return k;
}

static uint64_t next_heavy(const wo_in *in, uint64_t k)
{
    while (k < in->n && is_light(in, k)) ++k;
    return k;
}

static void put(uint64_t *bw, uint32_t *al, uint64_t b, u128 v, uint64_t a)
{
    st128(bw + 2 * b, v);
    al[b] = (uint32_t)a;
}

/* A bucket holding exactly the capacity needs no alias: it points to itself. */
static void canonicalise(uint64_t n, u128 Q, const uint64_t *bw, uint32_t *al)
{
    uint64_t b;
    for (b = 0; b < n; ++b)
        if (ld128(bw + 2 * b) == Q) al[b] = (uint32_t)b;
}

int wo_sweep(uint64_t n, const uint64_t *q, const uint64_t *Qin,
             uint64_t *bw, uint32_t *al)
{
    wo_in in = { n, q, ld128(Qin) };
    uint64_t i = next_light(&in, 0), j = next_heavy(&in, 0), k;
    u128 w;
    if (j == n) { /* all weights equal: every bucket is its own item */
        for (k = 0; k < n; ++k) {
            if (nq(&in, k) != in.Q) return WO_EINTERNAL;
            put(bw, al, k, nq(&in, k), k);
        }
        return WO_OK;
    }
    w = nq(&in, j);
    while (j < n) {
        if (w > in.Q) { /* pack a light bucket */
            if (i >= n) return WO_EINTERNAL;
            put(bw, al, i, nq(&in, i), j);
            w = (w + nq(&in, i)) - in.Q;
            i = next_light(&in, i + 1);
        } else { /* pack a heavy bucket */
            uint64_t jn = next_heavy(&in, j + 1);
            put(bw, al, j, w, jn < n ? jn : j);
            if (jn < n) w = (w + nq(&in, jn)) - in.Q;
            else if (w != in.Q) return WO_EINTERNAL; /* the last heavy ends full */
            j = jn;
        }
    }
    /* lights left once the heavies are used up must be exactly full */
    for (; i < n; i = next_light(&in, i + 1)) {
        if (nq(&in, i) != in.Q) return WO_EINTERNAL;
        put(bw, al, i, nq(&in, i), i);
    }
    canonicalise(n, in.Q, bw, al);
    return WO_OK;
}

/* ------------------------------------------------------------------------ */
/* Alg. 3 (Sec. 4.2): PSA.  Light list l and heavy list h in index order,     */
/* inclusive prefix sums L, H of their q, p-1 splits at n'_k = ceil(n*k/p),  */
/* then p independent packs.                                                  */
/*                                                                            */
/* split(n') reading: the paper asks for i + j = n' with                      */
/*   sigma = L[i] + H[j] <= n'W/n  and  sigma + w_{h[j+1]} > n'W/n,            */
/* which can hold for two neighbouring j.  This oracle takes the largest such */
/* j, i.e. j* = max{ j : n*(L[n'-j] + H[j]) <= n'*Q } over the feasible range */
/* [max(0, n'-|l|), min(n', |h|)]; that is exactly the state of Alg. 2 after */
/* n' buckets.  The spill is the residual of heavy h[j*] (0-based) after the  */
/* left part: r* = n*(L[i*] + H[j*] + q_{h[j*]}) - n'*Q (0 if j* = |h|).      */
/*                                                                            */
/* pack reading: subproblem k starts from split k-1's state (i, j, r) with    */
/* h[j] the current heavy item and r its unassigned part, runs exactly        */
/* n'_k - n'_{k-1} steps of the sweep rule and must end in split k's state.   */
/* ------------------------------------------------------------------------ */

typedef struct {
    const wo_in *in;
    uint64_t nl, nh;
    uint32_t *l, *h;
    u128 *L, *H;
} wo_lists;

typedef struct wo_psa_ctx wo_psa_ctx;

static int split_pred(const wo_lists *s, uint64_t np, uint64_t j)
{
    u128 sigma = s->L[np - j] + s->H[j];
    return (u128)s->in->n * sigma <= (u128)np * s->in->Q;
}

static int wo_split(const wo_lists *s, uint64_t np, uint64_t *ri, uint64_t *rj, u128 *rr)
{
    uint64_t lo = np > s->nl ? np - s->nl : 0;
    uint64_t hi = np < s->nh ? np : s->nh;
    uint64_t a, b, j, i;
    if (lo > hi || !split_pred(s, np, lo)) return WO_EINTERNAL;
    a = lo; b = hi; /* pred(a) holds; the answer lies in [a, b] */
    while (a < b) {
        uint64_t mid = a + (b - a + 1) / 2;
        if (split_pred(s, np, mid)) a = mid; else b = mid - 1;
    }
    j = a; i = np - j;
    *ri = i; *rj = j;
    if (j < s->nh) {
        u128 r = (u128)s->in->n * (s->L[i] + s->H[j] + ld128(s->in->q + 2 * (uint64_t)s->h[j]))
                 - (u128)np * s->in->Q;
        if (r == 0 || r > nq(s->in, s->h[j])) return WO_EINTERNAL;
        *rr = r;
    } else {
        *rr = 0;
    }
    return WO_OK;
}

/* The steps of Alg. 3 as separate calls, so that a driver can run the     */
/* p - 1 splits and the p packs (independent of each other, as the paper    */
/* runs them on p PEs) concurrently: begin (the two traversals and their    */
/* prefix sums), split(k) for 0 < k < p, pack(k) for 0 < k <= p once splits */
/* k - 1 and k exist, end (canonicalise, split records, free).  wo_psa runs */
/* them in order.                                                           */
struct wo_psa_ctx {
    wo_in in;
    wo_lists s;
    uint64_t p;
    uint64_t *si, *sj, *snp;
    u128 *sr;
    uint64_t *bw;
    uint32_t *al;
};

void wo_psa_free(wo_psa_ctx *c)
{
    if (!c) return;
    free(c->s.l); free(c->s.h); free(c->s.L); free(c->s.H);
    free(c->si); free(c->sj); free(c->snp); free(c->sr);
    free(c);
}

wo_psa_ctx *wo_psa_begin(uint64_t n, const uint64_t *q, const uint64_t *Qin, uint64_t p, uint64_t *bw, uint32_t *al)
{
    wo_psa_ctx *c;
    uint64_t x;
    if (p == 0 || p > n) return NULL;
    c = calloc(1, sizeof *c);
    if (!c) return NULL;
    c->in.n = n; c->in.q = q; c->in.Q = ld128(Qin);
    c->s.in = &c->in;
    c->p = p; c->bw = bw; c->al = al;
    c->s.l = malloc(n * sizeof *c->s.l); c->s.h = malloc(n * sizeof *c->s.h);
    c->s.L = malloc((n + 1) * sizeof *c->s.L); c->s.H = malloc((n + 1) * sizeof *c->s.H);
    c->si = malloc((p + 1) * sizeof *c->si); c->sj = malloc((p + 1) * sizeof *c->sj);
    c->snp = malloc((p + 1) * sizeof *c->snp); c->sr = malloc((p + 1) * sizeof *c->sr);
    if (!c->s.l || !c->s.h || !c->s.L || !c->s.H || !c->si || !c->sj || !c->snp || !c->sr) {
        wo_psa_free(c);
        return NULL;
    }
    {
        wo_in in = c->in;
        wo_lists s = c->s;
        /* the two parallel traversals of Alg. 3, plus prefix sums of their weights */
        s.L[0] = 0; s.H[0] = 0;
        for (x = 0; x < n; ++x) {
            u128 qx = ld128(q + 2 * x);
            if (is_light(&in, x)) { s.l[s.nl] = (uint32_t)x; s.L[s.nl + 1] = s.L[s.nl] + qx; ++s.nl; }
            else                  { s.h[s.nh] = (uint32_t)x; s.H[s.nh + 1] = s.H[s.nh] + qx; ++s.nh; }
        }
        c->s.nl = s.nl; c->s.nh = s.nh;
    }
    /* boundaries: k = 0 starts with the first heavy item whole; k = p is the end */
    c->snp[0] = 0; c->si[0] = 0; c->sj[0] = 0; c->sr[0] = c->s.nh ? nq(&c->in, c->s.h[0]) : 0;
    c->snp[p] = n; c->si[p] = c->s.nl; c->sj[p] = c->s.nh; c->sr[p] = 0;
    return c;
}

int wo_psa_split(wo_psa_ctx *c, uint64_t k)
{
    uint64_t n = c->in.n, p = c->p, *snp = c->snp;
    if (k == 0 || k >= p) return WO_EINVAL;
        snp[k] = (uint64_t)(((u128)n * k + p - 1) / p); /* ceil(n*k/p) */
    return wo_split(&c->s, snp[k], &c->si[k], &c->sj[k], &c->sr[k]);
}

int wo_psa_pack(wo_psa_ctx *c, uint64_t k)
{
    wo_in in = c->in;
    wo_lists s = c->s;
    uint64_t *bw = c->bw;
    uint32_t *al = c->al;
    uint64_t i, j, step;
    u128 r;
    if (k == 0 || k > c->p) return WO_EINVAL;
    s.in = &in;
    i = c->si[k - 1]; j = c->sj[k - 1]; r = c->sr[k - 1];
    for (step = c->snp[k - 1]; step < c->snp[k]; ++step) {
            if (j < s.nh && r <= in.Q) { /* heavy bucket h[j] */
                uint64_t jn = j + 1;
                put(bw, al, s.h[j], r, jn < s.nh ? s.h[jn] : s.h[j]);
                if (jn < s.nh) r = (r + nq(&in, s.h[jn])) - in.Q;
                else { if (r != in.Q) return WO_EINTERNAL; r = 0; }
                j = jn;
            } else { /* light bucket l[i] */
                if (i >= s.nl) return WO_EINTERNAL;
                put(bw, al, s.l[i], nq(&in, s.l[i]), j < s.nh ? s.h[j] : s.l[i]);
                if (j < s.nh) r = (r + nq(&in, s.l[i])) - in.Q;
                else if (nq(&in, s.l[i]) != in.Q) return WO_EINTERNAL;
                ++i;
            }
    }
    if (i != c->si[k] || j != c->sj[k] || (j < s.nh && r != c->sr[k])) return WO_EINTERNAL;
    return WO_OK;
}

/* splits (optional, 4 words per k = 0..p): n'_k, i_k, j_k, r_k low word */
void wo_psa_end(wo_psa_ctx *c, uint64_t *splits)
{
    uint64_t k;
    canonicalise(c->in.n, c->in.Q, c->bw, c->al);
    if (splits)
        for (k = 0; k <= c->p; ++k) {
            splits[4 * k + 0] = c->snp[k]; splits[4 * k + 1] = c->si[k];
            splits[4 * k + 2] = c->sj[k]; splits[4 * k + 3] = (uint64_t)c->sr[k];
        }
    wo_psa_free(c);
}

int wo_psa(uint64_t n, const uint64_t *q, const uint64_t *Qin, uint64_t p,
           uint64_t *bw, uint32_t *al, uint64_t *splits)
{
    uint64_t k;
    int rc = WO_OK;
    wo_psa_ctx *c;
    if (p == 0 || p > n) return WO_EINVAL;
    c = wo_psa_begin(n, q, Qin, p, bw, al);
    if (!c) return WO_EINVAL;
    for (k = 1; k < p && rc == WO_OK; ++k) rc = wo_psa_split(c, k);
    for (k = 1; k <= p && rc == WO_OK; ++k) rc = wo_psa_pack(c, k);
    if (rc) { wo_psa_free(c); return rc; }
    wo_psa_end(c, splits);
    return WO_OK;
}

/* ------------------------------------------------------------------------ */
/* Alg. 1 (Sec. 2.2): Vose-style construction with stacks of heavy and light */
/* items, in exact integers.  Reading: the stacks are filled in index order, */
/* so pop() returns the highest remaining index.  Items whose alias is still */
/* undefined at the end are exactly full and point to themselves.            */
/* ------------------------------------------------------------------------ */

int wo_vose(uint64_t n, const uint64_t *q, const uint64_t *Qin, uint64_t *bw, uint32_t *al)
{
    wo_in in = { n, q, ld128(Qin) };
    uint32_t *hs = malloc(n * sizeof *hs), *ls = malloc(n * sizeof *ls);
    uint8_t *set = calloc(n, 1);
    uint64_t nh = 0, nl = 0, k;
    int rc = WO_OK;
    if (!hs || !ls || !set) { rc = WO_EINVAL; goto out; }
    for (k = 0; k < n; ++k) {
        st128(bw + 2 * k, nq(&in, k));
        if (is_light(&in, k)) ls[nl++] = (uint32_t)k; else hs[nh++] = (uint32_t)k;
    }
    while (nh) {
        uint32_t j = hs[--nh];
        while (ld128(bw + 2 * (uint64_t)j) > in.Q) {
            uint32_t i;
            if (!nl) { rc = WO_EINTERNAL; goto out; }
            i = ls[--nl];
            al[i] = j; set[i] = 1;
            /* (b[j].w + b[i].w) - W/n, the cancellation-avoiding order */
            st128(bw + 2 * (uint64_t)j, (ld128(bw + 2 * (uint64_t)j) + ld128(bw + 2 * (uint64_t)i)) - in.Q);
        }
        ls[nl++] = j;
    }
    for (k = 0; k < n; ++k)
        if (!set[k]) {
            if (ld128(bw + 2 * k) != in.Q) { rc = WO_EINTERNAL; goto out; }
            al[k] = (uint32_t)k;
        }
    canonicalise(n, in.Q, bw, al);
out:
    free(hs); free(ls); free(set);
    return rc;
}

/* Alg. 1 in binary64, as the paper's classic sequential baseline.  Out: the */
/* coin probability of each bucket (b.w * n / W) and its alias.              */
int wo_vose_f64(uint64_t n, const double *w, double *prob, uint32_t *al)
{
    uint32_t *hs = malloc(n * sizeof *hs), *ls = malloc(n * sizeof *ls);
    double *bw = malloc(n * sizeof *bw);
    uint8_t *set = calloc(n, 1);
    double W = 0.0, cap;
    uint64_t nh = 0, nl = 0, k;
    int rc = WO_OK;
    if (!hs || !ls || !bw || !set) { rc = WO_EINVAL; goto out; }
    for (k = 0; k < n; ++k) W += w[k];
    cap = W / (double)n;
    for (k = 0; k < n; ++k) {
        bw[k] = w[k];
        if (w[k] <= cap) ls[nl++] = (uint32_t)k; else hs[nh++] = (uint32_t)k;
    }
    while (nh) {
        uint32_t j = hs[--nh];
        while (bw[j] > cap && nl) { /* rounding may exhaust the lights first */
            uint32_t i = ls[--nl];
            al[i] = j; set[i] = 1;
            bw[j] = (bw[j] + bw[i]) - cap;
        }
        ls[nl++] = j;
    }
    for (k = 0; k < n; ++k) {
        if (!set[k]) al[k] = (uint32_t)k;
        prob[k] = bw[k] / cap;
    }
out:
    free(hs); free(ls); free(bw); free(set);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Coin encoding (see the header comment): thr_b = bw_b >> s, Qp = Q >> s.   */
/* ------------------------------------------------------------------------ */

void wo_encode(uint64_t n, const uint64_t *bw, const uint64_t *Qin,
               uint64_t *thr, uint64_t *Qp_out, uint32_t *shift_out)
{
    u128 Q = ld128(Qin);
    int s = bitlen128(Q) - 64;
    uint64_t b;
    if (s < 0) s = 0;
    for (b = 0; b < n; ++b) thr[b] = (uint64_t)(ld128(bw + 2 * b) >> s);
    *Qp_out = (uint64_t)(Q >> s);
    *shift_out = (uint32_t)s;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC 2011): ten rounds of two 32x32->64 multiplications;  */
/* the key is bumped by the Weyl constants before every round but the first. */
/* ------------------------------------------------------------------------ */

void wo_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out)
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    int r;
    for (r = 0; r < 10; ++r) {
        uint64_t p0, p1;
        uint32_t n0, n1, n2, n3;
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        p0 = (uint64_t)0xD2511F53u * c0;
        p1 = (uint64_t)0xCD9E8D57u * c2;
        n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        n1 = (uint32_t)p1;
        n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* k independent alias queries (Sec. 2.2; Sec. 5, Cor. "kWR").  Sample s     */
/* draws 128 bits from Philox with counter (s, stream) and key seed: the low */
/* 64 bits u pick bucket r = floor(u*n / 2^64), the high 64 bits v toss the  */
/* coin, and the result is r on heads, its alias on tails.                   */
/* ------------------------------------------------------------------------ */

void wo_sample(uint64_t n, const uint64_t *thr, const uint32_t *al, uint64_t Qp,
               uint64_t k, uint64_t seed, uint64_t stream, uint32_t *out)
{
    uint64_t s;
    uint32_t key[2];
    key[0] = (uint32_t)seed; key[1] = (uint32_t)(seed >> 32);
    for (s = 0; s < k; ++s) {
        uint32_t ctr[4], x[4];
        uint64_t u, v, r;
        int heads;
        ctr[0] = (uint32_t)s; ctr[1] = (uint32_t)(s >> 32);
        ctr[2] = (uint32_t)stream; ctr[3] = (uint32_t)(stream >> 32);
        wo_philox4x32_10(ctr, key, x);
        u = (uint64_t)x[0] | ((uint64_t)x[1] << 32);
        v = (uint64_t)x[2] | ((uint64_t)x[3] << 32);
        r = (uint64_t)(((u128)u * n) >> 64);
        heads = (uint64_t)(((u128)v * Qp) >> 64) < thr[r];
        out[s] = heads ? (uint32_t)r : al[r];
    }
}

/* The same queries for an explicit list of sample indices s_idx[0..m). */
void wo_sample_at(uint64_t n, const uint64_t *thr, const uint32_t *al, uint64_t Qp,
                  uint64_t seed, uint64_t stream, const uint64_t *s_idx, uint64_t m, uint32_t *out)
{
    uint64_t t;
    for (t = 0; t < m; ++t) {
        uint32_t one;
        uint64_t s = s_idx[t];
        uint32_t key[2], ctr[4], x[4];
        uint64_t u, v, r;
        key[0] = (uint32_t)seed; key[1] = (uint32_t)(seed >> 32);
        ctr[0] = (uint32_t)s; ctr[1] = (uint32_t)(s >> 32);
        ctr[2] = (uint32_t)stream; ctr[3] = (uint32_t)(stream >> 32);
        wo_philox4x32_10(ctr, key, x);
        u = (uint64_t)x[0] | ((uint64_t)x[1] << 32);
        v = (uint64_t)x[2] | ((uint64_t)x[3] << 32);
        r = (uint64_t)(((u128)u * n) >> 64);
        one = ((uint64_t)(((u128)v * Qp) >> 64) < thr[r]) ? (uint32_t)r : al[r];
        out[t] = one;
    }
}

/* ------------------------------------------------------------------------ */
/* Two-level ("2lvl-sweep") tables, Sec. 6 "Distributed Alias Table          */
/* Construction" with the replicated top level, and Sec. 10 "Implementation  */
/* Details" (2lvl with Alg. 2 as the base case), applied recursively.        */
/*                                                                            */
/* Level 0 holds the n items in groups of G consecutive items (the last one  */
/* may be shorter).  Each group gets its own Alg. 2 table over its members in */
/* the group's own units: capacity Q_g = sum of its members' q, member m     */
/* weighs n_g * q_m (n_g = members of the group).  The groups' totals are    */
/* the items ("meta-items") of level 1, grouped the same way, and so on until */
/* a level has a single group.  Buckets are encoded per group (s_g, qp_g as  */
/* in wo_encode with Q_g); an alias is stored as the member's index within   */
/* its level.                                                                 */
/*                                                                            */
/* Sampling walks down from the top group: at depth d (0 at the top) Philox  */
/* with counter (s, stream) and key (seed_lo + d*0x9E3779B9, seed_hi +        */
/* d*0xBB67AE85) gives u and v; r = floor(u*n_g / 2^64) picks a bucket of the */
/* current group, the coin floor(v*qp_g / 2^64) < thr keeps r or takes the   */
/* alias, and the pick names the group of the next level down.  The pick at  */
/* level 0 is the sample.  With n <= G there is one level and one group, and */
/* table and samples are exactly those of wo_sweep + wo_encode + wo_sample.  */
/* ------------------------------------------------------------------------ */

#define WO_MAX_LEVELS 16

/* Entries per level: sizes[0] = n, sizes[l+1] = ceil(sizes[l] / G); returns L. */
int wo_2lvl_levels(uint64_t n, uint64_t G, uint64_t *sizes)
{
    int L = 0;
    uint64_t m = n;
    if (n == 0 || G < 2) return 0;
    for (;;) {
        sizes[L++] = m;
        if (m <= G || L == WO_MAX_LEVELS) break;
        m = (m + G - 1) / G;
    }
    return L;
}

/* thr, al: sum of sizes entries (level 0 first); qp, shift, tot (two words  */
/* each): one entry per group, level 0's groups first.                        */
int wo_2lvl_build(uint64_t n, const uint64_t *q, uint64_t G, uint64_t *thr, uint32_t *al,
                  uint64_t *qp, uint32_t *shift, uint64_t *tot)
{
    uint64_t sizes[WO_MAX_LEVELS];
    int L = wo_2lvl_levels(n, G, sizes), l;
    uint64_t off = 0, goff = 0;
    const uint64_t *w = q;
    uint64_t *bw, *next;
    if (L == 0) return WO_EINVAL;
    bw = (uint64_t *)malloc(2 * G * sizeof(uint64_t));
    next = (uint64_t *)malloc(2 * ((n + G - 1) / G + 1) * sizeof(uint64_t));
    if (!bw || !next) { free(bw); free(next); return WO_EINVAL; }
    for (l = 0; l < L; ++l) {
        const uint64_t N = sizes[l], ng_groups = (N + G - 1) / G;
        uint64_t g;
        for (g = 0; g < ng_groups; ++g) {
            const uint64_t b0 = g * G, ng = (N - b0 < G) ? N - b0 : G;
            uint64_t Qg[2], m, qpg;
            uint32_t sg;
            u128 S = 0;
            int rc;
            for (m = 0; m < ng; ++m) S += ld128(w + 2 * (b0 + m));
            st128(Qg, S);
            rc = wo_sweep(ng, w + 2 * b0, Qg, bw, al + off + b0);
            if (rc) { free(bw); free(next); return rc; }
            wo_encode(ng, bw, Qg, thr + off + b0, &qpg, &sg);
            for (m = 0; m < ng; ++m) al[off + b0 + m] += (uint32_t)b0;
            qp[goff + g] = qpg;
            shift[goff + g] = sg;
            st128(tot + 2 * (goff + g), S);
            st128(next + 2 * g, S);
        }
        /* the group totals are the next level's weights */
        if (l + 1 < L) {
            uint64_t *cur = (uint64_t *)malloc(2 * ng_groups * sizeof(uint64_t));
            if (!cur) { free(bw); free(next); return WO_EINVAL; }
            memcpy(cur, next, 2 * ng_groups * sizeof(uint64_t));
            if (w != q) free((void *)w);
            w = cur;
        }
        off += N;
        goff += ng_groups;
    }
    if (w != q) free((void *)w);
    free(bw);
    free(next);
    return WO_OK;
}

static uint32_t sample_2lvl_one(int L, const uint64_t *sizes, uint64_t G, const uint64_t *thr,
                                const uint32_t *al, const uint64_t *qp, uint64_t seed, uint64_t stream, uint64_t s)
{
    uint64_t offs[WO_MAX_LEVELS], goffs[WO_MAX_LEVELS], o = 0, go = 0, g = 0;
    int l, d;
    for (l = 0; l < L; ++l) { offs[l] = o; goffs[l] = go; o += sizes[l]; go += (sizes[l] + G - 1) / G; }
    for (d = 0; d < L; ++d) {
        const int lv = L - 1 - d;
        const uint64_t base = g * G, ng = (sizes[lv] - base < G) ? sizes[lv] - base : G;
        uint32_t key[2], ctr[4], x[4];
        uint64_t u, v, r, b;
        key[0] = (uint32_t)seed + (uint32_t)d * 0x9E3779B9u;
        key[1] = (uint32_t)(seed >> 32) + (uint32_t)d * 0xBB67AE85u;
        ctr[0] = (uint32_t)s; ctr[1] = (uint32_t)(s >> 32);
        ctr[2] = (uint32_t)stream; ctr[3] = (uint32_t)(stream >> 32);
        wo_philox4x32_10(ctr, key, x);
        u = (uint64_t)x[0] | ((uint64_t)x[1] << 32);
        v = (uint64_t)x[2] | ((uint64_t)x[3] << 32);
        r = (uint64_t)(((u128)u * ng) >> 64);
        b = offs[lv] + base + r;
        g = ((uint64_t)(((u128)v * qp[goffs[lv] + g]) >> 64) < thr[b]) ? base + r : al[b];
    }
    return (uint32_t)g;
}

void wo_2lvl_sample(uint64_t n, uint64_t G, const uint64_t *thr, const uint32_t *al, const uint64_t *qp,
                    uint64_t k, uint64_t seed, uint64_t stream, uint32_t *out)
{
    uint64_t sizes[WO_MAX_LEVELS], s;
    int L = wo_2lvl_levels(n, G, sizes);
    for (s = 0; s < k; ++s) out[s] = sample_2lvl_one(L, sizes, G, thr, al, qp, seed, stream, s);
}

void wo_2lvl_sample_at(uint64_t n, uint64_t G, const uint64_t *thr, const uint32_t *al, const uint64_t *qp,
                       uint64_t seed, uint64_t stream, const uint64_t *s_idx, uint64_t m, uint32_t *out)
{
    uint64_t sizes[WO_MAX_LEVELS], t;
    int L = wo_2lvl_levels(n, G, sizes);
    for (t = 0; t < m; ++t) out[t] = sample_2lvl_one(L, sizes, G, thr, al, qp, seed, stream, s_idx[t]);
}

/* ------------------------------------------------------------------------ */
/* Output-sensitive sampling with replacement, OS-ND variant (Sec. 5         */
/* "Output Sensitive Sampling With Replacement"; Sec. 10 "Optimizations":    */
/* descent aborted for fewer than 128 samples from at least half as many     */
/* items, no deduplication).  Reading: the divide-and-conquer tree is the    */
/* two-level structure above -- within a group a complete binary tree over   */
/* its members (node [a, b) splits at a + (b - a) / 2), whose leaves are     */
/* either items (level 0) or the groups one level down.  A node with c       */
/* samples gives Binomial(c, W_left / W_node) to its left child.  A group    */
/* receiving c < 128 samples with 2 n_g >= c draws them as c queries of its  */
/* alias table instead (level 0: one (item, 1) pair per query, duplicates    */
/* kept; higher levels: the picks are counted per member).                   */
/*                                                                            */
/* Random bits: Philox4x32-10 with key seed and counter (g, h | level << 12  */
/* | j << 14, stream) where g is the group, h the node's heap index (root 1, */
/* children 2h and 2h + 1; 0 for the alias queries), j the draw's index.    */
/* Binomial deviates: inversion when c * p < 10, else Hoermann's BTRS        */
/* (transformed rejection with squeeze, 1993), both with p <= 1/2 by          */
/* symmetry; log and exp are evaluated here from their series with basic     */
/* IEEE binary64 operations only (compile without contraction), so any      */
/* implementation that follows the same steps gets the same deviates.       */
/* ------------------------------------------------------------------------ */

static double det_ldexp(double x, int e)
{
    while (e > 1000) { x *= 0x1p1000; e -= 1000; }
    while (e < -1000) { x *= 0x1p-1000; e += 1000; }
    {
        union { uint64_t u; double d; } t;
        t.u = (uint64_t)(e + 1023) << 52;
        return x * t.d;
    }
}

/* nearest binary64 to the integer x (ties to even) */
static double det_u128_to_double(u128 x)
{
    int b = bitlen128(x), sh;
    u128 m, rem, half;
    if (b <= 53) return (double)(uint64_t)x;
    sh = b - 53;
    m = x >> sh;
    rem = x & (((u128)1 << sh) - 1);
    half = (u128)1 << (sh - 1);
    if (rem > half || (rem == half && (m & 1))) {
        m += 1;
        if (m >> 53) { m >>= 1; sh += 1; }
    }
    return det_ldexp((double)(uint64_t)m, sh);
}

/* 1/k for k = 1..40, each the nearest binary64 (folded by the compiler)  */
static const double DET_INV[41] = {0.0, 1.0 / 1.0, 1.0 / 2.0, 1.0 / 3.0, 1.0 / 4.0, 1.0 / 5.0, 1.0 / 6.0, 1.0 / 7.0, 1.0 / 8.0, 1.0 / 9.0, 1.0 / 10.0, 1.0 / 11.0, 1.0 / 12.0, 1.0 / 13.0, 1.0 / 14.0, 1.0 / 15.0, 1.0 / 16.0, 1.0 / 17.0, 1.0 / 18.0, 1.0 / 19.0, 1.0 / 20.0, 1.0 / 21.0, 1.0 / 22.0, 1.0 / 23.0, 1.0 / 24.0, 1.0 / 25.0, 1.0 / 26.0, 1.0 / 27.0, 1.0 / 28.0, 1.0 / 29.0, 1.0 / 30.0, 1.0 / 31.0, 1.0 / 32.0, 1.0 / 33.0, 1.0 / 34.0, 1.0 / 35.0, 1.0 / 36.0, 1.0 / 37.0, 1.0 / 38.0, 1.0 / 39.0, 1.0 / 40.0};

/* natural logarithm of x > 0: x = f 2^e with f in [sqrt(1/2), sqrt(2)),   */
/* log f = 2 atanh(s), s = (f - 1) / (f + 1), |s| < 0.172, series to s^25  */
static double det_log(double x)
{
    union { uint64_t u; double d; } t;
    int e;
    double f, s, s2, acc;
    int k;
    t.d = x;
    e = (int)((t.u >> 52) & 0x7FF);
    if (e == 0) { /* subnormal: scale up first */
        t.d = x * 0x1p64;
        e = (int)((t.u >> 52) & 0x7FF) - 64;
    }
    e -= 1023;
    t.u = (t.u & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull;
    f = t.d;
    if (f > 1.4142135623730951) { f = f * 0.5; e += 1; }
    s = (f - 1.0) / (f + 1.0);
    s2 = s * s;
    acc = DET_INV[25];
    for (k = 11; k >= 0; --k) acc = acc * s2 + DET_INV[2 * k + 1];
    return (double)e * 0.6931471805599453 + 2.0 * s * acc;
}

/* log(1 - p) for 0 <= p <= 1/2 without forming 1 - p when p is small:    */
/* -(p + p^2/2 + ... + p^40/40) for p < 1/4, else det_log(1 - p)           */
static double det_log1m(double p)
{
    double acc;
    int k;
    if (p >= 0.25) return det_log(1.0 - p);
    acc = DET_INV[40];
    for (k = 39; k >= 1; --k) acc = acc * p + DET_INV[k];
    return -p * acc;
}

/* e^x: x = k ln2 + r, |r| <= ln2 / 2 (+ rounding), Taylor to r^20 in     */
/* Horner form, each term's 1/j a constant: acc = 1 + (r / j) acc           */
static double det_exp(double x)
{
    double kd, r, acc;
    int k, j;
    if (x < -745.0) return 0.0;
    kd = floor(x / 0.6931471805599453 + 0.5);
    k = (int)kd;
    r = x - kd * 0.6931471805599453;
    acc = 1.0;
    for (j = 20; j >= 1; --j) acc = acc * (r * DET_INV[j]) + 1.0;
    return det_ldexp(acc, k);
}

typedef struct {
    uint32_t key[2], ctr[4];
    uint32_t j;      /* next Philox call of this node */
    uint32_t buf[4];
    int have;        /* uniforms left in buf (0..2) */
} os_rng;

static void os_rng_init(os_rng *r, uint64_t seed, uint64_t stream, uint32_t g, uint32_t h, uint32_t level)
{
    r->key[0] = (uint32_t)seed; r->key[1] = (uint32_t)(seed >> 32);
    r->ctr[0] = g; r->ctr[1] = h | (level << 12);
    r->ctr[2] = (uint32_t)stream; r->ctr[3] = (uint32_t)(stream >> 32);
    r->j = 0;
    r->have = 0;
}

/* uniform in [0, 1): the top 53 bits of a 64-bit word */
static double os_unif(os_rng *r)
{
    uint64_t w;
    if (r->have == 0) {
        uint32_t c[4];
        c[0] = r->ctr[0]; c[1] = r->ctr[1] | (r->j << 14); c[2] = r->ctr[2]; c[3] = r->ctr[3];
        wo_philox4x32_10(c, r->key, r->buf);
        r->j++;
        r->have = 2;
    }
    w = r->have == 2 ? ((uint64_t)r->buf[0] | ((uint64_t)r->buf[1] << 32))
                     : ((uint64_t)r->buf[2] | ((uint64_t)r->buf[3] << 32));
    r->have--;
    return (double)(w >> 11) * 0x1p-53;
}

/* log(k!) : exact product and det_log below 10, Stirling's series above  */
/* (with 1/(k+1) formed once)                                               */
static double det_lfact(uint64_t k)
{
    if (k < 10) {
        double f = 1.0;
        uint64_t i;
        for (i = 2; i <= k; ++i) f *= (double)i;
        return det_log(f);
    } else {
        double z = (double)k + 1.0, iz = 1.0 / z, iz2 = iz * iz;
        double corr = (1.0 / 12.0 - (1.0 / 360.0 - (1.0 / 1260.0 - (1.0 / 1680.0) * iz2) * iz2) * iz2) * iz;
        return ((double)k + 0.5) * det_log(z) - z + 0.5 * det_log(6.283185307179586) + corr;
    }
}

#define OS_MAX_DRAWS (1u << 18)

/* Binomial(n, p) with p = num / den, 0 < num < den; p <= 1/2 by symmetry */
static uint64_t os_binomial(uint64_t n, u128 num, u128 den, os_rng *rng)
{
    int flip = 0;
    double p, q;
    uint64_t x;
    if (2 * num > den) { num = den - num; flip = 1; }
    p = det_u128_to_double(num) / det_u128_to_double(den);
    q = 1.0 - p;
    if ((double)n * p < 10.0) { /* inversion */
        const double s = p / q, a = ((double)n + 1.0) * s, r0 = det_exp((double)n * det_log1m(p));
        for (;;) {
            double u = os_unif(rng), r = r0;
            x = 0;
            while (u > r) {
                u -= r;
                x++;
                /* with r = 0 every later term is 0 and u stays above it until */
                /* x > n: the try fails either way, so it stops here           */
                if (x > n || r == 0.0) { x = n + 1; break; }
                r *= (x <= 40 ? a * DET_INV[x] : a / (double)x) - s;
            }
            if (x <= n) break;
            if (rng->j >= OS_MAX_DRAWS) { x = (uint64_t)((double)n * p); break; }
        }
    } else { /* BTRS */
        const double spq = sqrt((double)n * p * q);
        const double b = 1.15 + 2.53 * spq, a = -0.0873 + 0.0248 * b + 0.01 * p, c = (double)n * p + 0.5;
        const double vr = 0.92 - 4.2 / b, alpha = (2.83 + 5.1 / b) * spq, lpq = det_log(p / q);
        const uint64_t m = (uint64_t)floor(((double)n + 1.0) * p);
        const double h = det_lfact(m) + det_lfact(n - m);
        for (;;) {
            double u = os_unif(rng) - 0.5, v = os_unif(rng), us = 0.5 - fabs(u), kd;
            if (rng->j >= OS_MAX_DRAWS) { x = m; break; }
            kd = floor((2.0 * a / us + b) * u + c);
            if (kd < 0.0 || kd > (double)n) continue;
            x = (uint64_t)kd;
            if (us >= 0.07 && v <= vr) break;
            v = det_log(v * alpha / (a / (us * us) + b));
            if (v <= h - det_lfact(x) - det_lfact(n - x) + ((double)x - (double)m) * lpq) break;
        }
    }
    return flip ? n - x : x;
}

typedef struct {
    int L;
    uint64_t sizes[WO_MAX_LEVELS], offs[WO_MAX_LEVELS], goffs[WO_MAX_LEVELS];
    uint64_t G;
    const uint64_t *q, *tot, *thr, *qp;
    const uint32_t *al;
    uint64_t seed, stream;
    uint32_t *out_item;
    uint64_t *out_count;
    uint64_t cap, nout;
    int overflow;
} os_ctx;

/* exact weight of member m of level `level` */
static u128 os_w(const os_ctx *x, int level, uint64_t m)
{
    return level == 0 ? ld128(x->q + 2 * m) : ld128(x->tot + 2 * (x->goffs[level - 1] + m));
}

static void os_emit(os_ctx *x, uint64_t item, uint64_t c)
{
    if (x->nout >= x->cap) { x->overflow = 1; return; }
    x->out_item[x->nout] = (uint32_t)item;
    x->out_count[x->nout] = c;
    x->nout++;
}

static void os_group(os_ctx *x, int level, uint64_t g, uint64_t c);

static void os_leaf(os_ctx *x, int level, uint64_t member, uint64_t c)
{
    if (level == 0) os_emit(x, member, c);
    else os_group(x, level - 1, member, c);
}

static void os_node(os_ctx *x, int level, uint64_t g, uint64_t base, uint64_t a, uint64_t b, uint64_t h, uint64_t c)
{
    uint64_t mid, i, cl;
    u128 wl = 0, wn = 0;
    if (c == 0) return;
    if (b - a == 1) { os_leaf(x, level, base + a, c); return; }
    mid = a + (b - a) / 2;
    for (i = a; i < b; ++i) {
        const u128 w = os_w(x, level, base + i);
        wn += w;
        if (i < mid) wl += w;
    }
    if (wl == 0) cl = 0;
    else if (wl == wn) cl = c;
    else {
        os_rng r;
        os_rng_init(&r, x->seed, x->stream, (uint32_t)g, (uint32_t)h, (uint32_t)level);
        cl = os_binomial(c, wl, wn, &r);
    }
    os_node(x, level, g, base, a, mid, 2 * h, cl);
    os_node(x, level, g, base, mid, b, 2 * h + 1, c - cl);
}

static void os_group(os_ctx *x, int level, uint64_t g, uint64_t c)
{
    const uint64_t base = g * x->G, N = x->sizes[level];
    const uint64_t ng = (N - base < x->G) ? N - base : x->G;
    if (c == 0) return;
    if (c < 128 && 2 * ng >= c) { /* OS-ND base case: c alias queries */
        uint64_t picks[128], cnt[128], np = 0, t, s;
        for (t = 0; t < c; ++t) {
            uint32_t ctr[4], key[2], o[4];
            uint64_t u, v, r, bkt, pick;
            key[0] = (uint32_t)x->seed; key[1] = (uint32_t)(x->seed >> 32);
            ctr[0] = (uint32_t)g; ctr[1] = ((uint32_t)level << 12) | ((uint32_t)t << 14);
            ctr[2] = (uint32_t)x->stream; ctr[3] = (uint32_t)(x->stream >> 32);
            wo_philox4x32_10(ctr, key, o);
            u = (uint64_t)o[0] | ((uint64_t)o[1] << 32);
            v = (uint64_t)o[2] | ((uint64_t)o[3] << 32);
            r = (uint64_t)(((u128)u * ng) >> 64);
            bkt = x->offs[level] + base + r;
            pick = ((uint64_t)(((u128)v * x->qp[x->goffs[level] + g]) >> 64) < x->thr[bkt]) ? base + r : x->al[bkt];
            if (level == 0) { os_emit(x, pick, 1); continue; }
            for (s = 0; s < np && picks[s] != pick; ++s) {}
            if (s == np) { picks[np] = pick; cnt[np] = 0; np++; }
            cnt[s]++;
        }
        /* higher levels: each picked member once, with its count, in pick order */
        for (s = 0; s < np; ++s) os_group(x, level - 1, picks[s], cnt[s]);
        return;
    }
    os_node(x, level, g, base, 0, ng, 1, c);
}

/* Writes up to cap (item, count) pairs; returns the number written, or      */
/* ~0 when cap was too small.  The table is wo_2lvl_build's output plus the  */
/* items' exact weights q.                                                    */
uint64_t wo_os_nd(uint64_t n, uint64_t G, const uint64_t *q, const uint64_t *thr, const uint32_t *al,
                  const uint64_t *qp, const uint64_t *tot, uint64_t k, uint64_t seed, uint64_t stream,
                  uint32_t *out_item, uint64_t *out_count, uint64_t cap)
{
    os_ctx x;
    int l;
    uint64_t o = 0, go = 0;
    memset(&x, 0, sizeof(x));
    x.L = wo_2lvl_levels(n, G, x.sizes);
    for (l = 0; l < x.L; ++l) { x.offs[l] = o; x.goffs[l] = go; o += x.sizes[l]; go += (x.sizes[l] + G - 1) / G; }
    x.G = G; x.q = q; x.tot = tot; x.thr = thr; x.qp = qp; x.al = al;
    x.seed = seed; x.stream = stream;
    x.out_item = out_item; x.out_count = out_count; x.cap = cap;
    os_group(&x, x.L - 1, 0, k);
    return x.overflow ? ~(uint64_t)0 : x.nout;
}

/* One deviate, for the distribution tests of the binomial generator. */
uint64_t wo_binomial(uint64_t n, uint64_t num, uint64_t den, uint64_t seed, uint64_t node)
{
    os_rng r;
    os_rng_init(&r, seed, 0, (uint32_t)node, (uint32_t)(node >> 32) & 0xFFFu, 0);
    if (num == 0) return 0;
    if (num >= den) return n;
    return os_binomial(n, num, den, &r);
}

double wo_det_log(double x) { return det_log(x); }
double wo_det_log1m(double p) { return det_log1m(p); }
double wo_det_lfact(uint64_t k) { return det_lfact(k); }
double wo_det_u128_to_double(uint64_t lo, uint64_t hi) { return det_u128_to_double(((u128)hi << 64) | lo); }
double wo_det_ldexp(double x, int e) { return det_ldexp(x, e); }
double wo_det_exp(double x) { return det_exp(x); }

/* ------------------------------------------------------------------------ */
/* PSA+ (Sec. 4.2 "Performance Optimization in Practice"): each tile of T    */
/* consecutive items (the PE's allotment) first runs Alg. 2 on its own items */
/* in the global units (capacity Q, item i weighs n q_i), stopping when the  */
/* next light or the next heavy item would lie outside the tile; the items   */
/* left over -- the heavy item current at the stop with its unassigned       */
/* residual, every other unassigned item with its full weight -- form, in    */
/* index order, a list on which Alg. 2 (equivalently PSA) builds the rest.   */
/* Reading: a heavy item is packed once its residual is <= Q, which needs    */
/* the next heavy item of the tile as its alias; a light item needs a        */
/* current heavy item.                                                        */
/* ------------------------------------------------------------------------ */

/* Alg. 2 on m items of scaled weights v (two words each; the capacity is  */
/* Q and sum v = m Q), writing bucket masses and aliases at idx[] of the     */
/* full table.                                                                */
static int sweep_scaled(uint64_t m, const uint64_t *v, const uint32_t *idx, u128 Q, uint64_t *bw, uint32_t *al)
{
    uint64_t i = 0, j = 0, k;
    u128 w;
#define V(t) ld128(v + 2 * (t))
    while (i < m && V(i) > Q) ++i;           /* first light */
    while (j < m && V(j) <= Q) ++j;          /* first heavy */
    if (j == m) {                            /* all full */
        for (k = 0; k < m; ++k) {
            if (V(k) != Q) return WO_EINTERNAL;
            put(bw, al, idx[k], Q, idx[k]);
        }
        return WO_OK;
    }
    w = V(j);
    while (j < m) {
        if (w > Q) {
            if (i >= m) return WO_EINTERNAL;
            put(bw, al, idx[i], V(i), idx[j]);
            w = (w + V(i)) - Q;
            do { ++i; } while (i < m && V(i) > Q);
        } else {
            uint64_t jn = j + 1;
            while (jn < m && V(jn) <= Q) ++jn;
            put(bw, al, idx[j], w, jn < m ? idx[jn] : idx[j]);
            if (jn < m) w = (w + V(jn)) - Q;
            else if (w != Q) return WO_EINTERNAL;
            j = jn;
        }
    }
    for (; i < m; ) {
        if (V(i) != Q) return WO_EINTERNAL;
        put(bw, al, idx[i], Q, idx[i]);
        do { ++i; } while (i < m && V(i) > Q);
    }
#undef V
    return WO_OK;
}

int wo_psa_plus(uint64_t n, const uint64_t *q, const uint64_t *Qin, uint64_t T, uint64_t *bw, uint32_t *al,
                uint64_t *n_left)
{
    wo_in in = { n, q, ld128(Qin) };
    const u128 Q = in.Q;
    uint64_t *lv = (uint64_t *)malloc(2 * (n + 1) * sizeof(uint64_t));
    uint32_t *lidx = (uint32_t *)malloc((n + 1) * sizeof(uint32_t));
    uint64_t m = 0, t0, b;
    int rc;
    if (!lv || !lidx || T == 0) { free(lv); free(lidx); return WO_EINVAL; }
    for (t0 = 0; t0 < n; t0 += T) {
        const uint64_t t1 = (n - t0 < T) ? n : t0 + T;
        uint64_t i = t0, j = t0, k, cur = t1; /* cur: the heavy item current at the stop */
        u128 w = 0;
        unsigned char *done = (unsigned char *)calloc(t1 - t0, 1);
        if (!done) { free(lv); free(lidx); return WO_EINVAL; }
        while (i < t1 && !is_light(&in, i)) ++i;
        while (j < t1 && is_light(&in, j)) ++j;
        if (j < t1) {
            w = nq(&in, j);
            for (;;) {
                if (w > Q) { /* needs a light */
                    if (i >= t1) break;
                    put(bw, al, i, nq(&in, i), j);
                    done[i - t0] = 1;
                    w = (w + nq(&in, i)) - Q;
                    do { ++i; } while (i < t1 && !is_light(&in, i));
                } else { /* pack heavy j: needs the next heavy */
                    uint64_t jn = j + 1;
                    while (jn < t1 && is_light(&in, jn)) ++jn;
                    if (jn >= t1) break;
                    put(bw, al, j, w, jn);
                    done[j - t0] = 1;
                    w = (w + nq(&in, jn)) - Q;
                    j = jn;
                }
            }
            cur = j;
        }
        for (k = t0; k < t1; ++k) {
            if (done[k - t0]) continue;
            st128(lv + 2 * m, k == cur ? w : nq(&in, k));
            lidx[m] = (uint32_t)k;
            ++m;
        }
        free(done);
    }
    rc = sweep_scaled(m, lv, lidx, Q, bw, al);
    free(lv);
    free(lidx);
    if (rc) return rc;
    for (b = 0; b < n; ++b)
        if (ld128(bw + 2 * b) == Q) al[b] = (uint32_t)b;
    if (n_left) *n_left = m;
    return WO_OK;
}
