// wrs_osnd.cuh -- output-sensitive sampling with replacement, OS-ND variant
// (wrs_table2_sample_os of include/wrs.h).  Included by wrs.cu only, after
// wrs_twolevel.cuh.
//
// Sec. 5 "Output Sensitive Sampling With Replacement" with the experiments'
// OS-ND optimisation (Sec. 10 "Optimizations": tree descent aborted for fewer
// than 128 samples from at least half as many items, no deduplication),
// over the two-level table: within a group a complete binary tree over its
// members (node [a, b) splits at a + (b - a) / 2) is the divide-and-conquer
// tree, whose leaves are items (level 0) or the groups one level down.  A node
// with c samples gives Binomial(c, W_left / W_node) of them to its left child;
// a group receiving c < 128 samples from at least c/2 members draws them as c
// queries of its alias table.  The output is a list of (item, count) pairs:
// one per item reached by the descent, one per alias query at level 0.
//
// Levels are processed top down: the groups that received samples form a
// device-resident frontier (group, count), one block per entry.  Random bits:
// Philox4x32-10 keyed by the seed, counter (g, h | level << 12 | j << 14,
// stream) with g the group, h the node's heap index (0 for the alias
// queries) and j the draw's index, so results do not depend on the order in
// which blocks run.  Binomial deviates: inversion when c p < 10, else
// Hoermann's transformed rejection with squeeze (BTRS), p <= 1/2 by symmetry;
// log and exp come from their series in basic binary64 operations, and this
// library is compiled without multiply-add contraction, so the deviates are a
// function of the random bits alone.
#pragma once

namespace wrs {

constexpr uint32_t kOsBase = 128;       // base case below this many samples
constexpr uint32_t kOsMaxDraws = 1u << 18;

__device__ __forceinline__ double os_ldexp(double x, int e)
{
    while (e > 1000) { x *= 0x1p1000; e -= 1000; }
    while (e < -1000) { x *= 0x1p-1000; e += 1000; }
    return x * __longlong_as_double((long long)((uint64_t)(e + 1023) << 52));
}

// nearest binary64 to x (ties to even)
__device__ __forceinline__ double os_u128_to_double(u128 x)
{
    const int b = bitlen128(x);
    if (b <= 53) return (double)(uint64_t)x;
    int sh = b - 53;
    u128 m = x >> sh;
    const u128 rem = x & (((u128)1 << sh) - 1), half = (u128)1 << (sh - 1);
    if (rem > half || (rem == half && (m & 1))) {
        m += 1;
        if (m >> 53) { m >>= 1; sh += 1; }
    }
    return os_ldexp((double)(uint64_t)m, sh);
}

// 1/k for k = 1..40, each the nearest binary64 (folded by the compiler)
__device__ const double kOsInv[41] = {0.0, 1.0 / 1.0, 1.0 / 2.0, 1.0 / 3.0, 1.0 / 4.0, 1.0 / 5.0, 1.0 / 6.0, 1.0 / 7.0, 1.0 / 8.0, 1.0 / 9.0, 1.0 / 10.0, 1.0 / 11.0, 1.0 / 12.0, 1.0 / 13.0, 1.0 / 14.0, 1.0 / 15.0, 1.0 / 16.0, 1.0 / 17.0, 1.0 / 18.0, 1.0 / 19.0, 1.0 / 20.0, 1.0 / 21.0, 1.0 / 22.0, 1.0 / 23.0, 1.0 / 24.0, 1.0 / 25.0, 1.0 / 26.0, 1.0 / 27.0, 1.0 / 28.0, 1.0 / 29.0, 1.0 / 30.0, 1.0 / 31.0, 1.0 / 32.0, 1.0 / 33.0, 1.0 / 34.0, 1.0 / 35.0, 1.0 / 36.0, 1.0 / 37.0, 1.0 / 38.0, 1.0 / 39.0, 1.0 / 40.0};

// natural logarithm of x > 0: x = f 2^e with f in [sqrt(1/2), sqrt(2)),
// log f = 2 atanh(s), s = (f - 1) / (f + 1), series to s^25
__device__ __forceinline__ double os_log(double x)
{
    uint64_t u = (uint64_t)__double_as_longlong(x);
    int e = (int)((u >> 52) & 0x7FF);
    if (e == 0) {
        u = (uint64_t)__double_as_longlong(x * 0x1p64);
        e = (int)((u >> 52) & 0x7FF) - 64;
    }
    e -= 1023;
    double f = __longlong_as_double((long long)((u & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull));
    if (f > 1.4142135623730951) { f = f * 0.5; e += 1; }
    const double s = (f - 1.0) / (f + 1.0), s2 = s * s;
    double acc = 1.0 / 25.0;
#pragma unroll
    for (int k = 11; k >= 0; --k) acc = acc * s2 + 1.0 / (double)(2 * k + 1); // constants once unrolled
    return (double)e * 0.6931471805599453 + 2.0 * s * acc;
}

// log(1 - p) for 0 <= p <= 1/2 without forming 1 - p when p is small:
// -(p + p^2/2 + ... + p^40/40) for p < 1/4, else os_log(1 - p)
__device__ __forceinline__ double os_log1m(double p)
{
    if (p >= 0.25) return os_log(1.0 - p);
    double acc = 1.0 / 40.0;
#pragma unroll
    for (int k = 39; k >= 1; --k) acc = acc * p + 1.0 / (double)k; // constants once unrolled
    return -p * acc;
}

// e^x: x = k ln2 + r, Taylor series of e^r to r^20 in Horner form with each
// term's 1/j a constant: acc = 1 + (r / j) acc
__device__ __forceinline__ double os_exp(double x)
{
    if (x < -745.0) return 0.0;
    const double kd = floor(x / 0.6931471805599453 + 0.5);
    const double r = x - kd * 0.6931471805599453;
    double acc = 1.0;
#pragma unroll
    for (int j = 20; j >= 1; --j) acc = acc * (r * (1.0 / (double)j)) + 1.0;
    return os_ldexp(acc, (int)kd);
}

struct OsRng {
    uint32_t key0, key1, c0, c1, c2, c3;
    uint32_t j;
    uint32_t buf[4];
    int have;
};

__device__ __forceinline__ void os_rng_init(OsRng &r, uint64_t seed, uint64_t stream, uint32_t g, uint32_t h,
                                            uint32_t level)
{
    r.key0 = (uint32_t)seed; r.key1 = (uint32_t)(seed >> 32);
    r.c0 = g; r.c1 = h | (level << 12); r.c2 = (uint32_t)stream; r.c3 = (uint32_t)(stream >> 32);
    r.j = 0;
    r.have = 0;
}

// uniform in [0, 1): the top 53 bits of a 64-bit word
__device__ __forceinline__ double os_unif(OsRng &r)
{
    if (r.have == 0) {
        P4 c;
        c.x0 = r.c0; c.x1 = r.c1 | (r.j << 14); c.x2 = r.c2; c.x3 = r.c3;
        const P4 o = philox4x32_10(c, r.key0, r.key1);
        r.buf[0] = o.x0; r.buf[1] = o.x1; r.buf[2] = o.x2; r.buf[3] = o.x3;
        r.j++;
        r.have = 2;
    }
    const uint64_t w = r.have == 2 ? ((uint64_t)r.buf[0] | ((uint64_t)r.buf[1] << 32))
                                   : ((uint64_t)r.buf[2] | ((uint64_t)r.buf[3] << 32));
    r.have--;
    return (double)(w >> 11) * 0x1p-53;
}

// log(k!): exact product and os_log below 10, Stirling's series above
// (with 1/(k+1) formed once); hl2pi = 0.5 * os_log(2 pi), passed in
__device__ __forceinline__ double os_lfact(uint64_t k, double hl2pi)
{
    if (k < 10) {
        double f = 1.0;
        for (uint64_t i = 2; i <= k; ++i) f *= (double)i;
        return os_log(f);
    }
    const double z = (double)k + 1.0, iz = 1.0 / z, iz2 = iz * iz;
    const double corr = (1.0 / 12.0 - (1.0 / 360.0 - (1.0 / 1260.0 - (1.0 / 1680.0) * iz2) * iz2) * iz2) * iz;
    return ((double)k + 0.5) * os_log(z) - z + hl2pi + corr;
}

// Binomial(n, num / den), 0 < num < den
__device__ uint64_t os_binomial(uint64_t n, u128 num, u128 den, OsRng &rng)
{
    bool flip = false;
    if (2 * num > den) { num = den - num; flip = true; }
    const double p = os_u128_to_double(num) / os_u128_to_double(den), q = 1.0 - p;
    uint64_t x;
    if ((double)n * p < 10.0) { // inversion
        const double s = p / q, a = ((double)n + 1.0) * s, r0 = os_exp((double)n * os_log1m(p));
        for (;;) {
            double u = os_unif(rng), r = r0;
            x = 0;
            // once the pmf terms have underflowed to 0 the try cannot end
            // before x > n: it is abandoned at once (same outcome, same draws)
            while (u > r) {
                u -= r;
                x++;
                if (x > n || r == 0.0) { x = n + 1; break; }
                r *= (x <= 40 ? a * kOsInv[x] : a / (double)x) - s;
            }
            if (x <= n) break;
            if (rng.j >= kOsMaxDraws) { x = (uint64_t)((double)n * p); break; }
        }
    } else { // BTRS
        const double spq = sqrt((double)n * p * q);
        const double b = 1.15 + 2.53 * spq, a = -0.0873 + 0.0248 * b + 0.01 * p, c = (double)n * p + 0.5;
        const double vr = 0.92 - 4.2 / b, alpha = (2.83 + 5.1 / b) * spq;
        const uint64_t m = (uint64_t)floor(((double)n + 1.0) * p);
        // log(p/q), log(m!) + log((n-m)!) and 0.5 log(2 pi) are needed only when
        // the quick acceptance test fails: formed then, once (same values)
        double lpq = 0.0, h = 0.0, hl2pi = 0.0;
        bool slow = false;
        for (;;) {
            const double u = os_unif(rng) - 0.5;
            double v = os_unif(rng);
            if (rng.j >= kOsMaxDraws) { x = m; break; }
            const double us = 0.5 - fabs(u);
            const double kd = floor((2.0 * a / us + b) * u + c);
            if (kd < 0.0 || kd > (double)n) continue;
            x = (uint64_t)kd;
            if (us >= 0.07 && v <= vr) break;
            if (!slow) {
                hl2pi = 0.5 * os_log(6.283185307179586);
                lpq = os_log(p / q);
                h = os_lfact(m, hl2pi) + os_lfact(n - m, hl2pi);
                slow = true;
            }
            v = os_log(v * alpha / (a / (us * us) + b));
            if (v <= h - os_lfact(x, hl2pi) - os_lfact(n - x, hl2pi) + ((double)x - (double)m) * lpq) break;
        }
    }
    return flip ? n - x : x;
}

struct OsNode {       // a node of a group's divide-and-conquer tree with samples
    uint64_t c;
    uint16_t a, b, h, pad;
};

struct OsSmem {
    u128 pre[kTile + 1];      // prefix sums of the members' exact weights
    OsNode node[2][kTile];    // nodes of the current and the next depth
    u128 red[kWarps];
    U2 scan[kWarps];
    uint32_t nnode[2];
    uint32_t pick[kOsBase];
    uint32_t cnt[kOsBase];
};

struct OsFront {      // frontier entry: a group of some level and its samples
    uint64_t c;
    uint32_t g, pad;
};

// Pairs past the caller's capacity are counted but not written.
__device__ __forceinline__ void os_emit(uint32_t *items, uint64_t *counts, unsigned long long *nout,
                                        uint64_t cap, uint32_t item, uint64_t c)
{
    const unsigned long long at = atomicAdd(nout, 1ull);
    if (at < cap) { items[at] = item; counts[at] = c; }
}

// The top frontier (the single top group with all k samples) and zeroed counters.
__global__ void k_os_init(OsFront *top, unsigned long long *ctr, uint32_t top_level, unsigned long long *nout,
                          uint64_t k)
{
    if (threadIdx.x < 8) ctr[threadIdx.x] = threadIdx.x == top_level ? 1ull : 0ull;
    if (threadIdx.x == 0) {
        OsFront f;
        f.c = k; f.g = 0; f.pad = 0;
        *top = f;
        *nout = 0;
    }
}

// A group of the level below receiving c samples: level-0 groups that will
// take the base case go to their own list (drawn by k_os_small0, a warp per
// group); all others to the next frontier.
__device__ __forceinline__ void os_push(uint32_t level, uint32_t member, uint64_t c, OsFront *next,
                                        unsigned long long *nnext, OsFront *next_small,
                                        unsigned long long *nnext_small, uint64_t N_next)
{
    OsFront f;
    f.c = c; f.g = member; f.pad = 0;
    const uint64_t ngn = min((uint64_t)kTile, N_next - (uint64_t)member * kTile);
    if (level == 1 && c < kOsBase && 2 * ngn >= c) next_small[atomicAdd(nnext_small, 1ull)] = f;
    else next[atomicAdd(nnext, 1ull)] = f;
}

// One frontier entry per block iteration.  SRC as k2_group.
template <int SRC>
__global__ void __launch_bounds__(kThreads) k_os_level(const void *__restrict__ src, int vec, uint64_t N,
                                                       uint32_t level, const uint4 *__restrict__ buckets,
                                                       const GroupRec *__restrict__ groups, DevHeader *hdr,
                                                       const OsFront *__restrict__ front,
                                                       const unsigned long long *__restrict__ nfront,
                                                       OsFront *__restrict__ next, unsigned long long *nnext,
                                                       OsFront *__restrict__ next_small,
                                                       unsigned long long *nnext_small, uint64_t N_next,
                                                       uint32_t *__restrict__ items, uint64_t *__restrict__ counts,
                                                       unsigned long long *nout, uint64_t cap, uint64_t seed,
                                                       uint64_t stream)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    OsSmem &S = *reinterpret_cast<OsSmem *>(smem_raw);
    if (block_stopped(hdr)) return;
    const int beta = hdr->beta;
    const uint64_t nf = *nfront;
    for (uint64_t e = blockIdx.x; e < nf; e += gridDim.x) {
        const OsFront F = front[e];
        const uint32_t g = F.g;
        const uint64_t c = F.c, base = (uint64_t)g * kTile;
        const uint32_t ng = (uint32_t)min((uint64_t)kTile, N - base);
        if (c < kOsBase && 2 * (uint64_t)ng >= c) { // base case: c alias queries
            const uint64_t qp = groups[g].qp;
            uint32_t pick = 0;
            if (threadIdx.x < c) {
                P4 ctr;
                ctr.x0 = g; ctr.x1 = (level << 12) | ((uint32_t)threadIdx.x << 14);
                ctr.x2 = (uint32_t)stream; ctr.x3 = (uint32_t)(stream >> 32);
                const P4 o = philox4x32_10(ctr, (uint32_t)seed, (uint32_t)(seed >> 32));
                const uint64_t u = o.x0 | ((uint64_t)o.x1 << 32), v = o.x2 | ((uint64_t)o.x3 << 32);
                const uint64_t r = __umul64hi(u, ng);
                const uint4 bk = buckets[base + r];
                const uint64_t thr = bk.x | ((uint64_t)bk.y << 32);
                pick = (__umul64hi(v, qp) < thr) ? (uint32_t)(base + r) : bk.z;
                if (level == 0) os_emit(items, counts, nout, cap, pick, 1);
                else S.pick[threadIdx.x] = pick;
            }
            if (level > 0) { // count the picks per member, one frontier entry each
                __syncthreads();
                if (threadIdx.x == 0) {
                    uint32_t np = 0;
                    for (uint32_t t = 0; t < (uint32_t)c; ++t) {
                        uint32_t s = 0;
                        while (s < np && S.pick[s] != S.pick[t]) ++s;
                        if (s == np) { S.pick[np] = S.pick[t]; S.cnt[np] = 0; ++np; }
                        ++S.cnt[s];
                    }
                    for (uint32_t s = 0; s < np; ++s)
                        os_push(level, S.pick[s], S.cnt[s], next, nnext, next_small, nnext_small, N_next);
                }
                __syncthreads();
            }
            continue;
        }
        // descent: prefix sums of the members' exact weights
        const uint64_t first = base + (uint64_t)threadIdx.x * kItems;
        u128 q[kItems];
        if (SRC == 2) {
            const uint4 *m = reinterpret_cast<const uint4 *>(src);
#pragma unroll
            for (int k = 0; k < kItems; ++k) {
                const uint4 v = first + k < N ? __ldg(m + first + k) : make_uint4(0, 0, 0, 0);
                q[k] = mk128(v.x | ((uint64_t)v.y << 32), v.z | ((uint64_t)v.w << 32));
            }
        } else {
            uint32_t x[kItems];
            load_items(static_cast<const uint32_t *>(src), N, vec, first, x);
#pragma unroll
            for (int k = 0; k < kItems; ++k) q[k] = first + k < N ? q_of(x[k], SRC == 1, beta) : (u128)0;
        }
        u128 part = 0;
#pragma unroll
        for (int k = 0; k < kItems; ++k) part += q[k];
        U2 tot;
        const U2 ex = block_exclusive_scan2(U2{part, 0}, tot, S.scan);
        {
            u128 run = ex.a;
#pragma unroll
            for (int k = 0; k < kItems; ++k) {
                S.pre[threadIdx.x * kItems + k] = run;
                run += q[k];
            }
            if (threadIdx.x == kThreads - 1) S.pre[kTile] = run;
        }
        if (threadIdx.x == 0) {
            OsNode r;
            r.c = c; r.a = 0; r.b = (uint16_t)ng; r.h = 1; r.pad = 0;
            S.node[0][0] = r;
            S.nnode[0] = 1;
            S.nnode[1] = 0;
        }
        __syncthreads();
        int cur = 0;
        while (S.nnode[cur] > 0) {
            const uint32_t nn = S.nnode[cur];
            for (uint32_t i = threadIdx.x; i < nn; i += kThreads) {
                const OsNode d = S.node[cur][i];
                if (d.b - d.a == 1) { // a leaf: an item, or a group one level down
                    if (level == 0) os_emit(items, counts, nout, cap, (uint32_t)(base + d.a), d.c);
                    else os_push(level, (uint32_t)(base + d.a), d.c, next, nnext, next_small, nnext_small, N_next);
                    continue;
                }
                const uint32_t mid = d.a + (d.b - d.a) / 2;
                const u128 wl = S.pre[mid] - S.pre[d.a], wn = S.pre[d.b] - S.pre[d.a];
                uint64_t cl;
                if (wl == 0) cl = 0;
                else if (wl == wn) cl = d.c;
                else {
                    OsRng r;
                    os_rng_init(r, seed, stream, g, d.h, level);
                    cl = os_binomial(d.c, wl, wn, r);
                }
                if (cl) {
                    OsNode l;
                    l.c = cl; l.a = d.a; l.b = (uint16_t)mid; l.h = (uint16_t)(2 * d.h); l.pad = 0;
                    S.node[cur ^ 1][atomicAdd(&S.nnode[cur ^ 1], 1u)] = l;
                }
                if (d.c - cl) {
                    OsNode rr;
                    rr.c = d.c - cl; rr.a = (uint16_t)mid; rr.b = d.b; rr.h = (uint16_t)(2 * d.h + 1); rr.pad = 0;
                    S.node[cur ^ 1][atomicAdd(&S.nnode[cur ^ 1], 1u)] = rr;
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) S.nnode[cur] = 0;
            cur ^= 1;
            __syncthreads();
        }
        __syncthreads();
    }
}

// Level-0 groups with fewer than 128 samples (and at least half as many
// members): a warp per group draws them as alias queries, one (item, 1) pair
// each, with one output atomic per 32 queries.
__global__ void __launch_bounds__(256) k_os_small0(uint64_t N, const uint4 *__restrict__ buckets,
                                                   const GroupRec *__restrict__ groups, const DevHeader *hdr,
                                                   const OsFront *__restrict__ front,
                                                   const unsigned long long *__restrict__ nfront,
                                                   uint32_t *__restrict__ items, uint64_t *__restrict__ counts,
                                                   unsigned long long *nout, uint64_t cap, uint64_t seed,
                                                   uint64_t stream)
{
    // one read per warp: its lanes leave together (warp collectives follow)
    if (__shfl_sync(0xFFFFFFFFu, *(volatile const uint32_t *)&hdr->status, 0)) return;
    const uint64_t nf = *nfront;
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t e = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < nf; e += nwarps) {
        const OsFront F = front[e];
        const uint64_t base = (uint64_t)F.g * kTile;
        const uint64_t ng = min((uint64_t)kTile, N - base);
        const uint64_t qp = groups[F.g].qp;
        for (uint32_t t0 = 0; t0 < (uint32_t)F.c; t0 += 32) {
            const uint32_t t = t0 + lane;
            const bool act = t < (uint32_t)F.c;
            uint32_t pick = 0;
            if (act) {
                P4 ctr;
                ctr.x0 = F.g; ctr.x1 = t << 14; // level 0, heap index 0
                ctr.x2 = (uint32_t)stream; ctr.x3 = (uint32_t)(stream >> 32);
                const P4 o = philox4x32_10(ctr, (uint32_t)seed, (uint32_t)(seed >> 32));
                const uint64_t u = o.x0 | ((uint64_t)o.x1 << 32), v = o.x2 | ((uint64_t)o.x3 << 32);
                const uint64_t r = __umul64hi(u, ng);
                const uint4 bk = buckets[base + r];
                const uint64_t thr = bk.x | ((uint64_t)bk.y << 32);
                pick = (__umul64hi(v, qp) < thr) ? (uint32_t)(base + r) : bk.z;
            }
            const uint32_t m = __ballot_sync(0xFFFFFFFFu, act);
            unsigned long long at = 0;
            if (lane == 0) at = atomicAdd(nout, (unsigned long long)__popc(m));
            at = __shfl_sync(0xFFFFFFFFu, at, 0) + lane; // the active lanes are a prefix
            if (act && at < cap) { items[at] = pick; counts[at] = 1; }
        }
    }
}

} // namespace wrs

namespace {

bool g_os_attr_done[64];

wrs_status os_attributes()
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return WRS_EDEVICE;
    if (g_os_attr_done[dev]) return WRS_OK;
    const int bytes = (int)sizeof(OsSmem);
    cudaError_t e = cudaFuncSetAttribute(k_os_level<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_os_level<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_os_level<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return WRS_EDEVICE;
    g_os_attr_done[dev] = true;
    return WRS_OK;
}

} // namespace

extern "C" {

wrs_status wrs_table2_sample_os(wrs_table2 *t, const void *d_weights, wrs_dtype dtype, uint64_t k, uint64_t seed,
                                uint64_t stream_id, uint32_t *d_items, uint64_t *d_counts, uint64_t capacity,
                                uint64_t *d_npairs, void *stream)
{
    if (!t || t->n == 0 || !d_weights || !d_npairs) return WRS_EINVAL;
    if ((dtype == WRS_F32) != (t->f32 != 0) || (dtype != WRS_U32 && dtype != WRS_F32)) return WRS_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_weights) % 4) != 0) return WRS_EINVAL;
    if (capacity > 0 && (!d_items || !d_counts)) return WRS_EINVAL;
    if (t->host_status > 0) return (wrs_status)t->host_status;
    wrs_status st = os_attributes();
    if (st != WRS_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const Levels &v = t->lv;
    const uint64_t ngroups = levels_groups(v);
    const uint64_t need = ngroups + (v.size[0] + kTile - 1) / kTile + 2; // + the level-0 small list
    if (t->os_cap < need) { // frontier buffers: one entry per group of every level, and counters
        if (t->os_front) { cudaDeviceSynchronize(); cudaFree(t->os_front); t->os_front = nullptr; t->os_cap = 0; }
        cudaError_t e = cudaMalloc(&t->os_front, need * sizeof(OsFront) + 8 * sizeof(unsigned long long));
        if (e != cudaSuccess) return cuda_err(e);
        t->os_cap = need;
    }
    OsFront *fr = static_cast<OsFront *>(t->os_front);
    OsFront *small0 = fr + ngroups; // level-0 groups for the base case
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(fr + t->os_cap); // [level] frontier sizes, [4] small0
    k_os_init<<<1, 32, 0, s>>>(fr + v.goff[v.L - 1], ctr, v.L - 1, reinterpret_cast<unsigned long long *>(d_npairs),
                               k);
    if (k == 0) return launch_err();
    const size_t smem = sizeof(OsSmem);
    const uint32_t cap_blocks = (uint32_t)sm_count() * 2;
    for (int l = (int)v.L - 1; l >= 0; --l) {
        const uint64_t lgroups = (v.size[l] + kTile - 1) / kTile;
        const uint32_t blocks = (uint32_t)(lgroups < cap_blocks ? lgroups : cap_blocks);
        const OsFront *cur = fr + v.goff[l];
        OsFront *nxt = l > 0 ? fr + v.goff[l - 1] : nullptr;
        unsigned long long *nnext = l > 0 ? ctr + (l - 1) : ctr + 7;
        const uint64_t N_next = l > 0 ? v.size[l - 1] : 0;
        const uint4 *bk = t->buckets + v.off[l];
        const GroupRec *gr = t->groups + v.goff[l];
        unsigned long long *nout = reinterpret_cast<unsigned long long *>(d_npairs);
        if (l == 0) {
            const int vec = (reinterpret_cast<uintptr_t>(d_weights) % 16) == 0;
            k_os_small0<<<(uint32_t)sm_count() * 8, 256, 0, s>>>(v.size[0], bk, gr, t->hdr, small0, ctr + 4, d_items,
                                                                 d_counts, nout, capacity, seed, stream_id);
            if (t->f32) k_os_level<1><<<blocks, kThreads, smem, s>>>(d_weights, vec, v.size[0], 0, bk, gr, t->hdr, cur, ctr + 0, nxt, nnext, small0, ctr + 4, N_next, d_items, d_counts, nout, capacity, seed, stream_id);
            else k_os_level<0><<<blocks, kThreads, smem, s>>>(d_weights, vec, v.size[0], 0, bk, gr, t->hdr, cur, ctr + 0, nxt, nnext, small0, ctr + 4, N_next, d_items, d_counts, nout, capacity, seed, stream_id);
        } else {
            const uint64_t *meta_in = t->meta + 2 * (v.off[l] - t->n);
            k_os_level<2><<<blocks, kThreads, smem, s>>>(meta_in, 1, v.size[l], (uint32_t)l, bk, gr, t->hdr, cur, ctr + l, nxt, nnext, small0, ctr + 4, N_next, d_items, d_counts, nout, capacity, seed, stream_id);
        }
    }
    return launch_err();
}

} // extern "C"
