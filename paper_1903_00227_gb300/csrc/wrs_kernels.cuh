// wrs_kernels.cuh -- the kernels of the build and of the query.  Included by
// wrs.cu only.
//
// Build (alias table of n weights; Alg. 3 "PSA", Sec. 4.2, producing the
// table of Alg. 2, Sec. 4.1, bucket for bucket):
//   k_stats, k_stats_combine  W := sum w_i, exactly (opening line of Alg. 3)
//   k_classify  per 2048-weight tile: light/heavy classification (Alg. 3's
//               two traversals) and the tile's light and heavy weight sums
//               and counts (Sec. 4.2.2 "Using Block-Wise Prefix Sums": tiles
//               play the role of the blocks), plus the offsets of the tile's
//               members of a class that has at most 32 of them
//   k_tilescan  inclusive prefix of the tile aggregates: a single-pass scan
//               with decoupled look-back between thread blocks
//   k_split     per tile, Alg. 3's split search on the tile prefix sums
//   k_sweep     per tile, the buckets of the tile's own items (Alg. 3's pack)
// Query:
//   k_sample    k alias queries (Sec. 2.2; Sec. 5 Cor. "kWR"), branchless
//               selection between bucket and alias (Sec. 10, "Optimizations").
//
// Units (exact): q_i is the integer weight, Q = sum q_i, a bucket holds Q and
// item i weighs n*q_i.  With the light list l and heavy list h in index
// order, light x (0-based rank) has key D[x] = x*Q - n*(q of lights before
// x) and heavy y has key E[y] = n*(q of heavies up to y) - (y+1)*Q.  Alg. 2
// packs heavy y before light x iff E[y] <= D[x] (its residual then fits).
// Hence the bucket of light x holds n*q with alias the first heavy y with
// E[y] > D[x], and the bucket of heavy y holds Q - (D[x] - E[y]) where x is
// the first light with D[x] >= E[y]; its alias is the next heavy item in
// index order (a full bucket points to itself).  Both are the split of
// Alg. 3 taken at one item: the state of Alg. 2 when that item is packed.
#pragma once

#include "wrs_device.cuh"

namespace wrs {

// ------------------------------------------------------------- loading
__device__ __forceinline__ void load_items(const uint32_t *__restrict__ w, uint64_t n, int vec,
                                           uint64_t first, uint32_t (&x)[kItems])
{
    if (vec && first + kItems <= n) {
        const uint4 *p = reinterpret_cast<const uint4 *>(w + first);
#pragma unroll
        for (int j = 0; j < kItems / 4; ++j) {
            uint4 v = __ldg(p + j);
            x[4 * j + 0] = v.x; x[4 * j + 1] = v.y; x[4 * j + 2] = v.z; x[4 * j + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kItems; ++k) x[k] = (first + k < n) ? __ldg(w + first + k) : 0u;
    }
}

__device__ __forceinline__ TileSum load_prefix(const TileSum *incl, uint32_t b)
{
    TileSum p;
    if (b == 0) {
        p.l_lo = p.l_hi = p.h_lo = p.h_hi = 0;
        p.cl = 0;
    } else {
        const uint4 *src = reinterpret_cast<const uint4 *>(incl + (b - 1));
        uint4 a = __ldcg(src), c = __ldcg(src + 1), d = __ldcg(src + 2);
        p.l_lo = a.x | ((uint64_t)a.y << 32); p.l_hi = a.z | ((uint64_t)a.w << 32);
        p.h_lo = c.x | ((uint64_t)c.y << 32); p.h_hi = c.z | ((uint64_t)c.w << 32);
        p.cl = d.x;
    }
    return p;
}

// ------------------------------------------------------------ k_stats
// Per block: the exact sum of q over a grid-stride share of the weights, in
// units of 2^base with base the lowest set bit seen so far (rebased when a
// smaller one appears), plus validity flags.
struct Acc {
    int base;
    u128 acc;
    uint32_t flags;
};

__device__ __forceinline__ void acc_merge(Acc &a, const Acc &b)
{
    a.flags |= b.flags;
    if (b.base == INT_MAX) return;
    if (a.base == INT_MAX) { a.base = b.base; a.acc = b.acc; return; }
    u128 lo_acc = a.acc, hi_acc = b.acc;
    int lo_base = a.base, d = b.base - a.base;
    if (d < 0) { lo_acc = b.acc; hi_acc = a.acc; lo_base = b.base; d = -d; }
    if (hi_acc) {
        if (bitlen128(hi_acc) + d > kQBits) a.flags |= kPartOverflow;
        else lo_acc += hi_acc << d;
    }
    a.base = lo_base;
    a.acc = lo_acc;
    if (hi64(a.acc) >> (kQBits - 64)) a.flags |= kPartOverflow;
}

// Add one weight.  Addends below 2^61 (shift <= 37) go to the 64-bit side
// accumulator a64, which the caller folds into acc at least every 8 items.
template <int F32>
__device__ __forceinline__ void acc_take(Acc &a, uint64_t &a64, uint32_t x)
{
    if (!F32) { a64 += x; return; }
    const uint32_t ex = (x >> 23) & 0xFFu;
    if ((x >> 31) || ex == 0xFFu) { a.flags |= kPartInvalid; return; }
    uint32_t m = x & 0x7FFFFFu;
    if (ex) m |= 0x800000u;
    if (!m) return;
    const int e = (ex ? (int)ex : 1) - 150;
    const int lsb = e + __ffs(m) - 1;
    if (lsb < a.base) { // rare: a lower set bit than any before; rebase
        a.acc += a64;
        a64 = 0;
        if (a.acc) {
            const int d = a.base - lsb;
            if (bitlen128(a.acc) + d > kQBits) { a.flags |= kPartOverflow; a.acc = 0; }
            else a.acc <<= d;
        }
        a.base = lsb;
    }
    const int sh = e - a.base;
    if (sh <= 37) {
        a64 += sh >= 0 ? ((uint64_t)m << sh) : (uint64_t)(m >> (-sh));
    } else {
        if ((32 - __clz(m)) + sh > kQBits) { a.flags |= kPartOverflow; return; }
        a.acc += (u128)m << sh;
    }
}

__device__ __forceinline__ void acc_fold(Acc &a, uint64_t &a64)
{
    a.acc += a64;
    a64 = 0;
    if (hi64(a.acc) >> (kQBits - 64)) { a.flags |= kPartOverflow; a.acc = 0; }
}

__device__ __forceinline__ Acc acc_shfl_down(const Acc &a, int d)
{
    Acc b;
    b.base = __shfl_down_sync(0xFFFFFFFFu, a.base, d);
    b.acc = shfl_down128(a.acc, d);
    b.flags = __shfl_down_sync(0xFFFFFFFFu, a.flags, d);
    return b;
}

__device__ Acc acc_block_reduce(Acc a)
{
    __shared__ int s_base[kWarps];
    __shared__ u128 s_acc[kWarps];
    __shared__ uint32_t s_flags[kWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        Acc b = acc_shfl_down(a, d);
        acc_merge(a, b);
    }
    if (lane == 0) { s_base[wid] = a.base; s_acc[wid] = a.acc; s_flags[wid] = a.flags; }
    __syncthreads();
    if (wid == 0) {
        Acc b;
        if (lane < kWarps) { b.base = s_base[lane]; b.acc = s_acc[lane]; b.flags = s_flags[lane]; }
        else { b.base = INT_MAX; b.acc = 0; b.flags = 0; }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            Acc c = acc_shfl_down(b, d);
            acc_merge(b, c);
        }
        a = b;
    }
    return a; // valid in thread 0
}

// Add the exact value S * 2^(e0 - 150) of some weights, whose lowest set bit
// is at 2^(e0 - 150 + ctz(o)), to an accumulator kept in units of 2^base
// (base: the lowest set bit seen so far).
__device__ __forceinline__ void acc_add_chunk(Acc &a, uint64_t S, uint64_t o, int e0)
{
    const int lsb = e0 - 150 + __ffsll((long long)o) - 1;
    if (lsb < a.base) { // a lower set bit than any before: rebase
        if (a.acc) {
            const int d = a.base - lsb;
            if (bitlen128(a.acc) + d > kQBits) { a.flags |= kPartOverflow; a.acc = 0; }
            else a.acc <<= d;
        }
        a.base = lsb;
    }
    const int sh = e0 - 150 - a.base; // >= -ctz(o), and S is a multiple of 2^ctz(o)
    a.acc += sh >= 0 ? ((u128)S << sh) : (u128)(S >> (-sh));
    if (hi64(a.acc) >> (kQBits - 64)) { a.flags |= kPartOverflow; a.acc = 0; }
}

// Block `bid` of `nblk` blocks sharing the weights of one table; thread 0
// writes the block's partial to *out.  Binary32 weights go in warp chunks
// of 256 (lane l: weights 8l .. 8l+7): when each of a lane's eight is a
// normal number and the exponents of a lane's eight span at most 31
// binades, the lane forms their exact sum in 64 bits as sum m * 2^(e - e0)
// (e0: its smallest exponent; one multiply-add per weight) and their lowest
// set bit from the OR of those terms, and adds it to its accumulator; other
// weights take the exact per-weight path.
template <int F32>
__device__ __forceinline__ void stats_body(const uint32_t *__restrict__ w, uint64_t n, int vec, uint32_t bid,
                                           uint32_t nblk, Partial *__restrict__ out)
{
    Acc a;
    a.base = F32 ? INT_MAX : 0;
    a.acc = 0;
    a.flags = 0;
    uint64_t a64 = 0;
    if (!F32) {
        const uint64_t tid = (uint64_t)bid * kThreads + threadIdx.x;
        const uint64_t nth = (uint64_t)nblk * kThreads;
        const uint64_t nv = vec ? n / 4 : 0;
        const uint4 *w4 = reinterpret_cast<const uint4 *>(w);
        uint64_t i = tid;
        for (; i + 3 * nth < nv; i += 4 * nth) {
            const uint4 v0 = __ldg(w4 + i), v1 = __ldg(w4 + i + nth), v2 = __ldg(w4 + i + 2 * nth), v3 = __ldg(w4 + i + 3 * nth);
            a64 += (uint64_t)v0.x + v0.y + v0.z + v0.w;
            a64 += (uint64_t)v1.x + v1.y + v1.z + v1.w;
            a64 += (uint64_t)v2.x + v2.y + v2.z + v2.w;
            a64 += (uint64_t)v3.x + v3.y + v3.z + v3.w;
        }
        for (; i < nv; i += nth) {
            const uint4 v = __ldg(w4 + i);
            a64 += (uint64_t)v.x + v.y + v.z + v.w;
        }
        for (uint64_t j = nv * 4 + tid; j < n; j += nth) a64 += __ldg(w + j);
        acc_fold(a, a64); // n < 2^32 words below 2^32: the total fits 64 bits
    } else {
        const uint32_t lane = threadIdx.x & 31;
        const uint64_t nchunks = (n + kChunk - 1) / kChunk;
        const uint64_t cw = (uint64_t)nblk * kWarps;
        uint32_t vmax = 0; // any word >= 0x7F800000 is Inf, NaN or has the sign bit set
        uint64_t c = (uint64_t)bid * kWarps + (threadIdx.x >> 5);
        uint32_t x[kItems];
        if (c < nchunks) load_items(w, n, vec, c * kChunk + lane * kItems, x);
        for (; c < nchunks; c += cw) {
            const uint64_t first = c * kChunk + lane * kItems;
            uint32_t xn[kItems];
            const bool more = c + cw < nchunks;
            if (more) load_items(w, n, vec, (c + cw) * kChunk + lane * kItems, xn);
            bool fast = (c + 1) * kChunk <= n; // a full chunk
            uint32_t e0 = 0;
            if (fast) {
                uint32_t emin = 0xFFFFFFFFu, emax = 0;
#pragma unroll
                for (int k = 0; k < kItems; ++k) {
                    vmax = max(vmax, x[k]);
                    const uint32_t ex = x[k] >> 23; // >= 255 for Inf, NaN and negative words
                    emin = min(emin, ex);
                    emax = max(emax, ex);
                }
                e0 = emin;
                fast = e0 >= 1 && emax < 255 && emax - e0 <= 31; // this lane's eight: normal, finite, 31 binades
            }
            if (fast) {
                uint64_t sum = 0, orr = 0;
#pragma unroll
                for (int k = 0; k < kItems; ++k) {
                    const uint32_t m = (x[k] & 0x7FFFFFu) | 0x800000u;
                    const uint64_t v = (uint64_t)m * (1u << ((x[k] >> 23) - e0)); // < 2^55
                    sum += v;
                    orr |= v;
                }
                acc_add_chunk(a, sum, orr, (int)e0); // this lane's eight terms (orr > 0: every m has its top bit)
            } else {
#pragma unroll
                for (int k = 0; k < kItems; ++k) {
                    if (first + k < n) {
                        acc_take<1>(a, a64, x[k]);
                        acc_fold(a, a64);
                    }
                }
            }
            if (more) {
#pragma unroll
                for (int k = 0; k < kItems; ++k) x[k] = xn[k];
            }
        }
        if (vmax >= 0x7F800000u) a.flags |= kPartInvalid;
    }
    a = acc_block_reduce(a);
    if (threadIdx.x == 0) {
        Partial p;
        p.lo = lo64(a.acc); p.hi = hi64(a.acc); p.base = a.base; p.flags = a.flags; p.pad = 0;
        *out = p;
    }
}

template <int F32>
__global__ void __launch_bounds__(kThreads) k_stats(const uint32_t *__restrict__ w, uint64_t n, int vec,
                                                    Partial *__restrict__ part)
{
    stats_body<F32>(w, n, vec, blockIdx.x, gridDim.x, part + blockIdx.x);
}

// Is n * val(v) <= Q * 2^beta for the binary32 pattern v (v >= +0, finite)?
__device__ bool f32_light(uint32_t v, uint64_t n, u128 Q, int beta)
{
    uint32_t ex = (v >> 23) & 0xFFu, m = v & 0x7FFFFFu;
    if (ex) m |= 0x800000u;
    if (!m) return true;
    int d = (ex ? (int)ex : 1) - 150 - beta;
    u128 nm = (u128)m * n;
    if (d >= 0) {
        if (bitlen128(nm) + d > 127) return false;
        return (nm << d) <= Q;
    }
    int dd = -d;
    if (bitlen128(Q) + dd > 127) return true;
    return nm <= (Q << dd);
}

__device__ __forceinline__ uint32_t write_header(const Acc &a, uint64_t n, uint32_t f32, DevHeader *hdr);

__device__ __forceinline__ void stats_combine_body(const Partial *__restrict__ part, uint32_t nparts, uint64_t n,
                                                   uint32_t f32, DevHeader *hdr)
{
    Acc a;
    a.base = INT_MAX; a.acc = 0; a.flags = 0;
    for (uint32_t i = threadIdx.x; i < nparts; i += kThreads) {
        Partial p = part[i];
        Acc b;
        b.base = p.base; b.acc = mk128(p.lo, p.hi); b.flags = p.flags;
        if (!f32) b.base = 0;
        acc_merge(a, b);
    }
    a = acc_block_reduce(a);
    if (threadIdx.x == 0) write_header(a, n, f32, hdr);
}

// The table header from the exact total (thread 0): status, beta, Q, shift,
// qp and the light threshold on the raw words.
__device__ __forceinline__ uint32_t write_header(const Acc &a, uint64_t n, uint32_t f32, DevHeader *hdr)
{
    uint32_t status = kOk;
    if (a.flags & kPartInvalid) status = kEInval;
    else if (a.flags & kPartOverflow) status = kEOverflow;
    else if (a.acc == 0) status = kEInval;
    const u128 Q = a.acc;
    int shift = bitlen128(Q) - 64;
    if (shift < 0) shift = 0;
    uint32_t light_max = 0;
    int beta = f32 ? (a.base == INT_MAX ? 0 : a.base) : 0;
    if (status == kOk) {
        if (!f32) {
            light_max = (uint32_t)(lo64(Q) / n); // Q < 2^64, Q/n < 2^32
        } else {
            uint32_t lo = 0, hi = 0x7F7FFFFFu; // largest v with f32_light(v)
            while (lo < hi) {
                uint32_t mid = lo + (hi - lo + 1) / 2;
                if (f32_light(mid, n, Q, beta)) lo = mid; else hi = mid - 1;
            }
            light_max = lo;
        }
    }
    hdr->tile_counter = 0;
    hdr->beta = beta;
    hdr->shift = (uint32_t)shift;
    hdr->q_lo = lo64(Q);
    hdr->q_hi = hi64(Q);
    hdr->qp = lo64(Q >> shift);
    hdr->light_max = light_max;
    hdr->f32 = f32;
    hdr->n = n;
    hdr->n_light = 0;
    hdr->pad[0] = 0;
    hdr->pad[1] = 0;
    __threadfence();
    hdr->status = status;
    return status;
}

__global__ void __launch_bounds__(kThreads) k_stats_combine(const Partial *__restrict__ part, uint32_t nparts,
                                                            uint64_t n, uint32_t f32, DevHeader *hdr)
{
    stats_combine_body(part, nparts, n, f32, hdr);
}

// ---------------------------------------------------------- k_classify
// q of a weight known to be below 2^61 (shift <= 37)
__device__ __forceinline__ uint64_t q64_of(uint32_t x, uint32_t f32, int beta)
{
    if (!f32) return x;
    const uint32_t ex = (x >> 23) & 0xFFu;
    uint32_t m = x & 0x7FFFFFu;
    if (ex) m |= 0x800000u;
    const int sh = (ex ? (int)ex : 1) - 150 - beta;
    return sh >= 0 ? ((uint64_t)m << sh) : (uint64_t)(m >> (-sh));
}

__device__ __forceinline__ void tilesum_st(TileSum *p, const TileSum &v)
{
    uint4 *d = reinterpret_cast<uint4 *>(p);
    d[0] = make_uint4((uint32_t)v.l_lo, (uint32_t)(v.l_lo >> 32), (uint32_t)v.l_hi, (uint32_t)(v.l_hi >> 32));
    d[1] = make_uint4((uint32_t)v.h_lo, (uint32_t)(v.h_lo >> 32), (uint32_t)v.h_hi, (uint32_t)(v.h_hi >> 32));
    d[2] = make_uint4(v.cl, v.nheavy, v.first_heavy, 0u);
}

__device__ __forceinline__ TileSum tilesum_ldcg(const TileSum *p)
{
    const uint4 *s = reinterpret_cast<const uint4 *>(p);
    uint4 a = __ldcg(s), c = __ldcg(s + 1), d = __ldcg(s + 2);
    TileSum r;
    r.l_lo = a.x | ((uint64_t)a.y << 32); r.l_hi = a.z | ((uint64_t)a.w << 32);
    r.h_lo = c.x | ((uint64_t)c.y << 32); r.h_hi = c.z | ((uint64_t)c.w << 32);
    r.cl = d.x; r.nheavy = d.y; r.first_heavy = d.z; r.pad = d.w;
    return r;
}

// Sum of a u128 over the warp, returned to every lane: the warp-wide
// reduction instruction adds 16-bit limbs exactly (each limb's sum over 32
// lanes is below 2^21); the high half is skipped when every lane's is zero.
__device__ __forceinline__ u128 warp_sum128(u128 v)
{
    const uint64_t lo = lo64(v), hi = hi64(v);
    u128 r = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c)
        r += (u128)__reduce_add_sync(0xFFFFFFFFu, (uint32_t)(lo >> (16 * c)) & 0xFFFFu) << (16 * c);
    if (__any_sync(0xFFFFFFFFu, hi != 0)) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
            r += (u128)__reduce_add_sync(0xFFFFFFFFu, (uint32_t)(hi >> (16 * c)) & 0xFFFFu) << (64 + 16 * c);
    }
    return r;
}

// Exclusive scan of a u32 over the warp.
__device__ __forceinline__ uint32_t warp_excl_scan_u32(uint32_t v)
{
    const int lane = threadIdx.x & 31;
    uint32_t s = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, s, d);
        if (lane >= d) s += o;
    }
    return s - v;
}

// Tiles t_first, t_first + t_stride, ... of one table, ONE WARP per tile
// (no block barrier per tile).  A tile is eight chunks of 256 weights; lane
// l holds weights 8l .. 8l+7 of a chunk.  Per tile: light count, light and
// heavy sums of q, heavy count, offset of the first heavy, and the offsets of
// its heavies when it has at most 32 of them.
template <int F32>
__device__ __forceinline__ void classify_body(const uint32_t *__restrict__ w, uint64_t n, int vec,
                                              const DevHeader *__restrict__ hdr, TileSum *__restrict__ agg,
                                              uint16_t *__restrict__ slist, uint32_t ntiles, uint32_t t_first,
                                              uint32_t t_stride)
{
    __shared__ uint16_t s_list[kWarps][kSparse];
    if (block_stopped(hdr)) return;
    const uint32_t light_max = hdr->light_max;
    const int beta = hdr->beta;
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint16_t *list = s_list[wid];
    uint32_t x[kItems];
    if (t_first < ntiles) load_items(w, n, vec, (uint64_t)t_first * kTile + lane * kItems, x);
    for (uint32_t t = t_first; t < ntiles; t += t_stride) {
        const uint64_t tile0 = (uint64_t)t * kTile;
        u128 Lp = 0, Hp = 0;             // this lane's light and heavy sums over the tile (units of 2^beta)
        uint32_t cl = 0, ch = 0;          // this lane's light and heavy counts
        uint32_t chp = 0, fh = kNone;     // heavies before the chunk (kept while at most kSparse), first heavy
#pragma unroll 1
        for (uint32_t c = 0; c < (uint32_t)kChunks; ++c) {
            const uint64_t first = tile0 + c * kChunk + lane * kItems;
            const bool full = tile0 + (c + 1) * kChunk <= n; // the same in every lane
            uint32_t lm = 0, vm = 0xFFu;
            uint32_t emin = 0xFFFFFFFFu, emax = 0;
            if (full) {
#pragma unroll
                for (int k = 0; k < kItems; ++k) {
                    if (x[k] <= light_max) lm |= 1u << k;
                    if (F32) {
                        const uint32_t ex = x[k] >> 23; // a valid word has its sign bit clear
                        emin = min(emin, ex);
                        emax = max(emax, ex);
                    }
                }
            } else {
                vm = 0;
#pragma unroll
                for (int k = 0; k < kItems; ++k) {
                    if (first + k < n) {
                        vm |= 1u << k;
                        if (x[k] <= light_max) lm |= 1u << k;
                    }
                }
            }
            const uint32_t hm = vm & ~lm;
            bool chunk_fast = false;
            uint32_t e0 = 0;
            if (F32 && full) {
                e0 = __reduce_min_sync(0xFFFFFFFFu, emin);
                chunk_fast = e0 >= 1 && __reduce_max_sync(0xFFFFFFFFu, emax) - e0 <= 31;
            }
            if (chunk_fast) {
                // every weight normal, exponents within 31 binades: m * 2^(e - e0)
                // in 64 bits (one multiply-add each, below 2^58 per lane), then
                // scaled to units of 2^beta (exact: every term q * 2^-sh is a
                // multiple of 2^-sh when sh < 0)
                uint64_t l64 = 0, h64 = 0;
#pragma unroll
                for (int k = 0; k < kItems; ++k) {
                    const uint64_t v = (uint64_t)((x[k] & 0x7FFFFFu) | 0x800000u) * (1u << ((x[k] >> 23) - e0));
                    if ((lm >> k) & 1u) l64 += v; else h64 += v;
                }
                const int sh = (int)e0 - 150 - beta;
                Lp += sh >= 0 ? (u128)l64 << sh : (u128)(l64 >> (-sh));
                Hp += sh >= 0 ? (u128)h64 << sh : (u128)(h64 >> (-sh));
            } else {
                bool narrow = true; // every q below 2^61: eight of them fit 64 bits
                if (F32) {
#pragma unroll
                    for (int k = 0; k < kItems; ++k) {
                        const uint32_t ex = (x[k] >> 23) & 0xFFu;
                        if (((vm >> k) & 1u) && (ex ? (int)ex : 1) - 150 - beta > 37) narrow = false;
                    }
                }
                if (narrow) {
                    uint64_t l64 = 0, h64 = 0;
#pragma unroll
                    for (int k = 0; k < kItems; ++k) {
                        const uint64_t q = q64_of(x[k], F32, beta);
                        if ((lm >> k) & 1u) l64 += q;
                        if ((hm >> k) & 1u) h64 += q;
                    }
                    Lp += l64;
                    Hp += h64;
                } else {
#pragma unroll
                    for (int k = 0; k < kItems; ++k) {
                        if ((vm >> k) & 1u) {
                            const u128 q = q_of(x[k], F32, beta);
                            if ((lm >> k) & 1u) Lp += q; else Hp += q;
                        }
                    }
                }
            }
            cl += (uint32_t)__popc(lm);
            ch += (uint32_t)__popc(hm);
            // prefetch the next chunk (or the next tile's first)
            const uint64_t nf = c + 1 < (uint32_t)kChunks ? first + kChunk
                                                          : (uint64_t)(t + t_stride) * kTile + lane * kItems;
            const bool more = c + 1 < (uint32_t)kChunks || t + t_stride < ntiles;
            if (chp <= (uint32_t)kSparse || fh == kNone) {
                const uint32_t hb = __ballot_sync(0xFFFFFFFFu, hm != 0);
                if (fh == kNone && hb) {
                    const int src = __ffs(hb) - 1;
                    const uint32_t hs = __shfl_sync(0xFFFFFFFFu, hm, src);
                    fh = c * kChunk + (uint32_t)src * kItems + (uint32_t)(__ffs(hs) - 1);
                }
                if (chp <= (uint32_t)kSparse && hb) { // offsets of the first heavies, in order
                    uint32_t pos = chp + warp_excl_scan_u32((uint32_t)__popc(hm));
#pragma unroll
                    for (int k = 0; k < kItems; ++k) {
                        if ((hm >> k) & 1u) {
                            if (pos < (uint32_t)kSparse) list[pos] = (uint16_t)(c * kChunk + lane * kItems + k);
                            ++pos;
                        }
                    }
                    chp += __reduce_add_sync(0xFFFFFFFFu, (uint32_t)__popc(hm));
                }
            }
            if (more) load_items(w, n, vec, nf, x);
        }
        const u128 L = warp_sum128(Lp), H = warp_sum128(Hp);
        const uint32_t tl = __reduce_add_sync(0xFFFFFFFFu, cl), th = __reduce_add_sync(0xFFFFFFFFu, ch);
        __syncwarp();
        if (lane == 0) {
            TileSum a;
            a.l_lo = lo64(L); a.l_hi = hi64(L); a.h_lo = lo64(H); a.h_hi = hi64(H);
            a.cl = tl; a.nheavy = th; a.first_heavy = fh; a.pad = 0;
            tilesum_st(agg + t, a);
        }
        if (th <= (uint32_t)kSparse && lane < th) slist[(uint64_t)t * kSparse + lane] = list[lane];
        __syncwarp();
    }
}

template <int F32>
__global__ void __launch_bounds__(kThreads) k_classify(const uint32_t *__restrict__ w, uint64_t n, int vec,
                                                       const DevHeader *__restrict__ hdr, TileSum *__restrict__ agg,
                                                       uint16_t *__restrict__ slist, uint32_t ntiles)
{
    classify_body<F32>(w, n, vec, hdr, agg, slist, ntiles, blockIdx.x * kWarps + (threadIdx.x >> 5),
                       gridDim.x * kWarps);
}

// ---------------------------------------------------------- k_tilescan
// Inclusive prefix of the tile aggregates.  Each block takes 256 consecutive
// tiles (block ids in launch order from an atomic counter, so every block it
// waits for is already running), scans them, publishes the chunk aggregate,
// then warp 0 looks back over the predecessors' published values until it
// meets an inclusive prefix, and publishes its own.  Every wait is bounded by
// `wait_limit` polls: a wait that runs out stores WRS_ETIMEOUT and the block
// carries on, so no block ever waits forever.
__device__ __forceinline__ void tilesum_add(TileSum &a, const TileSum &b)
{
    u128 l = mk128(a.l_lo, a.l_hi) + mk128(b.l_lo, b.l_hi);
    u128 h = mk128(a.h_lo, a.h_hi) + mk128(b.h_lo, b.h_hi);
    a.l_lo = lo64(l); a.l_hi = hi64(l); a.h_lo = lo64(h); a.h_hi = hi64(h);
    a.cl += b.cl;
}

__device__ __forceinline__ TileSum tilesum_shfl_xor(const TileSum &a, int m)
{
    TileSum b;
    b.l_lo = __shfl_xor_sync(0xFFFFFFFFu, a.l_lo, m); b.l_hi = __shfl_xor_sync(0xFFFFFFFFu, a.l_hi, m);
    b.h_lo = __shfl_xor_sync(0xFFFFFFFFu, a.h_lo, m); b.h_hi = __shfl_xor_sync(0xFFFFFFFFu, a.h_hi, m);
    b.cl = __shfl_xor_sync(0xFFFFFFFFu, a.cl, m);
    b.nheavy = 0; b.first_heavy = kNone; b.pad = 0;
    return b;
}

__device__ __forceinline__ void tilescan_body(DevHeader *hdr, const TileSum *__restrict__ agg, TileSum *chunk_agg,
                                              TileSum *chunk_incl, TileSum *__restrict__ incl, uint32_t *flags,
                                              uint32_t ntiles, uint32_t epoch, uint32_t wait_limit,
                                              uint32_t skip_chunk)
{
    __shared__ uint32_t s_chunk, s_status;
    __shared__ U2 s_scan[kWarps];
    __shared__ uint32_t s_cnt[kWarps];
    __shared__ TileSum s_ex;
    if (threadIdx.x == 0) {
        s_status = *(volatile uint32_t *)&hdr->status;
        s_chunk = s_status ? 0u : atomicAdd(&hdr->tile_counter, 1u);
    }
    __syncthreads();
    if (s_status) return;
    const uint32_t c = s_chunk;
    const uint32_t t = c * kScanChunk + threadIdx.x;
    TileSum a;
    if (t < ntiles) a = tilesum_ldcg(agg + t);
    else { a.l_lo = a.l_hi = a.h_lo = a.h_hi = 0; a.cl = 0; a.nheavy = 0; a.first_heavy = kNone; a.pad = 0; }
    U2 tot;
    const U2 ex = block_exclusive_scan2(U2{mk128(a.l_lo, a.l_hi), mk128(a.h_lo, a.h_hi)}, tot, s_scan);
    uint32_t ctot;
    const uint32_t cex = block_exclusive_scan_u32(a.cl, ctot, s_cnt);
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        TileSum ca;
        ca.l_lo = lo64(tot.a); ca.l_hi = hi64(tot.a); ca.h_lo = lo64(tot.b); ca.h_hi = hi64(tot.b);
        ca.cl = ctot; ca.nheavy = 0; ca.first_heavy = kNone; ca.pad = 0;
        const bool publish = (c != skip_chunk);
        TileSum exc;
        exc.l_lo = exc.l_hi = exc.h_lo = exc.h_hi = 0; exc.cl = 0; exc.nheavy = 0; exc.first_heavy = kNone; exc.pad = 0;
        if (c == 0) {
            if (lane == 0) {
                tilesum_st(chunk_incl, ca);
                if (publish) st_release(flags, (epoch << 2) | kFlagIncl);
            }
        } else {
            if (lane == 0) {
                tilesum_st(chunk_agg + c, ca);
                if (publish) st_release(flags + c, (epoch << 2) | kFlagAgg);
            }
            int64_t p = (int64_t)c - 1 - lane;
            bool timed_out = false;
            for (;;) {
                uint32_t st = kFlagIncl; // virtual predecessor before chunk 0
                if (p >= 0) {
                    uint32_t polls = 0;
                    for (;;) {
                        const uint32_t fv = ld_acquire(flags + p);
                        st = ((fv >> 2) == epoch) ? (fv & 3u) : 0u;
                        if (st != 0u || ++polls >= wait_limit) break;
                        __nanosleep(32);
                    }
                }
                if (__any_sync(0xFFFFFFFFu, st == 0u)) { timed_out = true; break; }
                const uint32_t incl_mask = __ballot_sync(0xFFFFFFFFu, st == kFlagIncl);
                const int stop = incl_mask ? __ffs(incl_mask) - 1 : 32;
                TileSum v;
                if (lane <= stop && p >= 0) v = tilesum_ldcg(st == kFlagIncl ? chunk_incl + p : chunk_agg + p);
                else { v.l_lo = v.l_hi = v.h_lo = v.h_hi = 0; v.cl = 0; }
#pragma unroll
                for (int m = 16; m > 0; m >>= 1) {
                    TileSum o = tilesum_shfl_xor(v, m);
                    tilesum_add(v, o);
                }
                tilesum_add(exc, v);
                if (incl_mask) break;
                p -= 32;
            }
            if (lane == 0) {
                if (timed_out) set_status(hdr, kETimeout);
                TileSum r = ca;
                tilesum_add(r, exc);
                tilesum_st(chunk_incl + c, r);
                if (publish) st_release(flags + c, (epoch << 2) | kFlagIncl);
            }
        }
        if (lane == 0) s_ex = exc;
    }
    __syncthreads();
    if (t < ntiles) {
        TileSum r;
        const u128 l = mk128(s_ex.l_lo, s_ex.l_hi) + ex.a + mk128(a.l_lo, a.l_hi);
        const u128 h = mk128(s_ex.h_lo, s_ex.h_hi) + ex.b + mk128(a.h_lo, a.h_hi);
        r.l_lo = lo64(l); r.l_hi = hi64(l); r.h_lo = lo64(h); r.h_hi = hi64(h);
        r.cl = s_ex.cl + cex + a.cl;
        r.nheavy = a.nheavy; r.first_heavy = a.first_heavy; r.pad = 0;
        tilesum_st(incl + t, r);
    }
}

__global__ void __launch_bounds__(kThreads) k_tilescan(DevHeader *hdr, const TileSum *__restrict__ agg,
                                                       TileSum *chunk_agg, TileSum *chunk_incl,
                                                       TileSum *__restrict__ incl, uint32_t *flags,
                                                       uint32_t ntiles, uint32_t epoch, uint32_t wait_limit,
                                                       uint32_t skip_chunk)
{
    tilescan_body(hdr, agg, chunk_agg, chunk_incl, incl, flags, ntiles, epoch, wait_limit, skip_chunk);
}

// ------------------------------------------------------------ k_split
// For every tile c, from the tile prefix sums: with D_c = D at the first
// light of tile c and E_c = E after the heavies before tile c,
//   hb = max{ b : E(b) <= D_c }  -- the tile holding the first heavy item
//        with E > D_c, the heavy current when tile c's first light is
//        packed (the split of Alg. 3 on the heavy prefix sums);
//   lb = max{ b : D(b) <= E_c }  -- a tile at or before the one holding the
//        first light that follows tile c's first heavy (split on the light
//        prefix sums);
//   next_heavy = position of the first heavy item after tile c.
struct Prefix {
    uint64_t cl, ch;
    u128 L, H;
};

__device__ __forceinline__ Prefix prefix_at(const TileSum *incl, uint32_t b, uint64_t n)
{
    TileSum t = load_prefix(incl, b);
    Prefix p;
    p.cl = t.cl;
    uint64_t end = (uint64_t)b * kTile;
    if (end > n) end = n;
    p.ch = end - p.cl;
    p.L = mk128(t.l_lo, t.l_hi);
    p.H = mk128(t.h_lo, t.h_hi);
    return p;
}

__device__ __forceinline__ u128 key_E(const Prefix &p, uint64_t n, u128 Q) { return times_n(p.H, n) - (u128)p.ch * Q; }
__device__ __forceinline__ u128 key_D(const Prefix &p, uint64_t n, u128 Q) { return (u128)p.cl * Q - times_n(p.L, n); }

// Tile c of one table (one thread per tile).
__device__ __forceinline__ void split_body(const TileSum *__restrict__ incl, uint32_t ntiles, uint64_t n,
                                           DevHeader *hdr, Split *__restrict__ split, uint32_t c)
{
    if (*(volatile uint32_t *)&hdr->status) return;
    const u128 Q = mk128(hdr->q_lo, hdr->q_hi);
    const uint64_t n_light = load_prefix(incl, ntiles).cl;
    if (c == 0) hdr->n_light = n_light;
    if (c >= ntiles) return;
    const Prefix pc = prefix_at(incl, c, n);
    const u128 Dc = key_D(pc, n, Q), Ec = key_E(pc, n, Q);
    uint32_t lo = 0, hi = ntiles;
    while (lo < hi) {
        uint32_t mid = lo + (hi - lo + 1) / 2;
        if (key_E(prefix_at(incl, mid, n), n, Q) <= Dc) lo = mid; else hi = mid - 1;
    }
    const uint32_t hb = lo;
    lo = 0; hi = ntiles;
    while (lo < hi) {
        uint32_t mid = lo + (hi - lo + 1) / 2;
        if (key_D(prefix_at(incl, mid, n), n, Q) <= Ec) lo = mid; else hi = mid - 1;
    }
    const uint32_t lb = lo;
    const Prefix pn = prefix_at(incl, c + 1, n);
    const uint64_t total_h = n - n_light;
    uint32_t nxt = kNone;
    if (pn.ch < total_h) { // heavy rank pn.ch is the first heavy of tile max{b : ch(b) <= pn.ch}
        lo = c + 1; hi = ntiles - 1;
        while (lo < hi) {
            uint32_t mid = lo + (hi - lo + 1) / 2;
            if (prefix_at(incl, mid, n).ch <= pn.ch) lo = mid; else hi = mid - 1;
        }
        const TileSum tb = tilesum_ldcg(incl + lo);
        nxt = lo * (uint32_t)kTile + tb.first_heavy;
    }
    Split s;
    s.hb = hb; s.lb = lb; s.next_heavy = nxt; s.pad = 0;
    split[c] = s;
}

__global__ void __launch_bounds__(kThreads) k_split(const TileSum *__restrict__ incl, uint32_t ntiles, uint64_t n,
                                                    DevHeader *hdr, Split *__restrict__ split)
{
    split_body(incl, ntiles, n, hdr, split, blockIdx.x * kThreads + threadIdx.x);
}



// ------------------------------------------------------------ k_sweep
// Tile c packs, as Alg. 3's pack does for one subproblem, the buckets of its
// own lights and of every heavy item whose key E lies in (D_c, D_c'] (D_c:
// key of the tile's first light, D_c': key after its last light): exactly
// the items Alg. 2 packs while it consumes this tile's lights.  The heavy
// items come tile by tile in index order from the tile k_split named
// (Alg. 3's split on the heavy prefix sums); the first such tile is loaded
// together with the own tile.  For each stream tile the block merges, in key
// order, the own lights whose current heavy lies in that tile with the
// tile's heavies in (D_c, D_c'] (heavy first when E <= D): a light step
// takes the current heavy as its alias, a heavy step gets bucket
// Q - (D_next - E) with D_next the key of the next light, and the next heavy
// as alias.  The merged sequence is split evenly over the threads by a
// merge-path co-rank search, then each thread walks its slice.
__device__ __forceinline__ u128 nq_of(uint32_t x, uint32_t f32, int beta, uint32_t n32)
{
    if (!f32) return (u128)((uint64_t)x * n32);
    const uint32_t ex = (x >> 23) & 0xFFu;
    uint32_t m = x & 0x7FFFFFu;
    if (ex) m |= 0x800000u;
    const uint64_t nm = (uint64_t)m * n32; // < 2^56
    const int sh = (ex ? (int)ex : 1) - 150 - beta;
    return sh >= 0 ? ((u128)nm << sh) : (u128)(nm >> (-sh)); // exact: m carries the low zero bits
}

__device__ __forceinline__ u128 block_exclusive_scan1(u128 v, u128 &total, u128 *sm)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    u128 inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const u128 o = shfl_up128(inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) sm[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        u128 t = lane < kWarps ? sm[lane] : (u128)0;
#pragma unroll
        for (int d = 1; d < kWarps; d <<= 1) {
            const u128 o = shfl_up128(t, d);
            if (lane >= d) t += o;
        }
        if (lane < kWarps) sm[lane] = t;
    }
    __syncthreads();
    const u128 base = wid ? sm[wid - 1] : (u128)0;
    total = sm[kWarps - 1];
    __syncthreads();
    return base + inc - v;
}

// 16-B elements, 8 per 128-B bank row: XOR the column with the row's low bits
// so that threads reading consecutive rows at one column hit distinct banks.
__device__ __forceinline__ uint32_t swz(uint32_t j) { return j ^ ((j >> 3) & 7u); }

struct SweepSmem {
    u128 okey[kTile];     // keys D of the own lights, in order (swizzled)
    u128 hkey[kTile];     // keys E of the current stream tile's heavies (swizzled)
    uint16_t ooff[kTile];   // offsets of the own lights in the tile
    uint16_t hoff[kTile];   // offsets of the stream tile's heavies
    u128 scan[kWarps];
    uint32_t cnt[kWarps];
    uint32_t hcount;
    uint32_t rng[4];      // light and heavy index ranges of the current round
};

// First index in [lo, hi) of the sorted keys whose key is > v (upper) or
// >= v (!upper), found by a whole warp: each round probes 32 evenly spaced
// keys and keeps the gap between the last probe before the answer and the
// first one after it, so a range of 2048 takes two rounds and a final probe
// of at most 32 keys.  Every lane returns the answer.
__device__ __forceinline__ uint32_t warp_search(const u128 *key, uint32_t lo, uint32_t hi, u128 v, bool upper)
{
    const uint32_t lane = threadIdx.x & 31;
    while (hi - lo > 32) {
        const uint32_t step = (hi - lo + 31) / 32;
        const uint32_t p = lo + step * lane;
        const bool before = p < hi && (upper ? key[swz(p)] <= v : key[swz(p)] < v);
        const uint32_t cnt = (uint32_t)__popc(__ballot_sync(0xFFFFFFFFu, before)); // probes before the answer
        if (cnt == 0) return lo;
        const uint32_t nhi = lo + step * cnt; // first probe not before the answer (or past hi)
        lo += step * (cnt - 1) + 1;
        hi = nhi < hi ? nhi : hi;
    }
    const uint32_t p = lo + lane;
    const bool before = p < hi && (upper ? key[swz(p)] <= v : key[swz(p)] < v);
    return lo + (uint32_t)__popc(__ballot_sync(0xFFFFFFFFu, before));
}

// Heavies of a stream tile up to which load_heavies compacts their words
// first: the keys of heavies 0 .. c-1 end below byte 16 (c + 8) of the key
// array, and the words sit in its top 4 c bytes (16 (c + 8) <= 32768 - 4 c).
constexpr uint32_t kCompactMax = 1600;

// Keys of stream tile t's heavies into S.hkey/S.hoff (all threads call).
template <int F32>
__device__ __forceinline__ void load_heavies(SweepSmem &S, uint32_t t, const uint32_t (&y)[kItems], uint32_t nheavy,
                                             uint64_t n, uint32_t n32, const TileSum *incl,
                                             const uint16_t *__restrict__ slist, const uint32_t *__restrict__ w,
                                             u128 Q, uint32_t light_max, int beta)
{
    const Prefix pf = prefix_at(incl, t, n);
    const u128 base = key_E(pf, n, Q);
    const uint64_t tile0 = (uint64_t)t * kTile;
    if (nheavy <= (uint32_t)kSparse) {
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            u128 d = 0;
            uint32_t off = 0;
            if ((uint32_t)lane < nheavy) {
                off = slist[(uint64_t)t * kSparse + lane];
                d = nq_of(__ldg(w + tile0 + off), F32, beta, n32) - Q;
            }
            u128 key = d;
#pragma unroll
            for (int s = 1; s < 32; s <<= 1) {
                const u128 o = shfl_up128(key, s);
                if (lane >= s) key += o;
            }
            if ((uint32_t)lane < nheavy) { S.hkey[swz(lane)] = base + key; S.hoff[lane] = (uint16_t)off; }
            if (lane == 0) S.hcount = nheavy;
        }
        __syncthreads();
        return;
    }
    const uint64_t first = tile0 + (uint64_t)threadIdx.x * kItems;
    uint32_t hm = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k)
        if (first + k < n && y[k] > light_max) hm |= 1u << k;
    uint32_t ctot;
    const uint32_t slot0 = block_exclusive_scan_u32((uint32_t)__popc(hm), ctot, S.cnt);
    if (ctot <= kCompactMax) {
        // Compacted first: the heavies' words go, in index order, to the top
        // of the key array (below it the keys of the first ctot heavies
        // never reach them), then thread t keys heavies [t q, t q + q),
        // q = ceil(ctot / 256): every lane runs the same number of steps
        // whatever the share of heavies in its eight words.
        uint32_t *raw = reinterpret_cast<uint32_t *>(S.hkey) + (kTile * 4 - ctot);
        {
            uint32_t slot = slot0;
#pragma unroll
            for (int k = 0; k < kItems; ++k) {
                if ((hm >> k) & 1u) {
                    raw[slot] = y[k];
                    S.hoff[slot] = (uint16_t)(threadIdx.x * kItems + k);
                    ++slot;
                }
            }
        }
        __syncthreads();
        const uint32_t q = (ctot + kThreads - 1) / kThreads;
        const uint32_t j0 = min(threadIdx.x * q, ctot), j1 = min(j0 + q, ctot);
        u128 sum = 0;
        for (uint32_t j = j0; j < j1; ++j) {
            const u128 e = nq_of(raw[j], F32, beta, n32) - Q;
            S.hkey[swz(j)] = e;
            sum += e;
        }
        u128 tot;
        u128 key = base + block_exclusive_scan1(sum, tot, S.scan);
        for (uint32_t j = j0; j < j1; ++j) {
            key += S.hkey[swz(j)];
            S.hkey[swz(j)] = key;
        }
        if (threadIdx.x == 0) S.hcount = ctot;
        __syncthreads();
        return;
    }
    // excesses n*q - Q into the key slots, then an in-place prefix
    u128 sum = 0;
    {
        uint32_t slot = slot0;
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            if ((hm >> k) & 1u) {
                const u128 e = nq_of(y[k], F32, beta, n32) - Q;
                S.hkey[swz(slot)] = e;
                S.hoff[slot] = (uint16_t)(threadIdx.x * kItems + k);
                sum += e;
                ++slot;
            }
        }
    }
    u128 tot;
    u128 key = base + block_exclusive_scan1(sum, tot, S.scan);
    {
        const uint32_t cnt = (uint32_t)__popc(hm);
        for (uint32_t j = 0; j < cnt; ++j) {
            key += S.hkey[swz(slot0 + j)];
            S.hkey[swz(slot0 + j)] = key;
        }
    }
    if (threadIdx.x == 0) S.hcount = ctot;
    __syncthreads();
}

constexpr int kSweepTiles = 8; // own tiles per block of k_sweep (they share stream tiles)

// Own tiles [c_first, c_last) of one table.
template <int F32>
__device__ __forceinline__ void sweep_body(const uint32_t *__restrict__ w, uint64_t n, int vec, DevHeader *hdr,
                                           const TileSum *__restrict__ incl, const Split *__restrict__ split,
                                           const uint16_t *__restrict__ slist, uint32_t ntiles,
                                           uint4 *__restrict__ table, uint32_t c_first, uint32_t c_last,
                                           bool force_wide = false)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SweepSmem &S = *reinterpret_cast<SweepSmem *>(smem_raw);
    if (block_stopped(hdr)) return;
    const uint32_t n32 = (uint32_t)n;
    const u128 Q = mk128(hdr->q_lo, hdr->q_hi);
    const uint32_t light_max = hdr->light_max;
    const int beta = hdr->beta;
    const uint32_t shift = hdr->shift;
    const bool narrow = shift == 0 && !force_wide; // Q < 2^64, the same for the whole grid
    bool bad = false;

    uint32_t x[kItems], y[kItems];
    load_items(w, n, vec, (uint64_t)c_first * kTile + (uint64_t)threadIdx.x * kItems, x);
    uint32_t s = split[c_first].hb;   // current stream tile
    uint32_t s_loaded = kNone;        // stream tile whose heavies are in S.hkey
    uint32_t y_tile = kNone;          // stream tile whose words are in y
    if (s < ntiles) { load_items(w, n, vec, (uint64_t)s * kTile + (uint64_t)threadIdx.x * kItems, y); y_tile = s; }

    for (uint32_t c = c_first; c < c_last; ++c) {
        const uint64_t tile0 = (uint64_t)c * kTile;
        const uint64_t first = tile0 + (uint64_t)threadIdx.x * kItems;
        // own lights: deficits Q - n*q, thresholds n*q >> shift, full lights
        uint32_t lmask = 0;
#pragma unroll
        for (int k = 0; k < kItems; ++k)
            if (first + k < n && x[k] <= light_max) lmask |= 1u << k;
        uint32_t nl;
        const uint32_t lslot0 = block_exclusive_scan_u32((uint32_t)__popc(lmask), nl, S.cnt); // syncs: okey free
        u128 def = 0;
        {
            uint32_t slot = lslot0;
#pragma unroll
            for (int k = 0; k < kItems; ++k) {
                if ((lmask >> k) & 1u) {
                    const u128 d = Q - nq_of(x[k], F32, beta, n32);
                    S.okey[swz(slot)] = d;
                    S.ooff[slot] = (uint16_t)(threadIdx.x * kItems + k);
                    def += d;
                    ++slot;
                }
            }
        }
        const Prefix pc = prefix_at(incl, c, n);
        const u128 D_start = key_D(pc, n, Q);
        u128 dtot;
        {
            u128 kl = D_start + block_exclusive_scan1(def, dtot, S.scan);
            const uint32_t cnt = (uint32_t)__popc(lmask);
            for (uint32_t j = 0; j < cnt; ++j) { // deficits -> exclusive keys, in place
                const u128 d = S.okey[swz(lslot0 + j)];
                S.okey[swz(lslot0 + j)] = kl;
                kl += d;
            }
        }
        const u128 D_end = D_start + dtot;
        // prefetch the next own tile
        if (c + 1 < c_last) load_items(w, n, vec, (uint64_t)(c + 1) * kTile + (uint64_t)threadIdx.x * kItems, x);
        if (nl == 0) continue; // no lights: nothing is packed for this tile
        uint32_t al = 0; // own lights resolved so far
        for (;;) {
            if (s >= ntiles) {
                // no heavy item left: the remaining own lights must be exactly full
                __syncthreads();
                for (uint32_t i = al + threadIdx.x; i < nl; i += kThreads) {
                    const u128 dn = (i + 1 < nl) ? S.okey[swz(i + 1)] : D_end;
                    const u128 nq = Q - (dn - S.okey[swz(i)]);
                    if (nq != Q) bad = true;
                    const uint32_t me = (uint32_t)(tile0 + S.ooff[i]);
                    put_bucket(table, me, lo64(nq >> shift), me, n, hdr);
                }
                break;
            }
            if (s != s_loaded) {
                const uint32_t nheavy = tilesum_ldcg(incl + s).nheavy;
                if (nheavy == 0) { // on to the tile of the first heavy after this one
                    const uint32_t nh = split[s].next_heavy;
                    s = nh == kNone ? ntiles : nh / (uint32_t)kTile;
                    continue;
                }
                if (y_tile != s && nheavy > (uint32_t)kSparse) {
                    load_items(w, n, vec, (uint64_t)s * kTile + (uint64_t)threadIdx.x * kItems, y);
                    y_tile = s;
                }
                __syncthreads(); // previous window consumed
                load_heavies<F32>(S, s, y, nheavy, n, n32, incl, slist, w, Q, light_max, beta);
                s_loaded = s;
                if (s + 1 < ntiles) { // prefetch the following stream tile
                    load_items(w, n, vec, (uint64_t)(s + 1) * kTile + (uint64_t)threadIdx.x * kItems, y);
                    y_tile = s + 1;
                }
            }
            const uint32_t hc = S.hcount;
            // position of the first heavy after stream tile s (kNone: none),
            // read while the block waits at the barrier
            const uint32_t hnext = split[s].next_heavy;
            __syncthreads(); // own keys and window complete
            if (threadIdx.x < 3 * 32) { // one warp per search
                const int q = threadIdx.x >> 5;
                uint32_t r;
                if (q == 0) r = warp_search(S.okey, al, nl, S.hkey[swz(hc - 1)], false); // lights answered here
                else if (q == 1) r = warp_search(S.hkey, 0, hc, D_start, true);          // heavies packed here:
                else r = warp_search(S.hkey, 0, hc, D_end, true);                        // E in (D_start, D_end]
                if ((threadIdx.x & 31) == 0) S.rng[1 + q] = r;
            }
            __syncthreads();
            const uint32_t a0 = al, a1 = S.rng[1], b0 = S.rng[2], b1 = S.rng[3];
            if (WRS_CHECK && !check_ok(hc <= (uint32_t)kTile && nl <= (uint32_t)kTile && a0 <= a1 && a1 <= nl &&
                                           b0 <= b1 && b1 <= hc, hdr))
                break;
            const uint32_t na = a1 - a0, nb = b1 > b0 ? b1 - b0 : 0, M = na + nb;
            const uint32_t per = (M + kThreads - 1) / kThreads;
            const uint64_t sbase = (uint64_t)s * kTile;
            const uint32_t d0 = threadIdx.x * per;
            if (d0 < M) {
                // co-rank: number of heavies among the first d0 merged elements
                uint32_t lo = d0 > na ? d0 - na : 0, hi = d0 < nb ? d0 : nb;
                while (lo < hi) {
                    const uint32_t mid = (lo + hi + 1) >> 1; // is heavy b0+mid-1 before light a0+d0-mid?
                    if (S.hkey[swz(b0 + mid - 1)] <= S.okey[swz(a0 + d0 - mid)]) lo = mid; else hi = mid - 1;
                }
                uint32_t j = b0 + lo, i = a0 + (d0 - lo);
                const uint32_t steps = min(per, M - d0);
                u128 ej = j < b1 ? S.hkey[swz(j)] : (u128)0;
                u128 di = i < nl ? S.okey[swz(i)] : D_end; // key of light i (D_end past the last)
                // positions of heavies j and j + 1 (the first heavy after the
                // stream tile past its last), kept in registers along the walk
                auto hpos = [&](uint32_t jj) -> uint32_t {
                    return jj < hc ? (uint32_t)(sbase + S.hoff[jj]) : hnext;
                };
                uint32_t hp = hpos(j), hp1 = hpos(j + 1);
                if (narrow) {
                    // Q < 2^64 (shift 0): a bucket's mass, a light's deficit
                    // and a heavy's gap D - E (< Q when the build is sound,
                    // checked in full) are 64-bit; only the keys are wider
                    const uint64_t Q64 = lo64(Q);
                    for (uint32_t st = 0; st < steps; ++st) {
                        const bool heavy_next = (j < b1) && (i >= a1 || ej <= di);
                        uint32_t me, alias;
                        uint64_t bw;
                        if (heavy_next) {
                            const u128 gap = di - ej;
                            if (hi64(gap) != 0 || lo64(gap) >= Q64) bad = true;
                            bw = Q64 - lo64(gap);
                            me = hp;
                            if (hp1 == kNone && bw != Q64) bad = true;
                            alias = (hp1 == kNone || bw == Q64) ? me : hp1;
                            ++j;
                            if (j < b1) ej = S.hkey[swz(j)];
                            hp = hp1;
                            hp1 = hpos(j + 1);
                        } else {
                            if (WRS_CHECK && !check_ok(i < a1, hdr)) break;
                            const u128 dn = (i + 1 < nl) ? S.okey[swz(i + 1)] : D_end;
                            const uint64_t def = lo64(dn) - lo64(di); // < Q: exact modulo 2^64
                            bw = Q64 - def;
                            me = (uint32_t)(tile0 + S.ooff[i]);
                            alias = (def == 0) ? me : hp;
                            ++i;
                            di = dn;
                        }
                        put_bucket(table, me, bw, alias, n, hdr);
                    }
                } else {
                    for (uint32_t st = 0; st < steps; ++st) {
                        const bool heavy_next = (j < b1) && (i >= a1 || ej <= di);
                        uint32_t me, alias;
                        u128 bw;
                        if (heavy_next) {
                            const u128 gap = di - ej;
                            if (gap >= Q) bad = true;
                            bw = Q - gap;
                            me = hp;
                            if (hp1 == kNone && bw != Q) bad = true;
                            alias = (hp1 == kNone || bw == Q) ? me : hp1;
                            ++j;
                            if (j < b1) ej = S.hkey[swz(j)];
                            hp = hp1;
                            hp1 = hpos(j + 1);
                        } else { // light i; j < hc: heavy j is its current heavy
                            if (WRS_CHECK && !check_ok(i < a1, hdr)) break;
                            const u128 dn = (i + 1 < nl) ? S.okey[swz(i + 1)] : D_end;
                            bw = Q - (dn - di);
                            me = (uint32_t)(tile0 + S.ooff[i]);
                            alias = (bw == Q) ? me : hp;
                            ++i;
                            di = dn;
                        }
                        put_bucket(table, me, lo64(bw >> shift), alias, n, hdr);
                    }
                }
            }
            al = a1;
            if (b1 < hc) { // the first heavy past D_end is in this tile: this own tile is done
                // end of the subproblem: the stream tile carried to the next
                // own tile is the one k_split found for it independently
                if (WRS_CHECK && threadIdx.x == 0 && c + 1 < ntiles) check_ok(split[c + 1].hb == s, hdr);
                break;
            }
            s = hnext == kNone ? ntiles : hnext / (uint32_t)kTile; // the next stream tile with a heavy
        }
    }
    if (bad) set_status(hdr, kEInternal);
}

// Block b packs own tiles [b * group, (b + 1) * group): one subproblem of
// Alg. 3 per block (group = kSweepTiles unless the caller asks for a split
// count); force_wide runs the 128-bit walk even when Q < 2^64.
template <int F32>
__global__ void __launch_bounds__(kThreads, 3) k_sweep(const uint32_t *__restrict__ w, uint64_t n, int vec,
                                                       DevHeader *hdr, const TileSum *__restrict__ incl,
                                                       const Split *__restrict__ split,
                                                       const uint16_t *__restrict__ slist, uint32_t ntiles,
                                                       uint4 *__restrict__ table, uint32_t group, int force_wide)
{
    const uint32_t c_first = blockIdx.x * group;
    sweep_body<F32>(w, n, vec, hdr, incl, split, slist, ntiles, table, c_first, min(c_first + group, ntiles),
                    force_wide != 0);
}

// The exact sum was asked to fit 64 bits (accumulator mode U64): Q >= 2^64
// fails the build with WRS_EOVERFLOW before the sweep.
__global__ void k_require_u64(DevHeader *hdr)
{
    if (threadIdx.x == 0 && hdr->status == 0 && hdr->q_hi != 0) set_status(hdr, kEOverflow);
}

// ----------------------------------------------------------- k_sample
// A query reads one random 16-B bucket.  The .L2::64B size hint makes the L2
// fetch 64 B per miss instead of 128 B: half the DRAM bytes per sample, a few
// percent faster (random sampling is bound by DRAM accesses, not bytes).
__device__ __forceinline__ uint4 ld_bucket(const uint4 *p)
{
    uint4 v;
    asm volatile("ld.global.nc.L2::64B.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

constexpr int kSampleUnroll = 8;

// Samples first, first + stride, ... (below k) of one table.
__device__ __forceinline__ void sample_body(const uint4 *__restrict__ tab, uint64_t n, uint64_t qp, uint64_t k,
                                            uint32_t key0, uint32_t key1, uint32_t sid0, uint32_t sid1,
                                            uint32_t *__restrict__ out, uint64_t first, uint64_t stride,
                                            const DevHeader *chk = nullptr)
{
    for (uint64_t s = first; s < k; s += kSampleUnroll * stride) {
        uint64_t r[kSampleUnroll], v[kSampleUnroll];
        uint4 b[kSampleUnroll];
#pragma unroll
        for (int j = 0; j < kSampleUnroll; ++j) {
            const uint64_t sj = s + j * stride;
            P4 c;
            c.x0 = (uint32_t)sj; c.x1 = (uint32_t)(sj >> 32); c.x2 = sid0; c.x3 = sid1;
            const P4 o = philox4x32_10(c, key0, key1);
            const uint64_t u = o.x0 | ((uint64_t)o.x1 << 32);
            v[j] = o.x2 | ((uint64_t)o.x3 << 32);
            r[j] = __umul64hi(u, n);
        }
#pragma unroll
        for (int j = 0; j < kSampleUnroll; ++j)
            if (s + j * stride < k) b[j] = ld_bucket(tab + r[j]);
#pragma unroll
        for (int j = 0; j < kSampleUnroll; ++j) {
            const uint64_t sj = s + j * stride;
            if (sj < k) {
                const uint64_t thr = b[j].x | ((uint64_t)b[j].y << 32);
                if (WRS_CHECK && chk) check_ok(b[j].z < n, const_cast<DevHeader *>(chk));
                const uint32_t pick = (__umul64hi(v[j], qp) < thr) ? (uint32_t)r[j] : b[j].z;
                __stcs(out + sj, pick);
            }
        }
    }
}

// Samples [s0, k) of one table.
__global__ void __launch_bounds__(256) k_sample(const uint4 *__restrict__ tab, uint64_t n,
                                                const DevHeader *__restrict__ hdr, uint64_t s0, uint64_t k,
                                                uint32_t key0, uint32_t key1, uint32_t sid0, uint32_t sid1,
                                                uint32_t *__restrict__ out)
{
    if (hdr->status) return;
    sample_body(tab, n, hdr->qp, k, key0, key1, sid0, sid1, out,
                s0 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, (uint64_t)gridDim.x * blockDim.x, hdr);
}

} // namespace wrs
