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

template <int F32>
__device__ __forceinline__ void acc_take(Acc &a, uint32_t x)
{
    if (!F32) { a.acc += x; return; }
    uint32_t ex = (x >> 23) & 0xFFu;
    if ((x >> 31) || ex == 0xFFu) { a.flags |= kPartInvalid; return; }
    uint32_t m = x & 0x7FFFFFu;
    if (ex) m |= 0x800000u;
    if (!m) return;
    int e = (ex ? (int)ex : 1) - 150;
    int lsb = e + __ffs(m) - 1;
    if (lsb < a.base) {
        if (a.acc) {
            int d = a.base - lsb;
            if (bitlen128(a.acc) + d > kQBits) { a.flags |= kPartOverflow; a.acc = 0; }
            else a.acc <<= d;
        }
        a.base = lsb;
    }
    int sh = e - a.base;
    u128 q;
    if (sh >= 0) {
        if ((32 - __clz(m)) + sh > kQBits) { a.flags |= kPartOverflow; return; }
        q = (u128)m << sh;
    } else {
        q = (u128)(m >> (-sh));
    }
    a.acc += q;
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

template <int F32>
__global__ void __launch_bounds__(kThreads) k_stats(const uint32_t *__restrict__ w, uint64_t n, int vec,
                                                    Partial *__restrict__ part)
{
    Acc a;
    a.base = F32 ? INT_MAX : 0;
    a.acc = 0;
    a.flags = 0;
    const uint64_t tid = (uint64_t)blockIdx.x * kThreads + threadIdx.x;
    const uint64_t nth = (uint64_t)gridDim.x * kThreads;
    const uint64_t nv = vec ? n / 4 : 0;
    const uint4 *w4 = reinterpret_cast<const uint4 *>(w);
    uint64_t i = tid;
    for (; i + 3 * nth < nv; i += 4 * nth) {
        uint4 v0 = __ldg(w4 + i), v1 = __ldg(w4 + i + nth), v2 = __ldg(w4 + i + 2 * nth), v3 = __ldg(w4 + i + 3 * nth);
        acc_take<F32>(a, v0.x); acc_take<F32>(a, v0.y); acc_take<F32>(a, v0.z); acc_take<F32>(a, v0.w);
        acc_take<F32>(a, v1.x); acc_take<F32>(a, v1.y); acc_take<F32>(a, v1.z); acc_take<F32>(a, v1.w);
        acc_take<F32>(a, v2.x); acc_take<F32>(a, v2.y); acc_take<F32>(a, v2.z); acc_take<F32>(a, v2.w);
        acc_take<F32>(a, v3.x); acc_take<F32>(a, v3.y); acc_take<F32>(a, v3.z); acc_take<F32>(a, v3.w);
    }
    for (; i < nv; i += nth) {
        uint4 v = __ldg(w4 + i);
        acc_take<F32>(a, v.x); acc_take<F32>(a, v.y); acc_take<F32>(a, v.z); acc_take<F32>(a, v.w);
    }
    for (uint64_t j = nv * 4 + tid; j < n; j += nth) acc_take<F32>(a, __ldg(w + j));
    a = acc_block_reduce(a);
    if (threadIdx.x == 0) {
        Partial p;
        p.lo = lo64(a.acc); p.hi = hi64(a.acc); p.base = a.base; p.flags = a.flags; p.pad = 0;
        part[blockIdx.x] = p;
    }
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

__global__ void __launch_bounds__(kThreads) k_stats_combine(const Partial *__restrict__ part, uint32_t nparts,
                                                            uint64_t n, uint32_t f32, DevHeader *hdr)
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
    if (threadIdx.x != 0) return;
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
    __threadfence();
    hdr->status = status;
}

// ---------------------------------------------------------- k_classify
// One 2048-weight tile per iteration of a grid-stride loop (no dependency
// between tiles): light count, light and heavy sums, the tile's heavy count
// and first heavy offset, and -- when one class has at most 32 members in the
// tile -- the offsets of those members.
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

template <int F32>
__global__ void __launch_bounds__(kThreads) k_classify(const uint32_t *__restrict__ w, uint64_t n, int vec,
                                                       const DevHeader *__restrict__ hdr, TileSum *__restrict__ agg,
                                                       uint16_t *__restrict__ slist, uint32_t ntiles)
{
    __shared__ U2 s_scan[kWarps];
    __shared__ uint32_t s_cnt[kWarps];
    __shared__ uint32_t s_first[kWarps];
    if (*(volatile const uint32_t *)&hdr->status) return;
    const uint32_t light_max = hdr->light_max;
    const int beta = hdr->beta;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint64_t tile0 = (uint64_t)t * kTile;
        const uint64_t first = tile0 + (uint64_t)threadIdx.x * kItems;
        uint32_t x[kItems];
        load_items(w, n, vec, first, x);
        uint32_t cl = 0, nh = 0, fh = kNone;
        u128 L = 0, H = 0;
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            if (first + k < n) {
                const u128 q = q_of(x[k], F32, beta);
                if (x[k] <= light_max) { ++cl; L += q; }
                else { ++nh; H += q; if (fh == kNone) fh = threadIdx.x * kItems + k; }
            }
        }
        U2 tot;
        block_exclusive_scan2(U2{L, H}, tot, s_scan);
        uint32_t ctot;
        const uint32_t cex = block_exclusive_scan_u32(cl | (nh << 16), ctot, s_cnt);
        uint32_t f = fh;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) f = min(f, __shfl_xor_sync(0xFFFFFFFFu, f, d));
        if (lane == 0) s_first[wid] = f;
        __syncthreads();
        const uint32_t tot_l = ctot & 0xFFFFu, tot_h = ctot >> 16;
        if (threadIdx.x == 0) {
            TileSum a;
            a.l_lo = lo64(tot.a); a.l_hi = hi64(tot.a); a.h_lo = lo64(tot.b); a.h_hi = hi64(tot.b);
            a.cl = tot_l; a.nheavy = tot_h; a.first_heavy = kNone; a.pad = 0;
#pragma unroll
            for (int i = 0; i < kWarps; ++i) a.first_heavy = min(a.first_heavy, s_first[i]);
            tilesum_st(agg + t, a);
        }
        // member list of a sparse class (heavies first)
        const bool list_heavy = tot_h <= (uint32_t)kSparse;
        const bool list_light = !list_heavy && tot_l <= (uint32_t)kSparse;
        if (list_heavy || list_light) {
            uint32_t slot = list_heavy ? (cex >> 16) : (cex & 0xFFFFu);
#pragma unroll
            for (int k = 0; k < kItems; ++k) {
                if (first + k < n) {
                    const bool is_light = x[k] <= light_max;
                    if (is_light == list_light) {
                        slist[(uint64_t)t * kSparse + slot] = (uint16_t)(threadIdx.x * kItems + k);
                        ++slot;
                    }
                }
            }
        }
        __syncthreads();
    }
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

__global__ void __launch_bounds__(kThreads) k_tilescan(DevHeader *hdr, const TileSum *__restrict__ agg,
                                                       TileSum *chunk_agg, TileSum *chunk_incl,
                                                       TileSum *__restrict__ incl, uint32_t *flags,
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

__global__ void __launch_bounds__(kThreads) k_split(const TileSum *__restrict__ incl, uint32_t ntiles, uint64_t n,
                                                    DevHeader *hdr, Split *__restrict__ split)
{
    if (*(volatile uint32_t *)&hdr->status) return;
    const uint32_t c = blockIdx.x * kThreads + threadIdx.x;
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

__device__ __forceinline__ uint32_t upper_bound_keys(const u128 *key, uint32_t cnt, u128 v)
{ // first index with key > v
    uint32_t lo = 0, hi = cnt;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (key[mid] <= v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t lower_bound_keys(const u128 *key, uint32_t cnt, u128 v)
{ // first index with key >= v
    uint32_t lo = 0, hi = cnt;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (key[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// ------------------------------------------------------------ k_sweep
// Tile c packs, as Alg. 3's pack does for one subproblem, the buckets of its
// own lights and of every heavy item whose key E lies in (D_c, D_c'] (D_c:
// key of the tile's first light, D_c': key after its last light), i.e. the
// heavy items Alg. 2 packs while it consumes this tile's lights.  The heavy
// items come in index order from the tile k_split named (the split of Alg. 3
// on the heavy prefix sums) into a window in shared memory (keys and
// positions); the first two tiles of that stream are loaded together with the
// own tile.  Thread t owns 8 consecutive items; with K_t the key of its first
// light and K_t' the key after its last, it resolves
//   its lights:  alias = first heavy with E > D (the current heavy);
//   the heavies with E in (K_t, K_t']:  bucket Q - (D_next - E), D_next = key
//                of the first light with D >= E, alias = the next heavy.
// A stream longer than the window is consumed in rounds.
struct Win {
    u128 key[kTile];
    uint32_t pos[kTile];
    uint32_t count;
    uint32_t done;       // the last entry ends the stream
    uint32_t tile;       // next stream tile
    uint32_t pad;
    uint64_t next_rank;  // heavy rank of the next entry to take
};

// Append heavies of stream tile t (words in x, loaded by the caller) to W:
// ranks >= W.next_rank with key > lo, up to and including the first key > hi,
// while W has room.  All threads call.
template <int F32>
__device__ void stream_tile(Win &W, uint32_t t, const uint32_t (&x)[kItems], uint64_t n, const TileSum *incl,
                            const uint16_t *__restrict__ slist, const uint32_t *__restrict__ w, u128 Q,
                            uint32_t light_max, int beta, u128 lo, u128 hi, U2 *s_scan,
                            unsigned long long *s_min)
{
    const Prefix pf = prefix_at(incl, t, n);
    const u128 base = key_E(pf, n, Q);
    const uint64_t rank0 = pf.ch;
    const uint64_t tile0 = (uint64_t)t * kTile;
    const uint32_t nheavy = tilesum_ldcg(incl + t).nheavy;
    const uint32_t count = W.count;
    const uint64_t next_rank = W.next_rank;
    const uint32_t room = (uint32_t)kTile - count;
    if (nheavy <= (uint32_t)kSparse) { // member list: one warp
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            u128 d = 0;
            uint32_t off = 0;
            if ((uint32_t)lane < nheavy) {
                off = slist[(uint64_t)t * kSparse + lane];
                d = times_n(q_of(__ldg(w + tile0 + off), F32, beta), n) - Q;
            }
            u128 key = d;
#pragma unroll
            for (int s = 1; s < 32; s <<= 1) {
                const u128 o = shfl_up128(key, s);
                if (lane >= s) key += o;
            }
            key += base;
            const uint64_t r = rank0 + lane;
            const bool mem = (uint32_t)lane < nheavy;
            const bool keep = mem && r >= next_rank && key > lo;
            const uint32_t km = __ballot_sync(0xFFFFFFFFu, keep);
            const uint32_t tm = __ballot_sync(0xFFFFFFFFu, mem && key > hi);
            const int first_keep = km ? __ffs(km) - 1 : 32;
            const int first_term = tm ? __ffs(tm) - 1 : 32;
            int end = (int)nheavy;
            if (first_term + 1 < end) end = first_term + 1;
            if (first_keep + (int)room < end) end = first_keep + (int)room;
            if (keep && lane < end) {
                const uint32_t slot = count + (uint32_t)(lane - first_keep);
                W.key[slot] = key;
                W.pos[slot] = (uint32_t)(tile0 + off);
            }
            if (lane == 0) {
                const int taken = first_keep < end ? end - first_keep : 0;
                W.count = count + (uint32_t)taken;
                if (first_keep < end) W.next_rank = rank0 + (uint64_t)end;
                if (first_term < end) W.done = 1;
                if (end >= (int)nheavy) W.tile = t + 1;
            }
        }
        __syncthreads();
        return;
    }
    const uint64_t first = tile0 + (uint64_t)threadIdx.x * kItems;
    uint32_t cnt = 0;
    u128 sum = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        if (first + k < n && x[k] > light_max) {
            sum += times_n(q_of(x[k], F32, beta), n) - Q;
            ++cnt;
        }
    }
    U2 tot;
    const U2 ex = block_exclusive_scan2(U2{(u128)cnt, sum}, tot, s_scan);
    if (threadIdx.x == 0) { s_min[0] = ~0ull; s_min[1] = ~0ull; }
    __syncthreads();
    {
        uint64_t r = rank0 + (uint64_t)ex.a;
        u128 key = base + ex.b;
        unsigned long long fk = ~0ull, ft = ~0ull;
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            if (first + k < n && x[k] > light_max) {
                key += times_n(q_of(x[k], F32, beta), n) - Q;
                if (fk == ~0ull && r >= next_rank && key > lo) fk = r;
                if (ft == ~0ull && key > hi) ft = r;
                ++r;
            }
        }
        if (fk != ~0ull) atomicMin(&s_min[0], fk);
        if (ft != ~0ull) atomicMin(&s_min[1], ft);
    }
    __syncthreads();
    const uint64_t r_start = s_min[0], r_term = s_min[1];
    const uint64_t r_tile_end = rank0 + (uint64_t)tot.a;
    uint64_t r_end = r_tile_end;
    if (r_term != ~0ull && r_term + 1 < r_end) r_end = r_term + 1;
    if (r_start != ~0ull && r_start + room < r_end) r_end = r_start + room;
    if (r_start != ~0ull) {
        uint64_t r = rank0 + (uint64_t)ex.a;
        u128 key = base + ex.b;
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            if (first + k < n && x[k] > light_max) {
                key += times_n(q_of(x[k], F32, beta), n) - Q;
                if (r >= r_start && r < r_end) {
                    const uint32_t slot = count + (uint32_t)(r - r_start);
                    W.key[slot] = key;
                    W.pos[slot] = (uint32_t)(first + k);
                }
                ++r;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (r_start != ~0ull) {
            W.count = count + (uint32_t)(r_end - r_start);
            W.next_rank = r_end;
            if (r_term != ~0ull && r_term < r_end) W.done = 1;
        }
        if (r_start == ~0ull || r_end == r_tile_end) W.tile = t + 1;
    }
    __syncthreads();
}

template <int F32>
__global__ void __launch_bounds__(kThreads, 2) k_sweep(const uint32_t *__restrict__ w, uint64_t n, int vec,
                                                       DevHeader *hdr, const TileSum *__restrict__ incl,
                                                       const Split *__restrict__ split,
                                                       const uint16_t *__restrict__ slist, uint32_t ntiles,
                                                       uint4 *__restrict__ table)
{
    __shared__ Win W;
    __shared__ U2 s_scan[kWarps];
    __shared__ unsigned long long s_min[2];
    if (*(volatile uint32_t *)&hdr->status) return;
    const uint32_t c = blockIdx.x;
    const Split sp = split[c];
    const u128 Q = mk128(hdr->q_lo, hdr->q_hi);
    const uint32_t light_max = hdr->light_max;
    const int beta = hdr->beta;
    const uint32_t shift = hdr->shift;
    const uint64_t tile0 = (uint64_t)c * kTile;
    const uint64_t first = tile0 + (uint64_t)threadIdx.x * kItems;

    // own tile and the first two stream tiles, loaded together
    uint32_t x[kItems], xa[kItems], xb[kItems];
    load_items(w, n, vec, first, x);
    const uint32_t s0 = sp.hb;
    if (s0 < ntiles) load_items(w, n, vec, (uint64_t)s0 * kTile + (uint64_t)threadIdx.x * kItems, xa);
    if (s0 + 1 < ntiles) load_items(w, n, vec, (uint64_t)(s0 + 1) * kTile + (uint64_t)threadIdx.x * kItems, xb);

    const Prefix pc = prefix_at(incl, c, n);
    const u128 D_start = key_D(pc, n, Q);
    uint32_t lmask = 0;
    u128 def = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        if (first + k < n && x[k] <= light_max) {
            lmask |= 1u << k;
            def += Q - times_n(q_of(x[k], F32, beta), n);
        }
    }
    U2 tot;
    const U2 ex = block_exclusive_scan2(U2{def, (u128)0}, tot, s_scan);
    const u128 K0 = D_start + ex.a; // key of my first light
    const u128 K1 = K0 + def;       // key after my last light
    const u128 D_end = D_start + tot.a;

    uint64_t rthr[kItems];
    uint32_t ralias[kItems];
#pragma unroll
    for (int k = 0; k < kItems; ++k) { rthr[k] = 0; ralias[k] = 0; }
    uint32_t pend = lmask;
    bool bad = false;
    if (threadIdx.x == 0) {
        W.count = 0;
        W.done = 0;
        W.tile = s0;
        W.next_rank = 0;
    }
    __syncthreads();
    if (!__syncthreads_or(lmask != 0)) return; // no lights: nothing is packed here

    for (int round = 0;; ++round) {
        // ---- fill the window
        if (threadIdx.x == 0) W.count = 0;
        __syncthreads();
        for (;;) {
            if (W.done || W.count >= (uint32_t)kTile) break;
            const uint32_t t = W.tile;
            if (t >= ntiles) {
                if (threadIdx.x == 0) {
                    W.key[W.count] = ~(u128)0;
                    W.pos[W.count] = kNone;
                    W.count += 1;
                    W.done = 1;
                }
                __syncthreads();
                break;
            }
            if (t == s0) stream_tile<F32>(W, t, xa, n, incl, slist, w, Q, light_max, beta, D_start, D_end, s_scan, s_min);
            else if (t == s0 + 1) stream_tile<F32>(W, t, xb, n, incl, slist, w, Q, light_max, beta, D_start, D_end, s_scan, s_min);
            else {
                uint32_t y[kItems];
                load_items(w, n, vec, (uint64_t)t * kTile + (uint64_t)threadIdx.x * kItems, y);
                stream_tile<F32>(W, t, y, n, incl, slist, w, Q, light_max, beta, D_start, D_end, s_scan, s_min);
            }
        }
        const uint32_t cnt = W.count;
        const bool complete = W.done != 0;
        // ---- my lights: alias = first heavy with E > D
        {
            u128 kl = K0;
            int yi = -1;
#pragma unroll
            for (int k = 0; k < kItems; ++k) {
                if ((lmask >> k) & 1u) {
                    const u128 nq = times_n(q_of(x[k], F32, beta), n);
                    const u128 key = kl;
                    kl += Q - nq;
                    if ((pend >> k) & 1u) {
                        if (yi < 0) yi = (int)upper_bound_keys(W.key, cnt, key);
                        else while ((uint32_t)yi < cnt && W.key[yi] <= key) ++yi;
                        if ((uint32_t)yi >= cnt) break;
                        const uint32_t al = W.pos[yi];
                        if (al == kNone && nq != Q) bad = true;
                        rthr[k] = lo64(nq >> shift);
                        ralias[k] = (al == kNone || nq == Q) ? (uint32_t)(first + k) : al;
                        pend &= ~(1u << k);
                    }
                }
            }
        }
        // ---- heavies with E in (K0, K1] among entries [0, cnt - 1)
        if (K1 > K0) {
            const uint32_t lim = cnt - 1;
            uint32_t ylo = upper_bound_keys(W.key, lim, K0);
            const uint32_t yhi = upper_bound_keys(W.key, lim, K1);
            u128 kl = K0;
            int k = 0;
            for (uint32_t yv = ylo; yv < yhi; ++yv) {
                const u128 e = W.key[yv];
                // advance to the first of my lights with key >= e (else K1)
                while (k < kItems) {
                    if ((lmask >> k) & 1u) {
                        if (kl >= e) break;
                        kl += Q - times_n(q_of(x[k], F32, beta), n);
                    }
                    ++k;
                }
                const u128 dnext = (k < kItems) ? kl : K1;
                const u128 gap = dnext - e;
                if (gap >= Q) bad = true;
                const u128 bw = Q - gap;
                const uint32_t me = W.pos[yv], nx = W.pos[yv + 1];
                if (nx == kNone && bw != Q) bad = true;
                const uint32_t al = (nx == kNone || bw == Q) ? me : nx;
                const uint64_t thr = lo64(bw >> shift);
                table[me] = make_uint4((uint32_t)thr, (uint32_t)(thr >> 32), al, 0u);
            }
        }
        if (complete) break;
        // the last entry waits for its successor: restart the stream there
        __syncthreads();
        if (threadIdx.x == 0) {
            W.next_rank = W.next_rank - 1;
            const uint32_t lastpos = W.pos[cnt - 1];
            W.tile = lastpos / (uint32_t)kTile;
        }
        __syncthreads();
    }
    if (pend) bad = true;
    if (bad) set_status(hdr, kEInternal);
    // ---- write my lights' buckets
#pragma unroll
    for (int k = 0; k < kItems; ++k)
        if ((lmask >> k) & 1u)
            table[first + k] = make_uint4((uint32_t)rthr[k], (uint32_t)(rthr[k] >> 32), ralias[k], 0u);
}

// ----------------------------------------------------------- k_sample
__device__ __forceinline__ uint4 ld_bucket(const uint4 *p)
{
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

constexpr int kSampleUnroll = 4;

__global__ void __launch_bounds__(256) k_sample(const uint4 *__restrict__ tab, uint64_t n,
                                                const DevHeader *__restrict__ hdr, uint64_t k, uint32_t key0,
                                                uint32_t key1, uint32_t sid0, uint32_t sid1,
                                                uint32_t *__restrict__ out)
{
    if (hdr->status) return;
    const uint64_t qp = hdr->qp;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < k; s += kSampleUnroll * stride) {
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
                const uint32_t pick = (__umul64hi(v[j], qp) < thr) ? (uint32_t)r[j] : b[j].z;
                __stcs(out + sj, pick);
            }
        }
    }
}

} // namespace wrs
