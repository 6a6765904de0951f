// wrs_device.cuh -- shared device definitions of libwrs (layouts, 128-bit
// helpers, Philox, block scans).  Included by wrs.cu only.
#pragma once

#include <cstdint>
#include <climits>

typedef unsigned __int128 u128;

namespace wrs {

// ---------------------------------------------------------------- layout
constexpr int kThreads = 256;               // threads per block of the build
constexpr int kItems = 8;                   // weights per thread
constexpr int kTile = kThreads * kItems;    // weights per tile (2048)
constexpr int kWarps = kThreads / 32;
constexpr int kChunk = 32 * kItems;         // weights of one warp's share of a tile (256)
constexpr int kChunks = kTile / kChunk;     // chunks per tile (8)
constexpr int kSparse = 32;                 // member lists of tiles with <= 32 heavies (or lights)
constexpr int kScanChunk = kThreads;        // tile aggregates per block of the look-back scan
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr int kQBits = 95;                  // Q < 2^95 keeps n*Q < 2^127
constexpr uint32_t kFlagAgg = 1u, kFlagIncl = 2u;

// status codes (mirror wrs_status)
constexpr uint32_t kOk = 0, kEInval = 1, kEOverflow = 3, kETimeout = 4, kEInternal = 6;

// Device-resident header of a table; written by the build, read by the
// sampler.  All fields but the first two are set by k_stats_combine.
struct DevHeader {
    uint32_t status;        // first error wins (atomicCAS from 0)
    uint32_t tile_counter;  // dynamic tile ids of the look-back scan
    int32_t beta;
    uint32_t shift;
    uint64_t q_lo, q_hi;    // Q
    uint64_t qp;            // Q >> shift
    uint32_t light_max;     // light iff raw word <= light_max
    uint32_t f32;
    uint64_t n;
    uint64_t n_light;       // filled by the sweep of the last tile
    uint64_t pad[2];        // zero; the check build counts failed checks in pad[0]
};

struct Partial {            // per-block result of k_stats
    uint64_t lo, hi;        // exact partial sum (units of 2^base)
    int32_t base;           // INT_MAX: no nonzero weight seen
    uint32_t flags;         // bit 0 invalid weight, bit 1 range exceeded
    uint64_t pad;
};
constexpr uint32_t kPartInvalid = 1u, kPartOverflow = 2u;

struct TileSum {            // per-tile aggregate, or inclusive prefix over tiles (48 B)
    uint64_t l_lo, l_hi;    // sum of q over light items
    uint64_t h_lo, h_hi;    // sum of q over heavy items
    uint32_t cl;            // number of light items
    uint32_t nheavy;        // heavy items in this tile alone (also kept in the prefix)
    uint32_t first_heavy;   // offset of the first heavy item in this tile, or kNone
    uint32_t pad;
};

struct Split {              // per-tile result of k_split
    uint32_t hb;            // tile holding the heavy current at this tile's first light
    uint32_t lb;            // a tile at or before the one holding the light that follows
                            // this tile's first heavy
    uint32_t next_heavy;    // position of the first heavy item after this tile
    uint32_t pad;
};

// ------------------------------------------------------------ 128-bit ops
__device__ __forceinline__ u128 mk128(uint64_t lo, uint64_t hi) { return ((u128)hi << 64) | lo; }
__device__ __forceinline__ uint64_t lo64(u128 v) { return (uint64_t)v; }
__device__ __forceinline__ uint64_t hi64(u128 v) { return (uint64_t)(v >> 64); }

__device__ __forceinline__ int bitlen128(u128 v)
{
    uint64_t h = hi64(v), l = lo64(v);
    return h ? 128 - __clzll((long long)h) : (l ? 64 - __clzll((long long)l) : 0);
}

__device__ __forceinline__ u128 shfl_up128(u128 v, int d)
{
    uint64_t l = __shfl_up_sync(0xFFFFFFFFu, lo64(v), d);
    uint64_t h = __shfl_up_sync(0xFFFFFFFFu, hi64(v), d);
    return mk128(l, h);
}

__device__ __forceinline__ u128 shfl_down128(u128 v, int d)
{
    uint64_t l = __shfl_down_sync(0xFFFFFFFFu, lo64(v), d);
    uint64_t h = __shfl_down_sync(0xFFFFFFFFu, hi64(v), d);
    return mk128(l, h);
}

__device__ __forceinline__ u128 shfl_idx128(u128 v, int src)
{
    uint64_t l = __shfl_sync(0xFFFFFFFFu, lo64(v), src);
    uint64_t h = __shfl_sync(0xFFFFFFFFu, hi64(v), src);
    return mk128(l, h);
}

// n * q for n < 2^32 and q < 2^95
__device__ __forceinline__ u128 times_n(u128 q, uint64_t n) { return q * (u128)n; }

// ------------------------------------------------ weights -> exact integers
// binary32 word -> q = w * 2^-beta (exact; caller guarantees validity)
__device__ __forceinline__ u128 q_of(uint32_t x, uint32_t f32, int beta)
{
    if (!f32) return (u128)x;
    uint32_t ex = (x >> 23) & 0xFFu;
    uint32_t m = x & 0x7FFFFFu;
    if (ex) m |= 0x800000u;
    if (!m) return 0;
    int sh = (ex ? (int)ex : 1) - 150 - beta;
    return sh >= 0 ? ((u128)m << sh) : (u128)(m >> (-sh));
}

// ----------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): per round two
// 32x32->64 products of counter words 0 and 2 with fixed multipliers, mixed
// with words 1 and 3 and the key; the key advances by the Weyl constants
// between rounds.
struct P4 { uint32_t x0, x1, x2, x3; };

__device__ __forceinline__ P4 philox4x32_10(P4 c, uint32_t k0, uint32_t k1)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(M0, c.x0), lo0 = M0 * c.x0;
        uint32_t hi1 = __umulhi(M1, c.x2), lo1 = M1 * c.x2;
        P4 d;
        d.x0 = hi1 ^ c.x1 ^ k0;
        d.x1 = lo1;
        d.x2 = hi0 ^ c.x3 ^ k1;
        d.x3 = lo0;
        c = d;
        k0 += W0;
        k1 += W1;
    }
    return c;
}

// ------------------------------------------------------- memory ordering
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void set_status(DevHeader *h, uint32_t code)
{
    atomicCAS(&h->status, 0u, code);
}

// ------------------------------------------------------- check build
// libwrs_check.so is this library compiled with -DWRS_CHECK=1.  There, every
// bucket store adds one to the bucket's reserved fourth word instead of
// storing 0 (the build clears the buckets first, so a table in which every
// bucket was written exactly once has 1 in every reserved word), a bucket
// index or alias outside the table is refused, and the index checks placed
// on the sweep's shared-memory reads and on its end-of-subproblem state
// hold.  A check that fails counts itself in the header's first reserved
// word, sets WRS_EINTERNAL and skips the access.  In the standard build all
// of this compiles away and the reserved word is stored as 0.
#ifndef WRS_CHECK
#define WRS_CHECK 0
#endif

__device__ __noinline__ void check_fail(DevHeader *h)
{
    atomicAdd(reinterpret_cast<unsigned long long *>(&h->pad[0]), 1ull);
    set_status(h, kEInternal);
}

// True when cond holds; in the check build a false cond is recorded.
__device__ __forceinline__ bool check_ok(bool cond, DevHeader *h)
{
    if (WRS_CHECK && !cond) {
        check_fail(h);
        return false;
    }
    return true;
}

// Bucket me of a table of `limit` buckets: threshold thr, alias.
__device__ __forceinline__ void put_bucket(uint4 *table, uint64_t me, uint64_t thr, uint32_t alias, uint64_t limit,
                                           DevHeader *h)
{
#if WRS_CHECK
    if (me >= limit || alias >= limit) {
        check_fail(h);
        return;
    }
    uint32_t *p = reinterpret_cast<uint32_t *>(table + me);
    *reinterpret_cast<uint2 *>(p) = make_uint2((uint32_t)thr, (uint32_t)(thr >> 32));
    p[2] = alias;
    atomicAdd(p + 3, 1u);
#else
    (void)limit;
    (void)h;
    table[me] = make_uint4((uint32_t)thr, (uint32_t)(thr >> 32), alias, 0u);
#endif
}

// The table's status, read once for the whole block: every thread returns
// or none does, so no later block barrier waits for threads that left.
__device__ __forceinline__ bool block_stopped(const DevHeader *hdr)
{
    __shared__ uint32_t s_status_word;
    if (threadIdx.x == 0) s_status_word = *(volatile const uint32_t *)&hdr->status;
    __syncthreads();
    return s_status_word != 0;
}

// --------------------------------------------------------- block scans
// Exclusive scan of a u32 over the block (all threads call; uses sm[kWarps]).
__device__ __forceinline__ uint32_t block_exclusive_scan_u32(uint32_t v, uint32_t &total, uint32_t *sm)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t o = __shfl_up_sync(0xFFFFFFFFu, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) sm[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint32_t t = lane < kWarps ? sm[lane] : 0u;
#pragma unroll
        for (int d = 1; d < kWarps; d <<= 1) {
            uint32_t o = __shfl_up_sync(0xFFFFFFFFu, t, d);
            if (lane >= d) t += o;
        }
        if (lane < kWarps) sm[lane] = t;
    }
    __syncthreads();
    const uint32_t base = wid ? sm[wid - 1] : 0u;
    total = sm[kWarps - 1];
    __syncthreads();
    return base + inc - v;
}

// Minimum of a u128 over the block, returned to every thread (uses sm[kWarps]).
__device__ __forceinline__ u128 block_min_u128(u128 v, u128 *sm)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        u128 o = shfl_down128(v, d);
        if (o < v) v = o;
    }
    if (lane == 0) sm[wid] = v;
    __syncthreads();
    u128 m = sm[0];
#pragma unroll
    for (int i = 1; i < kWarps; ++i)
        if (sm[i] < m) m = sm[i];
    __syncthreads();
    return m;
}

// Exclusive scan of two u128 values over the block; `total` gets the sums.
// Must be called by all threads; uses `sm` (kWarps entries).
struct U2 { u128 a, b; };

__device__ __forceinline__ U2 block_exclusive_scan2(U2 v, U2 &total, U2 *sm)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    U2 inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        u128 a = shfl_up128(inc.a, d), b = shfl_up128(inc.b, d);
        if (lane >= d) { inc.a += a; inc.b += b; }
    }
    if (lane == 31) sm[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        U2 t = lane < kWarps ? sm[lane] : U2{0, 0};
#pragma unroll
        for (int d = 1; d < kWarps; d <<= 1) {
            u128 a = shfl_up128(t.a, d), b = shfl_up128(t.b, d);
            if (lane >= d) { t.a += a; t.b += b; }
        }
        if (lane < kWarps) sm[lane] = t;
    }
    __syncthreads();
    U2 base = wid ? sm[wid - 1] : U2{0, 0};
    total = sm[kWarps - 1];
    __syncthreads();
    U2 r;
    r.a = base.a + inc.a - v.a;
    r.b = base.b + inc.b - v.b;
    return r;
}

} // namespace wrs
