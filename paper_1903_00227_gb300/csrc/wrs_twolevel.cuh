// wrs_twolevel.cuh -- two-level ("2lvl-sweep") alias tables (the
// wrs_table2_* entry points of include/wrs.h).  Included by wrs.cu only.
//
// Sec. 6 ("Distributed Alias Table Construction", replicated top level) and
// Sec. 10 ("Implementation Details": 2lvl with Alg. 2 as the base case),
// applied recursively on one GPU: the n items are cut into groups of 2048
// consecutive items; each group gets its own Alg. 2 table in the group's own
// units (capacity Q_g = the group's total, member m weighs n_g * q_m with n_g
// the group's size); the group totals are the items of the next level, and so
// on up to a single group (n < 2^32 gives at most three levels).  A sample
// walks down from the top group: one Philox draw per level (key offset by the
// depth), a bucket of the current group, its coin, and the pick names the
// group one level down.
//
// Each group is built by ONE block, entirely in shared memory: exact member
// weights, the group total, light/heavy classification against it, the
// deficit and excess keys of Alg. 2 (the keys of the single-table sweep with
// the group as the whole input), and an evenly split merge of the two key
// sequences.  No global prefix, split search or cross-block traffic exists:
// besides the weight-total pass every weight is read once.
#pragma once

namespace wrs {

constexpr int kMaxLevels = WRS_TABLE2_MAX_LEVELS;

struct GroupRec {          // per group (mirrors wrs_group)
    uint64_t qp;           // Q_g >> shift
    uint32_t shift;        // max(0, bitlen(Q_g) - 64)
    uint32_t members;
};
static_assert(sizeof(GroupRec) == sizeof(wrs_group), "layout");
static_assert(kTile == WRS_TABLE2_GROUP, "group size");

struct Levels {
    uint32_t L;
    uint32_t pad;
    uint64_t size[kMaxLevels];  // members of each level (level 0: the n items)
    uint64_t off[kMaxLevels];   // first bucket of each level
    uint64_t goff[kMaxLevels];  // first group record of each level
};

struct Walk {              // the levels in the sampler's order: depth 0 = the top level
    uint32_t L;
    uint32_t pad;
    uint64_t size[kMaxLevels], off[kMaxLevels], goff[kMaxLevels];
};

struct GroupSmem {
    u128 okey[kTile];       // keys D of the group's lights, in order (swizzled; u64 keys use the front half)
    u128 hkey[kTile];       // keys E of the group's heavies
    uint16_t ooff[kTile];   // their offsets in the group
    uint16_t hoff[kTile];
    U2 scan[kWarps];        // pair scan (u128 pairs, or u64 pairs at the front)
    u128 red[kWarps];
    uint32_t cnt[kWarps];
};

__device__ __forceinline__ u128 block_sum128(u128 v, u128 *sm)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum128(v);
    if (lane == 0) sm[wid] = v;
    __syncthreads();
    u128 t = 0;
#pragma unroll
    for (int i = 0; i < kWarps; ++i) t += sm[i];
    return t;
}

// Keys of width K in shared memory: u128 (8 per 128-B bank row) or u64 (16
// per row); the column is XORed with the row's low bits so that threads
// reading rows at a fixed stride hit distinct banks.
template <typename K> __device__ __forceinline__ uint32_t swzk(uint32_t j);
template <> __device__ __forceinline__ uint32_t swzk<u128>(uint32_t j) { return j ^ ((j >> 3) & 7u); }
template <> __device__ __forceinline__ uint32_t swzk<uint64_t>(uint32_t j) { return j ^ ((j >> 4) & 15u); }

template <typename K> __device__ __forceinline__ K shfl_up_k(K v, int d);
template <> __device__ __forceinline__ u128 shfl_up_k<u128>(u128 v, int d) { return shfl_up128(v, d); }
template <> __device__ __forceinline__ uint64_t shfl_up_k<uint64_t>(uint64_t v, int d)
{
    return __shfl_up_sync(0xFFFFFFFFu, v, d);
}

template <typename K> struct PairK { K a, b; };

// Exclusive block scan of two values per thread; total = the block's sums.
template <typename K>
__device__ __forceinline__ PairK<K> block_exclusive_scan_pair(PairK<K> v, PairK<K> &total, PairK<K> *sm)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    PairK<K> inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const K a = shfl_up_k<K>(inc.a, d), b = shfl_up_k<K>(inc.b, d);
        if (lane >= d) { inc.a += a; inc.b += b; }
    }
    if (lane == 31) sm[wid] = inc;
    __syncthreads();
    PairK<K> base{0, 0};
    for (int i = 0; i < wid; ++i) { base.a += sm[i].a; base.b += sm[i].b; }
    total = PairK<K>{0, 0};
#pragma unroll
    for (int i = 0; i < kWarps; ++i) { total.a += sm[i].a; total.b += sm[i].b; }
    PairK<K> r;
    r.a = base.a + inc.a - v.a;
    r.b = base.b + inc.b - v.b;
    return r;
}

template <typename K> __device__ __forceinline__ uint64_t thr_of(K bw, uint32_t shift);
template <> __device__ __forceinline__ uint64_t thr_of<u128>(u128 bw, uint32_t shift) { return lo64(bw >> shift); }
template <> __device__ __forceinline__ uint64_t thr_of<uint64_t>(uint64_t bw, uint32_t) { return bw; }

// Alg. 2 on one group with keys of width K (u64 when n_g * Q_g < 2^63): the
// group's lights get exclusive prefix keys D of their deficits Q_g - n_g q,
// its heavies inclusive prefix keys E of their excesses n_g q - Q_g, and the
// two sequences are merged (heavy first when E <= D) over the threads.
template <typename K>
__device__ __forceinline__ bool group_build(GroupSmem &S, const u128 (&q)[kItems], u128 Qg128, uint32_t ng,
                                            uint64_t N, uint64_t first, uint64_t base, uint32_t shift,
                                            uint4 *__restrict__ buckets, DevHeader *hdr)
{
    K *okey = reinterpret_cast<K *>(S.okey);
    K *hkey = reinterpret_cast<K *>(S.hkey);
    PairK<K> *sm = reinterpret_cast<PairK<K> *>(S.scan);
    const K Qg = (K)Qg128;
    uint32_t lmask = 0, hmask = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        if (first + k < N) {
            if ((K)q[k] * (K)ng <= Qg) lmask |= 1u << k; else hmask |= 1u << k;
        }
    }
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan_u32((uint32_t)__popc(lmask) | ((uint32_t)__popc(hmask) << 16), tot,
                                                 S.cnt); // syncs: key arrays free
    const uint32_t nl = tot & 0xFFFFu, nh = tot >> 16;
    K sd = 0, se = 0;
    {
        uint32_t ls = ex & 0xFFFFu, hs = ex >> 16;
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const K nq = (K)q[k] * (K)ng;
            const uint16_t off = (uint16_t)(threadIdx.x * kItems + k);
            if ((lmask >> k) & 1u) {
                const K d = Qg - nq; // deficit
                okey[swzk<K>(ls)] = d;
                S.ooff[ls] = off;
                sd += d;
                ++ls;
            } else if ((hmask >> k) & 1u) {
                const K e = nq - Qg; // excess
                hkey[swzk<K>(hs)] = e;
                S.hoff[hs] = off;
                se += e;
                ++hs;
            }
        }
    }
    PairK<K> sums;
    const PairK<K> exs = block_exclusive_scan_pair<K>(PairK<K>{sd, se}, sums, sm);
    {   // deficits -> exclusive prefix D, excesses -> inclusive prefix E, in place
        const uint32_t l0 = ex & 0xFFFFu, h0 = ex >> 16;
        K kl = exs.a, ke = exs.b;
        for (uint32_t j = 0; j < (uint32_t)__popc(lmask); ++j) {
            const K d = okey[swzk<K>(l0 + j)];
            okey[swzk<K>(l0 + j)] = kl;
            kl += d;
        }
        for (uint32_t j = 0; j < (uint32_t)__popc(hmask); ++j) {
            ke += hkey[swzk<K>(h0 + j)];
            hkey[swzk<K>(h0 + j)] = ke;
        }
    }
    const K D_end = sums.a; // total deficit (= total excess)
    __syncthreads();

    bool bad = sums.a != sums.b;
    const uint32_t M = ng;
    const uint32_t per = (M + kThreads - 1) / kThreads;
    const uint32_t d0 = threadIdx.x * per;
    if (d0 < M) {
        uint32_t lo = d0 > nl ? d0 - nl : 0, hi = d0 < nh ? d0 : nh;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1; // is heavy mid-1 before light d0-mid?
            if (hkey[swzk<K>(mid - 1)] <= okey[swzk<K>(d0 - mid)]) lo = mid; else hi = mid - 1;
        }
        uint32_t j = lo, i = d0 - lo;
        const uint32_t steps = min(per, M - d0);
        K ej = j < nh ? hkey[swzk<K>(j)] : (K)0;
        K di = i < nl ? okey[swzk<K>(i)] : D_end;
        for (uint32_t st = 0; st < steps; ++st) {
            if ((j < nh) && (i >= nl || ej <= di)) { // heavy j: bucket Q_g - (D_i - E_j), alias the next heavy
                const K gap = di - ej;
                if (gap > Qg) bad = true;
                const uint32_t me = (uint32_t)(base + S.hoff[j]);
                const uint32_t nx = j + 1 < nh ? (uint32_t)(base + S.hoff[j + 1]) : kNone;
                if (nx == kNone && gap != 0) bad = true;
                const uint32_t alias = (nx == kNone || gap == 0) ? me : nx;
                const uint64_t thr = thr_of<K>(Qg - gap, shift);
                put_bucket(buckets, me, thr, alias, N, hdr);
                ++j;
                if (j < nh) ej = hkey[swzk<K>(j)];
            } else { // light i: its own weight, alias the current heavy (itself when full)
                const K dn = i + 1 < nl ? okey[swzk<K>(i + 1)] : D_end;
                const K nq = Qg - (dn - di);
                const uint32_t me = (uint32_t)(base + S.ooff[i]);
                uint32_t alias = me;
                if (nq != Qg) {
                    if (j < nh) alias = (uint32_t)(base + S.hoff[j]);
                    else bad = true;
                }
                const uint64_t thr = thr_of<K>(nq, shift);
                put_bucket(buckets, me, thr, alias, N, hdr);
                ++i;
                di = dn;
            }
        }
    }
    return bad;
}

// One group of a level per block.  SRC 0: u32 words, 1: binary32 words
// (both level 0), 2: exact 128-bit member weights (two words, levels >= 1).
template <int SRC>
__global__ void __launch_bounds__(kThreads, 3) k2_group(const void *__restrict__ src, uint64_t N, int vec,
                                                        DevHeader *hdr, uint4 *__restrict__ buckets,
                                                        GroupRec *__restrict__ groups, uint64_t *__restrict__ meta)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GroupSmem &S = *reinterpret_cast<GroupSmem *>(smem_raw);
    if (block_stopped(hdr)) return;
    const int beta = hdr->beta;
    const uint64_t base = (uint64_t)blockIdx.x * kTile;
    const uint32_t ng = (uint32_t)min((uint64_t)kTile, N - base);
    const uint64_t first = base + (uint64_t)threadIdx.x * kItems;

    u128 q[kItems];
    if (SRC == 2) {
        const uint4 *m = reinterpret_cast<const uint4 *>(src);
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            uint4 v = first + k < N ? __ldg(m + first + k) : make_uint4(0, 0, 0, 0);
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
    const u128 Qg = block_sum128(part, S.red); // the group's capacity
    const int bits = bitlen128(Qg);
    const uint32_t shift = bits > 64 ? (uint32_t)(bits - 64) : 0u;
    if (threadIdx.x == 0) {
        GroupRec r;
        r.qp = lo64(Qg >> shift);
        r.shift = shift;
        r.members = ng;
        groups[blockIdx.x] = r;
        if (meta) { meta[2 * blockIdx.x] = lo64(Qg); meta[2 * blockIdx.x + 1] = hi64(Qg); }
    }
    // n_g <= 2^11, so every scaled quantity and key is below n_g * Q_g < 2^63
    // when Q_g < 2^52: 64-bit arithmetic is exact (the common case)
    const bool bad = bits <= 52 ? group_build<uint64_t>(S, q, Qg, ng, N, first, base, shift, buckets, hdr)
                                : group_build<u128>(S, q, Qg, ng, N, first, base, shift, buckets, hdr);
    if (bad) set_status(hdr, kEInternal);
}

// k walks from the top group down (see the file comment); samples [s0, k).
constexpr int kSample2Unroll = 4;

__global__ void __launch_bounds__(256) k2_sample(const uint4 *__restrict__ buckets,
                                                 const GroupRec *__restrict__ groups, Walk lv,
                                                 const DevHeader *__restrict__ hdr, uint64_t s0, uint64_t k,
                                                 uint32_t key0, uint32_t key1, uint32_t sid0, uint32_t sid1,
                                                 uint32_t *__restrict__ out)
{
    if (hdr->status) return;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = s0 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < k; s += kSample2Unroll * stride) {
        uint32_t g[kSample2Unroll]; // indices below 2^32 (n < 2^32): 32-bit state, more blocks per SM
#pragma unroll
        for (int j = 0; j < kSample2Unroll; ++j) g[j] = 0;
#pragma unroll
        for (int d = 0; d < kMaxLevels; ++d) {
            if (d >= (int)lv.L) break;
            uint64_t v[kSample2Unroll], qp[kSample2Unroll];
            uint32_t r[kSample2Unroll], b0[kSample2Unroll];
            uint4 bk[kSample2Unroll];
#pragma unroll
            for (int j = 0; j < kSample2Unroll; ++j) {
                const uint64_t sj = s + j * stride;
                P4 c;
                c.x0 = (uint32_t)sj; c.x1 = (uint32_t)(sj >> 32); c.x2 = sid0; c.x3 = sid1;
                const P4 o = philox4x32_10(c, key0 + (uint32_t)d * 0x9E3779B9u, key1 + (uint32_t)d * 0xBB67AE85u);
                const uint64_t u = o.x0 | ((uint64_t)o.x1 << 32);
                v[j] = o.x2 | ((uint64_t)o.x3 << 32);
                b0[j] = g[j] * (uint32_t)kTile;
                const uint64_t ngj = min((uint64_t)kTile, lv.size[d] - b0[j]);
                r[j] = (uint32_t)__umul64hi(u, ngj);
            }
#pragma unroll
            for (int j = 0; j < kSample2Unroll; ++j) {
                if (s + j * stride < k) {
                    bk[j] = ld_bucket(buckets + lv.off[d] + (uint64_t)(b0[j] + r[j]));
                    qp[j] = __ldg(&groups[lv.goff[d] + g[j]].qp);
                }
            }
#pragma unroll
            for (int j = 0; j < kSample2Unroll; ++j) {
                if (s + j * stride < k) {
                    const uint64_t thr = bk[j].x | ((uint64_t)bk[j].y << 32);
                    g[j] = (__umul64hi(v[j], qp[j]) < thr) ? b0[j] + r[j] : bk[j].z;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kSample2Unroll; ++j) {
            const uint64_t sj = s + j * stride;
            if (sj < k) __stcs(out + sj, (uint32_t)g[j]);
        }
    }
}

} // namespace wrs

struct wrs_table2 {
    uint64_t cap;
    uint64_t n;            // items of the last build (0: never built)
    int device;
    uint32_t f32;
    Levels lv;             // of the last build
    uint8_t *ws;           // header, k_stats partials, group records, meta weights
    DevHeader *hdr;
    Partial *part;
    GroupRec *groups;
    uint64_t *meta;        // member weights of levels >= 1, two words each
    uint64_t meta_cap;     // entries
    uint4 *buckets;        // all levels, level 0 first
    int host_status;
    void *os_front;        // OS-ND frontiers (one entry per group of every level) and counters
    uint64_t os_cap;
};

namespace {

Levels levels_for(uint64_t n)
{
    Levels v;
    std::memset(&v, 0, sizeof(v));
    uint64_t m = n, o = 0, go = 0;
    for (;;) {
        v.size[v.L] = m;
        v.off[v.L] = o;
        v.goff[v.L] = go;
        o += m;
        go += (m + kTile - 1) / kTile;
        ++v.L;
        if (m <= (uint64_t)kTile || v.L == kMaxLevels) break;
        m = (m + kTile - 1) / kTile;
    }
    return v;
}

uint64_t levels_buckets(const Levels &v) { return v.off[v.L - 1] + v.size[v.L - 1]; }
uint64_t levels_groups(const Levels &v) { return v.goff[v.L - 1] + (v.size[v.L - 1] + kTile - 1) / kTile; }

bool g_two_attr_done[64];

wrs_status twolevel_attributes()
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return WRS_EDEVICE;
    if (g_two_attr_done[dev]) return WRS_OK;
    const int bytes = (int)sizeof(GroupSmem);
    cudaError_t e = cudaFuncSetAttribute(k2_group<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k2_group<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k2_group<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return WRS_EDEVICE;
    g_two_attr_done[dev] = true;
    return WRS_OK;
}

wrs_status launch_sample2(const wrs_table2 *t, uint64_t s0, uint64_t s1, uint64_t seed, uint64_t stream_id,
                          uint32_t *d_out, cudaStream_t s)
{
    const uint64_t k = s1 - s0;
    const uint64_t want = (k + 256ull * kSample2Unroll - 1) / (256ull * kSample2Unroll);
    const uint64_t cap = (uint64_t)sm_count() * 16;
    const uint32_t blocks = (uint32_t)(want < cap ? (want < 1 ? 1 : want) : cap);
    Walk wk;
    std::memset(&wk, 0, sizeof(wk));
    wk.L = t->lv.L;
    for (uint32_t d = 0; d < t->lv.L; ++d) {
        const uint32_t l = t->lv.L - 1 - d;
        wk.size[d] = t->lv.size[l];
        wk.off[d] = t->lv.off[l];
        wk.goff[d] = t->lv.goff[l];
    }
    k2_sample<<<blocks, 256, 0, s>>>(t->buckets, t->groups, wk, t->hdr, s0, s1, (uint32_t)seed,
                                     (uint32_t)(seed >> 32), (uint32_t)stream_id, (uint32_t)(stream_id >> 32), d_out);
    return launch_err();
}

} // namespace

extern "C" {

wrs_status wrs_table2_create(uint64_t capacity_n, wrs_table2 **out)
{
    if (!out) return WRS_EINVAL;
    *out = nullptr;
    if (capacity_n == 0 || capacity_n >= (1ull << 32)) return WRS_EINVAL;
    wrs_status st = twolevel_attributes();
    if (st != WRS_OK) return st;
    wrs_table2 *t = new (std::nothrow) wrs_table2();
    if (!t) return WRS_ENOMEM;
    std::memset(t, 0, sizeof(*t));
    t->cap = capacity_n;
    t->host_status = -1;
    cudaGetDevice(&t->device);
    const Levels v = levels_for(capacity_n);
    const uint64_t nb = levels_buckets(v), ngr = levels_groups(v);
    t->meta_cap = nb - capacity_n + 1;
    uint64_t o = 0;
    auto carve = [&](uint64_t bytes) { const uint64_t at = o; o = align_up(o + bytes, 256); return at; };
    const uint64_t o_hdr = carve(sizeof(DevHeader));
    const uint64_t o_part = carve(kMaxParts * sizeof(Partial));
    const uint64_t o_groups = carve(ngr * sizeof(GroupRec));
    const uint64_t o_meta = carve(t->meta_cap * 2 * sizeof(uint64_t));
    cudaError_t e = cudaMalloc(&t->ws, o);
    if (e != cudaSuccess) { delete t; return cuda_err(e); }
    e = cudaMalloc(&t->buckets, nb * sizeof(uint4));
    if (e != cudaSuccess) { cudaFree(t->ws); delete t; return cuda_err(e); }
    t->hdr = reinterpret_cast<DevHeader *>(t->ws + o_hdr);
    t->part = reinterpret_cast<Partial *>(t->ws + o_part);
    t->groups = reinterpret_cast<GroupRec *>(t->ws + o_groups);
    t->meta = reinterpret_cast<uint64_t *>(t->ws + o_meta);
    e = cudaMemset(t->ws, 0, o);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { wrs_table2_free(t); return cuda_err(e); }
    *out = t;
    return WRS_OK;
}

wrs_status wrs_table2_build(wrs_table2 *t, const void *d_weights, uint64_t n, wrs_dtype dtype, void *stream)
{
    if (!t || !d_weights || n == 0 || n > t->cap) return WRS_EINVAL;
    if (dtype != WRS_U32 && dtype != WRS_F32) return WRS_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_weights) % 4) != 0) return WRS_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint32_t *w = static_cast<const uint32_t *>(d_weights);
    const int vec = (reinterpret_cast<uintptr_t>(w) % 16) == 0;
    const uint32_t f32 = dtype == WRS_F32;
    // exact total, beta and validity: the weight-total pass of the single table
    uint64_t want = (n + (uint64_t)kThreads * 16 - 1) / ((uint64_t)kThreads * 16);
    uint32_t nparts = (uint32_t)(want < 1 ? 1 : (want > kMaxParts ? kMaxParts : want));
    const uint32_t blocks_cap = (uint32_t)sm_count() * 8;
    if (nparts > blocks_cap) nparts = blocks_cap;
    const Levels v = levels_for(n);
    {
        const wrs_status st = check_clear(t->buckets, levels_buckets(v), s);
        if (st != WRS_OK) return st;
    }
    if (f32) k_stats<1><<<nparts, kThreads, 0, s>>>(w, n, vec, t->part);
    else k_stats<0><<<nparts, kThreads, 0, s>>>(w, n, vec, t->part);
    k_stats_combine<<<1, kThreads, 0, s>>>(t->part, nparts, n, f32, t->hdr);
    const size_t smem = sizeof(GroupSmem);
    for (uint32_t l = 0; l < v.L; ++l) {
        const uint32_t ngroups = (uint32_t)((v.size[l] + kTile - 1) / kTile);
        uint64_t *meta_out = (l + 1 < v.L) ? t->meta + 2 * (v.off[l + 1] - n) : nullptr;
        uint4 *bk = t->buckets + v.off[l];
        GroupRec *gr = t->groups + v.goff[l];
        if (l == 0) {
            if (f32) k2_group<1><<<ngroups, kThreads, smem, s>>>(w, v.size[0], vec, t->hdr, bk, gr, meta_out);
            else k2_group<0><<<ngroups, kThreads, smem, s>>>(w, v.size[0], vec, t->hdr, bk, gr, meta_out);
        } else {
            const uint64_t *meta_in = t->meta + 2 * (v.off[l] - n);
            k2_group<2><<<ngroups, kThreads, smem, s>>>(meta_in, v.size[l], 1, t->hdr, bk, gr, meta_out);
        }
    }
    const wrs_status st = launch_err();
    if (st == WRS_OK) {
        t->n = n;
        t->lv = v;
        t->f32 = f32;
        t->host_status = -1;
    }
    return st;
}

wrs_status wrs_table2_sample(const wrs_table2 *t, uint64_t k, uint64_t seed, uint64_t stream_id, uint32_t *d_out,
                             void *stream)
{
    if (!t || t->n == 0) return WRS_EINVAL;
    if (k == 0) return WRS_OK;
    if (!d_out) return WRS_EINVAL;
    if (t->host_status > 0) return (wrs_status)t->host_status;
    return launch_sample2(t, 0, k, seed, stream_id, d_out, static_cast<cudaStream_t>(stream));
}

wrs_status wrs_table2_status(const wrs_table2 *t)
{
    if (!t || t->n == 0) return WRS_EINVAL;
    uint32_t st = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&st, &t->hdr->status, sizeof(st), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(e);
    const_cast<wrs_table2 *>(t)->host_status = (int)st;
    return (wrs_status)st;
}

wrs_status wrs_table2_layout(const wrs_table2 *t, uint32_t *h_levels, uint64_t *h_sizes)
{
    if (!t || t->n == 0 || !h_levels) return WRS_EINVAL;
    *h_levels = t->lv.L;
    if (h_sizes)
        for (uint32_t l = 0; l < t->lv.L; ++l) h_sizes[l] = t->lv.size[l];
    return WRS_OK;
}

wrs_status wrs_table2_download(const wrs_table2 *t, void *h_buckets, uint64_t bucket_bytes, void *h_groups,
                               uint64_t group_bytes)
{
    if (!t || t->n == 0) return WRS_EINVAL;
    const uint64_t nb = levels_buckets(t->lv), ngr = levels_groups(t->lv);
    if ((h_buckets && bucket_bytes < nb * sizeof(uint4)) || (h_groups && group_bytes < ngr * sizeof(GroupRec)))
        return WRS_EINVAL;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && h_buckets) e = cudaMemcpy(h_buckets, t->buckets, nb * sizeof(uint4), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h_groups) e = cudaMemcpy(h_groups, t->groups, ngr * sizeof(GroupRec), cudaMemcpyDeviceToHost);
    return cuda_err(e);
}

void wrs_table2_free(wrs_table2 *t)
{
    if (!t) return;
    cudaDeviceSynchronize();
    if (t->buckets) cudaFree(t->buckets);
    if (t->ws) cudaFree(t->ws);
    if (t->os_front) cudaFree(t->os_front);
    delete t;
}

} // extern "C"
