// wrs_batch.cuh -- many independent tables built and sampled together
// (the wrs_batch_* entry points of include/wrs.h).  Included by wrs.cu only,
// after the single-table runtime.
//
// Every stage of the build is one launch over all tables: a block looks up
// (table, block within the table) in a per-stage map and runs the same body
// as the single-table kernel on that table's slice of the concatenated
// arrays.  Tables of at most one tile (2048 weights) skip those stages: one
// block builds each of them whole in shared memory (kb_small: total, exact
// units, light threshold and Alg. 2 in the table's own units, which for a
// single group are the units of the whole table).  Tables never read each other's data, so table t's buckets and
// samples are exactly those of a single-table build of its weights (and of
// wrs_sample with stream id stream_id + t).  Nothing on the launch path reads
// a host value that changes between builds -- the look-back generation lives
// in device memory -- so a build and a sample can be captured once in a CUDA
// graph and replayed.
#pragma once

#include <algorithm>
#include <vector>

namespace wrs {

struct BatchTable {       // per table (device copy in wrs_batch::d_tables)
    uint64_t off;         // first weight and first bucket of the table
    uint64_t n;
    uint32_t ntiles, tile0;   // tiles, first tile in the per-tile arrays
    uint32_t part0, nparts;   // k_stats partials
    uint32_t chunk0, group;   // first look-back chunk; own tiles per sweep block
    uint64_t k, k_off;        // samples of the current plan, first output
    uint32_t sblocks, pad;    // blocks of the sampler
};

struct BlockMap {         // one per block of a batch launch
    uint32_t table, local;
};

constexpr int kBatchClasses = WRS_BATCH_CLASSES; // sweep size classes by tiles: 1, 2-4, 5-32, 33-256, more
constexpr uint32_t kBatchGroups[] = {1, 2, 4, 8}; // tuner's candidates for own tiles per sweep block
constexpr uint32_t kBatchPartWeights = 16384;    // weights per k_stats block (at least)

inline int batch_class(uint32_t ntiles)
{
    return ntiles <= 1 ? 0 : ntiles <= 4 ? 1 : ntiles <= 32 ? 2 : ntiles <= 256 ? 3 : 4;
}

template <int F32>
__global__ void __launch_bounds__(kThreads) kb_stats(const uint32_t *__restrict__ w, int vec,
                                                     const BatchTable *__restrict__ bt,
                                                     const BlockMap *__restrict__ map, Partial *__restrict__ part)
{
    const BlockMap m = map[blockIdx.x];
    const BatchTable &T = bt[m.table];
    stats_body<F32>(w + T.off, T.n, vec, m.local, T.nparts, part + T.part0 + m.local);
}

// One block per table; block 0 also advances the look-back generation.
// Tables of one tile are built by kb_small instead.
__global__ void __launch_bounds__(kThreads) kb_stats_combine(const BatchTable *__restrict__ bt,
                                                             const Partial *__restrict__ part, uint32_t f32,
                                                             DevHeader *hdr, uint32_t *epoch)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        uint32_t e = *epoch + 1;
        if (e >= (1u << 30)) e = 1;
        *epoch = e;
    }
    const BatchTable &T = bt[blockIdx.x];
    if (T.ntiles <= 1) return;
    stats_combine_body(part + T.part0, T.nparts, T.n, f32, hdr + blockIdx.x);
}

// A table of at most one tile, whole, in one block: validity, exact total
// and lowest set bit (as k_stats + k_stats_combine), the header, then Alg. 2
// on its n items with capacity Q and item weights n * q (group_build: the
// table is a single group), and the light count.  The buckets and header
// equal those of the tile pipeline.
template <int F32>
__global__ void __launch_bounds__(kThreads, 3) kb_small(const uint32_t *__restrict__ w, int vec,
                                                        const BatchTable *__restrict__ bt,
                                                        const BlockMap *__restrict__ map, DevHeader *hdr_all,
                                                        uint4 *__restrict__ buckets)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GroupSmem &S = *reinterpret_cast<GroupSmem *>(smem_raw);
    __shared__ uint32_t s_status;
    const BlockMap m = map[blockIdx.x];
    const BatchTable &T = bt[m.table];
    DevHeader *hdr = hdr_all + m.table;
    const uint64_t N = T.n;
    const uint32_t *wt = w + T.off;
    const uint64_t first = (uint64_t)threadIdx.x * kItems;
    uint32_t x[kItems];
    load_items(wt, N, vec, first, x);
    Acc a;
    a.base = F32 ? INT_MAX : 0;
    a.acc = 0;
    a.flags = 0;
    uint64_t a64 = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        if (first + k < N) {
            acc_take<F32>(a, a64, x[k]);
            if (F32) acc_fold(a, a64);
        }
    }
    acc_fold(a, a64);
    a = acc_block_reduce(a);
    if (threadIdx.x == 0) s_status = write_header(a, N, F32, hdr);
    __syncthreads();
    if (s_status) return;
    const u128 Q = mk128(hdr->q_lo, hdr->q_hi);
    const int beta = hdr->beta;
    const uint32_t shift = hdr->shift;
    u128 q[kItems];
    uint32_t cl = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        q[k] = first + k < N ? q_of(x[k], F32, beta) : (u128)0;
        if (first + k < N && q[k] * (u128)N <= Q) ++cl;
    }
    uint32_t nl;
    block_exclusive_scan_u32(cl, nl, S.cnt);
    if (threadIdx.x == 0) hdr->n_light = nl;
    const bool bad = bitlen128(Q) <= 52
                         ? group_build<uint64_t>(S, q, Q, (uint32_t)N, N, first, 0, shift, buckets + T.off, hdr)
                         : group_build<u128>(S, q, Q, (uint32_t)N, N, first, 0, shift, buckets + T.off, hdr);
    if (bad) set_status(hdr, kEInternal);
}

template <int F32>
__global__ void __launch_bounds__(kThreads) kb_classify(const uint32_t *__restrict__ w, int vec,
                                                        const BatchTable *__restrict__ bt,
                                                        const BlockMap *__restrict__ map, const DevHeader *hdr,
                                                        TileSum *__restrict__ agg, uint16_t *__restrict__ slist)
{
    const BlockMap m = map[blockIdx.x]; // block m.local: tiles 8 m.local .. 8 m.local + 7, one per warp
    const BatchTable &T = bt[m.table];
    classify_body<F32>(w + T.off, T.n, vec, hdr + m.table, agg + T.tile0, slist + (uint64_t)T.tile0 * kSparse,
                       T.ntiles, m.local * kWarps + (threadIdx.x >> 5), T.ntiles);
}

__global__ void __launch_bounds__(kThreads) kb_tilescan(const BatchTable *__restrict__ bt,
                                                        const BlockMap *__restrict__ map, DevHeader *hdr,
                                                        const TileSum *__restrict__ agg, TileSum *chunk_agg,
                                                        TileSum *chunk_incl, TileSum *__restrict__ incl,
                                                        uint32_t *flags, const uint32_t *epoch, uint32_t wait_limit)
{
    const BlockMap m = map[blockIdx.x];
    const BatchTable &T = bt[m.table];
    tilescan_body(hdr + m.table, agg + T.tile0, chunk_agg + T.chunk0, chunk_incl + T.chunk0, incl + T.tile0,
                  flags + T.chunk0, T.ntiles, __ldcg(epoch), wait_limit, kNone);
}

__global__ void __launch_bounds__(kThreads) kb_split(const BatchTable *__restrict__ bt,
                                                     const BlockMap *__restrict__ map,
                                                     const TileSum *__restrict__ incl, DevHeader *hdr,
                                                     Split *__restrict__ split)
{
    const BlockMap m = map[blockIdx.x];
    const BatchTable &T = bt[m.table];
    split_body(incl + T.tile0, T.ntiles, T.n, hdr + m.table, split + T.tile0, m.local * kThreads + threadIdx.x);
}

template <int F32>
__global__ void __launch_bounds__(kThreads, 3) kb_sweep(const uint32_t *__restrict__ w, int vec,
                                                        const BatchTable *__restrict__ bt,
                                                        const BlockMap *__restrict__ map, DevHeader *hdr,
                                                        const TileSum *__restrict__ incl,
                                                        const Split *__restrict__ split,
                                                        const uint16_t *__restrict__ slist, uint4 *__restrict__ buckets)
{
    const BlockMap m = map[blockIdx.x];
    const BatchTable &T = bt[m.table];
    const uint32_t c_first = m.local * T.group;
    sweep_body<F32>(w + T.off, T.n, vec, hdr + m.table, incl + T.tile0, split + T.tile0,
                    slist + (uint64_t)T.tile0 * kSparse, T.ntiles, buckets + T.off, c_first,
                    min(c_first + T.group, T.ntiles));
}

__global__ void __launch_bounds__(256) kb_sample(const BatchTable *__restrict__ bt, const BlockMap *__restrict__ map,
                                                 const uint4 *__restrict__ buckets,
                                                 const DevHeader *__restrict__ hdr, uint32_t key0, uint32_t key1,
                                                 uint64_t sid, uint32_t *__restrict__ out)
{
    const BlockMap m = map[blockIdx.x];
    const BatchTable &T = bt[m.table];
    if (hdr[m.table].status) return;
    const uint64_t st = sid + m.table;
    sample_body(buckets + T.off, T.n, hdr[m.table].qp, T.k, key0, key1, (uint32_t)st, (uint32_t)(st >> 32),
                out + T.k_off, (uint64_t)m.local * 256 + threadIdx.x, (uint64_t)T.sblocks * 256);
}

// Many sample requests against many resident tables in one launch.  Task i
// draws k_i samples into out[out_offset_i ...]; the tasks' outputs are
// consecutive (out_offset ascending, each the previous one plus its k).
// Block b covers outputs [b * kManyPerBlock, ...): thread 0 finds the task
// holding the first one by binary search, then the block walks the tasks
// that overlap its range.  Sample s of a task is sample s of wrs_sample on
// its table with the task's seed and stream id.
constexpr uint32_t kManyPerBlock = 256 * 16;

struct SampleTask {       // mirrors wrs_sample_task
    const uint4 *buckets;
    const DevHeader *hdr;
    uint64_t n, k, seed, stream_id, out_offset, reserved;
};

static_assert(sizeof(SampleTask) == sizeof(wrs_sample_task), "layout");
static_assert(offsetof(SampleTask, hdr) == offsetof(wrs_sample_task, header), "layout");
static_assert(offsetof(SampleTask, k) == offsetof(wrs_sample_task, k), "layout");
static_assert(offsetof(SampleTask, out_offset) == offsetof(wrs_sample_task, out_offset), "layout");

__global__ void __launch_bounds__(256) k_sample_many(const SampleTask *__restrict__ tasks, uint32_t ntasks,
                                                     uint64_t total_k, uint32_t *__restrict__ out)
{
    __shared__ uint32_t s_first;
    const uint64_t begin = (uint64_t)blockIdx.x * kManyPerBlock;
    const uint64_t end = min(begin + kManyPerBlock, total_k);
    if (threadIdx.x == 0) { // last task with out_offset <= begin
        uint32_t lo = 0, hi = ntasks - 1;
        while (lo < hi) {
            const uint32_t mid = lo + (hi - lo + 1) / 2;
            if (tasks[mid].out_offset <= begin) lo = mid; else hi = mid - 1;
        }
        s_first = lo;
    }
    __syncthreads();
    for (uint32_t i = s_first; i < ntasks; ++i) {
        const SampleTask T = tasks[i];
        if (T.out_offset >= end) break;
        const uint64_t lo = max(begin, T.out_offset), hi = min(end, T.out_offset + T.k);
        if (lo >= hi || T.hdr->status) continue;
        // local sample indices [lo - off, hi - off), written at out + off + s
        sample_body(T.buckets, T.n, T.hdr->qp, hi - T.out_offset, (uint32_t)T.seed, (uint32_t)(T.seed >> 32),
                    (uint32_t)T.stream_id, (uint32_t)(T.stream_id >> 32), out + T.out_offset,
                    lo - T.out_offset + threadIdx.x, 256);
    }
}

} // namespace wrs

struct wrs_batch {
    int device;
    uint32_t ntables;
    uint64_t total_w;      // weights and buckets, including the alignment gaps
    uint32_t total_tiles, total_parts, total_chunks;
    uint64_t total_k;
    std::vector<BatchTable> h;
    uint32_t groups[kBatchClasses];
    uint8_t *ws;           // one allocation: tables, headers, per-part/tile/chunk arrays, epoch
    BatchTable *d_tables;
    DevHeader *hdr;
    Partial *part;
    TileSum *agg, *incl, *cagg, *cincl;
    uint32_t *flags, *epoch;
    Split *split;
    uint16_t *slist;
    uint4 *buckets;
    BlockMap *map[7];      // stats, small tables, classify, tilescan, split, sweep, sample
    uint32_t nb[7];        // blocks of each launch
    uint32_t map_cap[7];
    int built;             // a build was enqueued
};

namespace {

enum { kMapStats = 0, kMapSmall = 1, kMapClassify = 2, kMapScan = 3, kMapSplit = 4, kMapSweep = 5, kMapSample = 6 };

// Offsets of the tables' weights: 4-weight (16-byte) aligned, in order.
void batch_offsets(uint32_t ntables, const uint64_t *n, uint64_t *off)
{
    uint64_t o = 0;
    for (uint32_t t = 0; t < ntables; ++t) {
        off[t] = o;
        o += (n[t] + 3) / 4 * 4;
    }
    off[ntables] = o;
}

wrs_status upload_map(wrs_batch *b, int which, const std::vector<BlockMap> &m)
{
    if (m.size() > b->map_cap[which]) {
        if (b->map[which]) { cudaFree(b->map[which]); b->map[which] = nullptr; b->map_cap[which] = 0; }
        cudaError_t e = cudaMalloc(&b->map[which], m.size() * sizeof(BlockMap));
        if (e != cudaSuccess) return cuda_err(e);
        b->map_cap[which] = (uint32_t)m.size();
    }
    b->nb[which] = (uint32_t)m.size();
    if (m.empty()) return WRS_OK;
    return cuda_err(cudaMemcpy(b->map[which], m.data(), m.size() * sizeof(BlockMap), cudaMemcpyHostToDevice));
}

wrs_status upload_tables(wrs_batch *b)
{
    return cuda_err(cudaMemcpy(b->d_tables, b->h.data(), b->h.size() * sizeof(BatchTable), cudaMemcpyHostToDevice));
}

// Sweep group of every table from its class, and the sweep's block map.
wrs_status apply_groups(wrs_batch *b)
{
    std::vector<BlockMap> m;
    for (uint32_t t = 0; t < b->ntables; ++t) {
        BatchTable &T = b->h[t];
        T.group = b->groups[batch_class(T.ntiles)];
        if (T.ntiles <= 1) continue; // built whole by kb_small
        const uint32_t nblk = (T.ntiles + T.group - 1) / T.group;
        for (uint32_t i = 0; i < nblk; ++i) m.push_back(BlockMap{t, i});
    }
    wrs_status st = upload_map(b, kMapSweep, m);
    if (st == WRS_OK) st = upload_tables(b);
    return st;
}

wrs_status batch_enqueue_build(wrs_batch *b, const uint32_t *w, uint32_t f32, cudaStream_t s, cudaEvent_t sweep0,
                               cudaEvent_t sweep1)
{
    const int vec = (reinterpret_cast<uintptr_t>(w) % 16) == 0;
    {
        const wrs_status st = check_clear(b->buckets, b->total_w, s);
        if (st != WRS_OK) return st;
    }
    if (b->nb[kMapSmall]) {
        const size_t gs = sizeof(GroupSmem);
        if (f32) kb_small<1><<<b->nb[kMapSmall], kThreads, gs, s>>>(w, vec, b->d_tables, b->map[kMapSmall], b->hdr, b->buckets);
        else kb_small<0><<<b->nb[kMapSmall], kThreads, gs, s>>>(w, vec, b->d_tables, b->map[kMapSmall], b->hdr, b->buckets);
    }
    if (b->nb[kMapStats] == 0) { // every table is small: the pipeline has no work
        if (sweep0) cudaEventRecord(sweep0, s);
        if (sweep1) cudaEventRecord(sweep1, s);
        return launch_err();
    }
    if (f32) kb_stats<1><<<b->nb[kMapStats], kThreads, 0, s>>>(w, vec, b->d_tables, b->map[kMapStats], b->part);
    else kb_stats<0><<<b->nb[kMapStats], kThreads, 0, s>>>(w, vec, b->d_tables, b->map[kMapStats], b->part);
    kb_stats_combine<<<b->ntables, kThreads, 0, s>>>(b->d_tables, b->part, f32, b->hdr, b->epoch);
    if (f32) kb_classify<1><<<b->nb[kMapClassify], kThreads, 0, s>>>(w, vec, b->d_tables, b->map[kMapClassify], b->hdr, b->agg, b->slist);
    else kb_classify<0><<<b->nb[kMapClassify], kThreads, 0, s>>>(w, vec, b->d_tables, b->map[kMapClassify], b->hdr, b->agg, b->slist);
    kb_tilescan<<<b->nb[kMapScan], kThreads, 0, s>>>(b->d_tables, b->map[kMapScan], b->hdr, b->agg, b->cagg,
                                                      b->cincl, b->incl, b->flags, b->epoch, g_wait_limit.load());
    kb_split<<<b->nb[kMapSplit], kThreads, 0, s>>>(b->d_tables, b->map[kMapSplit], b->incl, b->hdr, b->split);
    if (sweep0) cudaEventRecord(sweep0, s);
    const size_t smem = sizeof(SweepSmem);
    if (f32) kb_sweep<1><<<b->nb[kMapSweep], kThreads, smem, s>>>(w, vec, b->d_tables, b->map[kMapSweep], b->hdr, b->incl, b->split, b->slist, b->buckets);
    else kb_sweep<0><<<b->nb[kMapSweep], kThreads, smem, s>>>(w, vec, b->d_tables, b->map[kMapSweep], b->hdr, b->incl, b->split, b->slist, b->buckets);
    if (sweep1) cudaEventRecord(sweep1, s);
    return launch_err();
}

wrs_status batch_enqueue_sweep(wrs_batch *b, const uint32_t *w, uint32_t f32, cudaStream_t s)
{
    if (b->nb[kMapSweep] == 0) return WRS_OK;
    const int vec = (reinterpret_cast<uintptr_t>(w) % 16) == 0;
    const size_t smem = sizeof(SweepSmem);
    if (f32) kb_sweep<1><<<b->nb[kMapSweep], kThreads, smem, s>>>(w, vec, b->d_tables, b->map[kMapSweep], b->hdr, b->incl, b->split, b->slist, b->buckets);
    else kb_sweep<0><<<b->nb[kMapSweep], kThreads, smem, s>>>(w, vec, b->d_tables, b->map[kMapSweep], b->hdr, b->incl, b->split, b->slist, b->buckets);
    return launch_err();
}

bool g_batch_attr_done[64];

wrs_status batch_kernel_attributes()
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return WRS_EDEVICE;
    if (g_batch_attr_done[dev]) return WRS_OK;
    const int bytes = (int)sizeof(SweepSmem), gbytes = (int)sizeof(GroupSmem);
    cudaError_t e = cudaFuncSetAttribute(kb_sweep<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kb_sweep<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kb_small<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, gbytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kb_small<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, gbytes);
    if (e != cudaSuccess) return WRS_EDEVICE;
    g_batch_attr_done[dev] = true;
    return WRS_OK;
}

wrs_status batch_check_args(const wrs_batch *b, const void *d_weights, wrs_dtype dtype)
{
    if (!b || !d_weights) return WRS_EINVAL;
    if (dtype != WRS_U32 && dtype != WRS_F32) return WRS_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_weights) % 4) != 0) return WRS_EINVAL;
    return WRS_OK;
}

} // namespace

extern "C" {

wrs_status wrs_batch_offsets(uint32_t ntables, const uint64_t *h_n, uint64_t *h_offsets)
{
    if (ntables == 0 || !h_n || !h_offsets) return WRS_EINVAL;
    for (uint32_t t = 0; t < ntables; ++t)
        if (h_n[t] == 0 || h_n[t] >= (1ull << 32)) return WRS_EINVAL;
    batch_offsets(ntables, h_n, h_offsets);
    return WRS_OK;
}

wrs_status wrs_batch_create(uint32_t ntables, const uint64_t *h_n, wrs_batch **out)
{
    if (!out) return WRS_EINVAL;
    *out = nullptr;
    if (ntables == 0 || ntables >= (1u << 31)) return WRS_EINVAL;
    std::vector<uint64_t> off(ntables + 1u);
    wrs_status st = wrs_batch_offsets(ntables, h_n, off.data());
    if (st != WRS_OK) return st;
    st = batch_kernel_attributes();
    if (st != WRS_OK) return st;
    wrs_batch *b = new (std::nothrow) wrs_batch();
    if (!b) return WRS_ENOMEM;
    b->ntables = ntables;
    b->h.resize(ntables);
    cudaGetDevice(&b->device);
    uint64_t tiles = 0, parts = 0, chunks = 0;
    for (uint32_t t = 0; t < ntables; ++t) {
        BatchTable &T = b->h[t];
        std::memset(&T, 0, sizeof(T));
        T.off = off[t];
        T.n = h_n[t];
        T.ntiles = (uint32_t)((T.n + kTile - 1) / kTile);
        T.tile0 = (uint32_t)tiles;
        uint64_t np = (T.n + kBatchPartWeights - 1) / kBatchPartWeights;
        T.nparts = (uint32_t)std::min<uint64_t>(np, (uint64_t)sm_count() * 8);
        T.part0 = (uint32_t)parts;
        T.chunk0 = (uint32_t)chunks;
        tiles += T.ntiles;
        parts += T.nparts;
        chunks += (T.ntiles + kScanChunk - 1) / kScanChunk;
    }
    if (tiles >= (1ull << 32) || parts >= (1ull << 32)) { delete b; return WRS_EINVAL; }
    b->total_w = off[ntables];
    b->total_tiles = (uint32_t)tiles;
    b->total_parts = (uint32_t)parts;
    b->total_chunks = (uint32_t)chunks;
    for (int c = 0; c < kBatchClasses; ++c) b->groups[c] = c == 0 ? 1 : kSweepTiles;

    uint64_t o = 0;
    auto carve = [&](uint64_t bytes) { const uint64_t at = o; o = align_up(o + bytes, 256); return at; };
    const uint64_t o_tab = carve(ntables * sizeof(BatchTable));
    const uint64_t o_hdr = carve(ntables * sizeof(DevHeader));
    const uint64_t o_part = carve(parts * sizeof(Partial));
    const uint64_t o_agg = carve(tiles * sizeof(TileSum));
    const uint64_t o_incl = carve(tiles * sizeof(TileSum));
    const uint64_t o_cagg = carve(chunks * sizeof(TileSum));
    const uint64_t o_cincl = carve(chunks * sizeof(TileSum));
    const uint64_t o_flags = carve(chunks * sizeof(uint32_t));
    const uint64_t o_split = carve(tiles * sizeof(Split));
    const uint64_t o_slist = carve(tiles * kSparse * sizeof(uint16_t));
    const uint64_t o_epoch = carve(sizeof(uint32_t));
    cudaError_t e = cudaMalloc(&b->ws, o);
    if (e != cudaSuccess) { delete b; return cuda_err(e); }
    e = cudaMalloc(&b->buckets, b->total_w * sizeof(uint4));
    if (e != cudaSuccess) { cudaFree(b->ws); delete b; return cuda_err(e); }
    b->d_tables = reinterpret_cast<BatchTable *>(b->ws + o_tab);
    b->hdr = reinterpret_cast<DevHeader *>(b->ws + o_hdr);
    b->part = reinterpret_cast<Partial *>(b->ws + o_part);
    b->agg = reinterpret_cast<TileSum *>(b->ws + o_agg);
    b->incl = reinterpret_cast<TileSum *>(b->ws + o_incl);
    b->cagg = reinterpret_cast<TileSum *>(b->ws + o_cagg);
    b->cincl = reinterpret_cast<TileSum *>(b->ws + o_cincl);
    b->flags = reinterpret_cast<uint32_t *>(b->ws + o_flags);
    b->split = reinterpret_cast<Split *>(b->ws + o_split);
    b->slist = reinterpret_cast<uint16_t *>(b->ws + o_slist);
    b->epoch = reinterpret_cast<uint32_t *>(b->ws + o_epoch);
    e = cudaMemset(b->ws, 0, o);
    if (e != cudaSuccess) { wrs_batch_free(b); return cuda_err(e); }

    std::vector<BlockMap> ms, msmall, mc, mscan, msplit;
    for (uint32_t t = 0; t < ntables; ++t) {
        const BatchTable &T = b->h[t];
        if (T.ntiles <= 1) { msmall.push_back(BlockMap{t, 0}); continue; } // one block builds it whole
        for (uint32_t i = 0; i < T.nparts; ++i) ms.push_back(BlockMap{t, i});
        for (uint32_t i = 0; i < (T.ntiles + kWarps - 1) / kWarps; ++i) mc.push_back(BlockMap{t, i});
        for (uint32_t i = 0; i < (T.ntiles + kScanChunk - 1) / kScanChunk; ++i) mscan.push_back(BlockMap{t, i});
        for (uint32_t i = 0; i < (T.ntiles + kThreads - 1) / kThreads; ++i) msplit.push_back(BlockMap{t, i});
    }
    st = upload_map(b, kMapStats, ms);
    if (st == WRS_OK) st = upload_map(b, kMapSmall, msmall);
    if (st == WRS_OK) st = upload_map(b, kMapClassify, mc);
    if (st == WRS_OK) st = upload_map(b, kMapScan, mscan);
    if (st == WRS_OK) st = upload_map(b, kMapSplit, msplit);
    if (st == WRS_OK) st = upload_map(b, kMapSample, {});
    if (st == WRS_OK) st = apply_groups(b); // also uploads the table descriptors
    if (st == WRS_OK) st = cuda_err(cudaDeviceSynchronize());
    if (st != WRS_OK) { wrs_batch_free(b); return st; }
    *out = b;
    return WRS_OK;
}

wrs_status wrs_batch_layout(const wrs_batch *b, uint64_t *h_offsets)
{
    if (!b || !h_offsets) return WRS_EINVAL;
    for (uint32_t t = 0; t < b->ntables; ++t) h_offsets[t] = b->h[t].off;
    h_offsets[b->ntables] = b->total_w;
    return WRS_OK;
}

const wrs_bucket *wrs_batch_buckets(const wrs_batch *b)
{
    return b ? reinterpret_cast<const wrs_bucket *>(b->buckets) : nullptr;
}

wrs_status wrs_batch_build(wrs_batch *b, const void *d_weights, wrs_dtype dtype, void *stream)
{
    const wrs_status st = batch_check_args(b, d_weights, dtype);
    if (st != WRS_OK) return st;
    const wrs_status r = batch_enqueue_build(b, static_cast<const uint32_t *>(d_weights), dtype == WRS_F32,
                                             static_cast<cudaStream_t>(stream), nullptr, nullptr);
    if (r == WRS_OK) b->built = 1;
    return r;
}

wrs_status wrs_batch_set_samples(wrs_batch *b, const uint64_t *h_k, uint64_t *h_k_offsets)
{
    if (!b || !h_k) return WRS_EINVAL;
    std::vector<BlockMap> m;
    uint64_t ko = 0;
    const uint64_t cap = (uint64_t)sm_count() * 8;
    for (uint32_t t = 0; t < b->ntables; ++t) {
        BatchTable &T = b->h[t];
        T.k = h_k[t];
        T.k_off = ko;
        if (h_k_offsets) h_k_offsets[t] = ko;
        ko += T.k;
        const uint64_t want = (T.k + 256ull * kSampleUnroll - 1) / (256ull * kSampleUnroll);
        T.sblocks = (uint32_t)std::min(want, cap);
        for (uint32_t i = 0; i < T.sblocks; ++i) m.push_back(BlockMap{t, i});
    }
    if (h_k_offsets) h_k_offsets[b->ntables] = ko;
    if (m.size() >= (1ull << 31)) return WRS_EINVAL;
    b->total_k = ko;
    wrs_status st = upload_map(b, kMapSample, m);
    if (st == WRS_OK) st = upload_tables(b);
    return st;
}

wrs_status wrs_batch_sample(const wrs_batch *b, uint64_t seed, uint64_t stream_id, uint32_t *d_out, void *stream)
{
    if (!b || !b->built) return WRS_EINVAL;
    if (b->total_k == 0) return WRS_OK;
    if (!d_out) return WRS_EINVAL;
    kb_sample<<<b->nb[kMapSample], 256, 0, static_cast<cudaStream_t>(stream)>>>(
        b->d_tables, b->map[kMapSample], b->buckets, b->hdr, (uint32_t)seed, (uint32_t)(seed >> 32), stream_id,
        d_out);
    return launch_err();
}

wrs_status wrs_batch_status(const wrs_batch *b, int32_t *h_status)
{
    if (!b || !b->built) return WRS_EINVAL;
    std::vector<DevHeader> h(b->ntables);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), b->hdr, h.size() * sizeof(DevHeader), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(e);
    wrs_status first = WRS_OK;
    for (uint32_t t = 0; t < b->ntables; ++t) {
        if (h_status) h_status[t] = (int32_t)h[t].status;
        if (first == WRS_OK && h[t].status) first = (wrs_status)h[t].status;
    }
    return first;
}

wrs_status wrs_batch_table_info(const wrs_batch *b, uint32_t table, wrs_table_info *info)
{
    if (!b || !b->built || !info || table >= b->ntables) return WRS_EINVAL;
    DevHeader h;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&h, b->hdr + table, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(e);
    info->n = b->h[table].n;
    info->q_lo = h.q_lo;
    info->q_hi = h.q_hi;
    info->beta = h.beta;
    info->shift = h.shift;
    info->qp = h.qp;
    info->n_light = h.n_light;
    info->light_max = h.light_max;
    info->status = (int32_t)h.status;
    return WRS_OK;
}

wrs_status wrs_batch_download(const wrs_batch *b, void *h_buckets, uint64_t bytes)
{
    if (!b || !h_buckets || bytes < b->total_w * sizeof(uint4)) return WRS_EINVAL;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(h_buckets, b->buckets, b->total_w * sizeof(uint4), cudaMemcpyDeviceToHost);
    return cuda_err(e);
}

wrs_status wrs_batch_groups(const wrs_batch *b, uint32_t *h_groups)
{
    if (!b || !h_groups) return WRS_EINVAL;
    for (int c = 0; c < kBatchClasses; ++c) h_groups[c] = b->groups[c];
    return WRS_OK;
}

wrs_status wrs_batch_set_groups(wrs_batch *b, const uint32_t *h_groups)
{
    if (!b || !h_groups) return WRS_EINVAL;
    for (int c = 0; c < kBatchClasses; ++c)
        if (h_groups[c] == 0 || h_groups[c] > 64) return WRS_EINVAL;
    for (int c = 0; c < kBatchClasses; ++c) b->groups[c] = h_groups[c];
    return apply_groups(b);
}

wrs_status wrs_batch_tune(wrs_batch *b, const void *d_weights, wrs_dtype dtype, void *stream, float *h_sweep_ms)
{
    wrs_status st = batch_check_args(b, d_weights, dtype);
    if (st != WRS_OK) return st;
    const uint32_t *w = static_cast<const uint32_t *>(d_weights);
    const uint32_t f32 = dtype == WRS_F32;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    bool present[kBatchClasses] = {};
    for (const BatchTable &T : b->h)
        if (T.ntiles > 1) present[batch_class(T.ntiles)] = true; // one-tile tables: kb_small, no sweep
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return WRS_EDEVICE;
    }
    // stages before the sweep once; the sweep only reads their results
    st = batch_enqueue_build(b, w, f32, s, nullptr, nullptr);
    b->built = st == WRS_OK;
    auto time_sweep = [&](float &best) -> wrs_status {
        best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, s);
            wrs_status r = batch_enqueue_sweep(b, w, f32, s);
            cudaEventRecord(e1, s);
            if (r != WRS_OK) return r;
            if (cudaEventSynchronize(e1) != cudaSuccess) return WRS_EDEVICE;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            best = std::min(best, ms);
        }
        return WRS_OK;
    };
    for (int c = 0; c < kBatchClasses && st == WRS_OK; ++c) {
        if (!present[c]) continue;
        uint32_t best_g = b->groups[c];
        float best_ms = 1e30f;
        for (uint32_t g : kBatchGroups) {
            b->groups[c] = g;
            st = apply_groups(b);
            float ms = 0.f;
            if (st == WRS_OK) st = time_sweep(ms);
            if (st != WRS_OK) break;
            if (ms < best_ms) { best_ms = ms; best_g = g; }
        }
        b->groups[c] = best_g;
    }
    if (st == WRS_OK) st = apply_groups(b);
    if (st == WRS_OK) st = batch_enqueue_build(b, w, f32, s, nullptr, nullptr); // buckets of the final choice
    if (st == WRS_OK && h_sweep_ms) st = time_sweep(*h_sweep_ms);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

const void *wrs_batch_device_header(const wrs_batch *b, uint32_t table)
{
    return (b && table < b->ntables) ? static_cast<const void *>(b->hdr + table) : nullptr;
}

const void *wrs_table_device_header(const wrs_table *t)
{
    return t ? static_cast<const void *>(t->hdr) : nullptr;
}

wrs_status wrs_sample_many(const wrs_sample_task *d_tasks, uint32_t ntasks, uint64_t total_k, uint32_t *d_out,
                           void *stream)
{
    if (total_k == 0) return WRS_OK;
    if (!d_tasks || ntasks == 0 || !d_out) return WRS_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_tasks) % 16) != 0) return WRS_EINVAL;
    const uint64_t blocks = (total_k + kManyPerBlock - 1) / kManyPerBlock;
    if (blocks >= (1ull << 31)) return WRS_EINVAL;
    k_sample_many<<<(uint32_t)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const SampleTask *>(d_tasks), ntasks, total_k, d_out);
    return launch_err();
}

void wrs_batch_free(wrs_batch *b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    for (int i = 0; i < 7; ++i)
        if (b->map[i]) cudaFree(b->map[i]);
    if (b->buckets) cudaFree(b->buckets);
    if (b->ws) cudaFree(b->ws);
    delete b;
}

} // extern "C"
