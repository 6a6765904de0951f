// wrs.cu -- libwrs: the C ABI declared in include/wrs.h and the table
// runtime around the kernels of wrs_kernels.cuh (workspace layout, launch
// configuration, stream ordering, status handling).
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>

#include "wrs.h"
#include "wrs_kernels.cuh"

using namespace wrs;

constexpr int kStages = 6; // stats, stats_combine, classify, tilescan, split, sweep
constexpr int kOpSlots = 8; // streams whose last operation on a table is tracked

// The last operation a table enqueued on each stream it was used with, and
// the end of its last build: the waits of the host-side calls (status,
// info, download, upload, free) wait for these events only, never for the
// whole device.
struct OpLog {
    std::mutex mu;
    cudaStream_t priv = nullptr;  // library-private stream (read-backs, uploads, frees), made on first need
    cudaEvent_t build_ev = nullptr;
    bool built = false;
    cudaStream_t slot_stream[kOpSlots] = {};
    cudaEvent_t slot_ev[kOpSlots] = {};
    int nslots = 0, next = 0;
};

struct wrs_table {
    uint64_t cap;          // capacity in weights
    uint64_t n;            // weights of the last build (0: never built)
    uint32_t ntiles_cap;
    uint32_t epoch;        // look-back flag generation
    int device;
    uint8_t *ws;           // workspace block
    DevHeader *hdr;
    Partial *part;
    TileSum *agg, *incl;        // per tile
    TileSum *cagg, *cincl;      // per look-back chunk (256 tiles)
    uint32_t *flags;            // per chunk
    Split *split;
    uint16_t *slist;            // per tile, kSparse offsets
    uint4 *buckets;        // wrs_bucket[cap]
    void *stage_w;         // host-API staging (weights), bytes = stage_w_bytes
    uint64_t stage_w_bytes;
    uint32_t *stage_out;   // host-API staging (samples)
    uint64_t stage_out_cap;
    cudaStream_t copy_stream; // host-API: device-to-host copies overlapped with sampling
    cudaEvent_t copy_ev;
    int host_status;       // last status read back (-1: unknown)
    cudaEvent_t ev[kStages + 1]; // stage timing (created when enabled)
    int timing;            // record ev[] around the build's kernels
    int timed_build;       // the last build recorded ev[]
    uint8_t *pp_ws;        // PSA+ scratch (allocated by the first PSA+ build)
    uint64_t pp_n;         // n of the last PSA+ build (0: the last build was not PSA+)
    OpLog *log;            // per-stream completion events
};

namespace {

constexpr uint32_t kMaxParts = 2048;     // blocks of k_stats
std::atomic<uint32_t> g_wait_limit{1u << 22};
std::atomic<int64_t> g_skip_tile{-1};

inline uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

struct Layout {
    uint64_t hdr, part, agg, incl, cagg, cincl, flags, split, slist, total;
};

Layout layout_for(uint32_t ntiles)
{
    const uint32_t nchunks = (ntiles + kScanChunk - 1) / kScanChunk;
    Layout L;
    uint64_t o = 0;
    L.hdr = o; o = align_up(o + sizeof(DevHeader), 256);
    L.part = o; o = align_up(o + kMaxParts * sizeof(Partial), 256);
    L.agg = o; o = align_up(o + (uint64_t)ntiles * sizeof(TileSum), 256);
    L.incl = o; o = align_up(o + (uint64_t)ntiles * sizeof(TileSum), 256);
    L.cagg = o; o = align_up(o + (uint64_t)nchunks * sizeof(TileSum), 256);
    L.cincl = o; o = align_up(o + (uint64_t)nchunks * sizeof(TileSum), 256);
    L.flags = o; o = align_up(o + (uint64_t)nchunks * sizeof(uint32_t), 256);
    L.split = o; o = align_up(o + (uint64_t)ntiles * sizeof(Split), 256);
    L.slist = o; o = align_up(o + (uint64_t)ntiles * kSparse * sizeof(uint16_t), 256);
    L.total = o;
    return L;
}

inline wrs_status cuda_err(cudaError_t e)
{
    if (e == cudaSuccess) return WRS_OK;
    if (e == cudaErrorMemoryAllocation) return WRS_ENOMEM;
    return WRS_EDEVICE;
}

inline wrs_status launch_err() { return cuda_err(cudaGetLastError()); }

// Check build: the buckets start at zero before a build, so that their
// reserved words count the stores that reach them.  Nothing in the standard
// build.
inline wrs_status check_clear(void *buckets, uint64_t count, cudaStream_t s)
{
#if WRS_CHECK
    return cuda_err(cudaMemsetAsync(buckets, 0, count * sizeof(uint4), s));
#else
    (void)buckets;
    (void)count;
    (void)s;
    return WRS_OK;
#endif
}

int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

std::atomic<bool> g_attr_done[64];
std::mutex g_attr_mu;

wrs_status set_kernel_attributes()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return WRS_EDEVICE;
    if (g_attr_done[dev].load(std::memory_order_acquire)) return WRS_OK;
    std::lock_guard<std::mutex> lock(g_attr_mu);
    if (g_attr_done[dev].load(std::memory_order_relaxed)) return WRS_OK;
    const int bytes = (int)sizeof(SweepSmem);
    cudaError_t e = cudaFuncSetAttribute(k_sweep<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sweep<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return WRS_EDEVICE;
    g_attr_done[dev].store(true, std::memory_order_release);
    return WRS_OK;
}

// Record the end of an operation on table t enqueued on stream s (and of its
// build, when it is one).  A stream beyond the tracked slots takes the slot
// used longest ago, after the host has waited for that slot's operation.
wrs_status log_op(wrs_table *t, cudaStream_t s, bool build)
{
    OpLog &L = *t->log;
    std::lock_guard<std::mutex> lock(L.mu);
    cudaError_t e = cudaSuccess;
    if (build) {
        e = cudaEventRecord(L.build_ev, s);
        if (e != cudaSuccess) return cuda_err(e);
        L.built = true;
    }
    int k = 0;
    while (k < L.nslots && L.slot_stream[k] != s) ++k;
    if (k == L.nslots) {
        if (L.nslots < kOpSlots) {
            e = cudaEventCreateWithFlags(&L.slot_ev[k], cudaEventDisableTiming);
            if (e != cudaSuccess) return cuda_err(e);
            ++L.nslots;
        } else {
            k = L.next;
            L.next = (L.next + 1) % kOpSlots;
            e = cudaEventSynchronize(L.slot_ev[k]);
            if (e != cudaSuccess) return cuda_err(e);
        }
        L.slot_stream[k] = s;
    }
    return cuda_err(cudaEventRecord(L.slot_ev[k], s));
}

// Host wait for the table's last build only.
wrs_status wait_build(const wrs_table *t)
{
    OpLog &L = *t->log;
    std::lock_guard<std::mutex> lock(L.mu);
    return L.built ? cuda_err(cudaEventSynchronize(L.build_ev)) : WRS_OK;
}

// The table's private stream, created on first need: a table that is only
// built and sampled (a serving pool holds thousands) owns no stream.
wrs_status ensure_priv(OpLog &L)
{
    if (L.priv) return WRS_OK;
    return cuda_err(cudaStreamCreateWithFlags(&L.priv, cudaStreamNonBlocking));
}

// Make the private stream wait for every tracked operation on the table
// (device-side ordering; the host does not wait).
wrs_status order_after_all(const wrs_table *t)
{
    OpLog &L = *t->log;
    std::lock_guard<std::mutex> lock(L.mu);
    const wrs_status st = ensure_priv(L);
    if (st != WRS_OK) return st;
    for (int k = 0; k < L.nslots; ++k) {
        cudaError_t e = cudaStreamWaitEvent(L.priv, L.slot_ev[k], 0);
        if (e != cudaSuccess) return cuda_err(e);
    }
    return WRS_OK;
}

// Copy device bytes of the table to host memory after its last build, on
// the private stream.
wrs_status read_back(const wrs_table *t, void *h, const void *d, size_t bytes)
{
    wrs_status st = wait_build(t);
    if (st != WRS_OK) return st;
    {
        std::lock_guard<std::mutex> lock(t->log->mu);
        st = ensure_priv(*t->log);
    }
    if (st != WRS_OK) return st;
    cudaError_t e = cudaMemcpyAsync(h, d, bytes, cudaMemcpyDeviceToHost, t->log->priv);
    if (e == cudaSuccess) e = cudaStreamSynchronize(t->log->priv);
    return cuda_err(e);
}

// Build options after validation: own tiles per sweep block (one subproblem
// of Alg. 3 each), the accumulator mode.
struct BuildOpts {
    uint32_t group = kSweepTiles;
    int acc = WRS_ACC_AUTO;
};

wrs_status enqueue_build(wrs_table *t, const void *d_weights, uint64_t n, wrs_dtype dtype, cudaStream_t s,
                         const BuildOpts &o = BuildOpts())
{
    {
        const wrs_status st = set_kernel_attributes();
        if (st != WRS_OK) return st;
    }
    const uint32_t *w = static_cast<const uint32_t *>(d_weights);
    const int vec = (reinterpret_cast<uintptr_t>(w) % 16) == 0;
    const uint32_t ntiles = (uint32_t)((n + kTile - 1) / kTile);
    const uint32_t f32 = dtype == WRS_F32;
    uint64_t want = (n + (uint64_t)kThreads * 16 - 1) / ((uint64_t)kThreads * 16);
    uint32_t nparts = (uint32_t)(want < 1 ? 1 : (want > kMaxParts ? kMaxParts : want));
    uint32_t blocks_cap = (uint32_t)sm_count() * 8;
    if (nparts > blocks_cap) nparts = blocks_cap;

    t->epoch = t->epoch + 1;
    if (t->epoch >= (1u << 30)) t->epoch = 1;
    const uint32_t epoch = t->epoch;
    const uint32_t wait_limit = g_wait_limit.load();
    const int64_t skip = g_skip_tile.exchange(-1);
    const uint32_t skip_tile = skip < 0 ? kNone : (uint32_t)skip;

    const uint32_t nchunks = (ntiles + kScanChunk - 1) / kScanChunk;
    uint32_t cls_blocks = (uint32_t)sm_count() * 8; // one warp per tile
    if (cls_blocks > (ntiles + kWarps - 1) / kWarps) cls_blocks = (ntiles + kWarps - 1) / kWarps;
    {
        const wrs_status st = check_clear(t->buckets, n, s);
        if (st != WRS_OK) return st;
    }
    const bool tm = t->timing != 0;
    if (tm) cudaEventRecord(t->ev[0], s);
    if (f32) k_stats<1><<<nparts, kThreads, 0, s>>>(w, n, vec, t->part);
    else k_stats<0><<<nparts, kThreads, 0, s>>>(w, n, vec, t->part);
    if (tm) cudaEventRecord(t->ev[1], s);
    k_stats_combine<<<1, kThreads, 0, s>>>(t->part, nparts, n, f32, t->hdr);
    if (tm) cudaEventRecord(t->ev[2], s);
    if (f32) k_classify<1><<<cls_blocks, kThreads, 0, s>>>(w, n, vec, t->hdr, t->agg, t->slist, ntiles);
    else k_classify<0><<<cls_blocks, kThreads, 0, s>>>(w, n, vec, t->hdr, t->agg, t->slist, ntiles);
    if (tm) cudaEventRecord(t->ev[3], s);
    k_tilescan<<<nchunks, kThreads, 0, s>>>(t->hdr, t->agg, t->cagg, t->cincl, t->incl, t->flags, ntiles, epoch,
                                            wait_limit, skip_tile);
    if (tm) cudaEventRecord(t->ev[4], s);
    k_split<<<(ntiles + kThreads - 1) / kThreads, kThreads, 0, s>>>(t->incl, ntiles, n, t->hdr, t->split);
    if (o.acc == WRS_ACC_U64) k_require_u64<<<1, 32, 0, s>>>(t->hdr);
    if (tm) cudaEventRecord(t->ev[5], s);
    const size_t sweep_smem = sizeof(SweepSmem);
    const uint32_t sweep_blocks = (ntiles + o.group - 1) / o.group;
    const int wide = o.acc == WRS_ACC_U128;
    if (f32) k_sweep<1><<<sweep_blocks, kThreads, sweep_smem, s>>>(w, n, vec, t->hdr, t->incl, t->split, t->slist, ntiles, t->buckets, o.group, wide);
    else k_sweep<0><<<sweep_blocks, kThreads, sweep_smem, s>>>(w, n, vec, t->hdr, t->incl, t->split, t->slist, ntiles, t->buckets, o.group, wide);
    if (tm) cudaEventRecord(t->ev[6], s);
    t->timed_build = tm;
    wrs_status st = launch_err();
    if (st == WRS_OK) st = log_op(t, s, true);
    if (st == WRS_OK) {
        t->n = n;
        t->host_status = -1;
        t->pp_n = 0;
    }
    return st;
}

// Samples [s0, s1) of the table into d_out[s0 ...].
wrs_status launch_sample(const wrs_table *t, uint64_t s0, uint64_t s1, uint64_t seed, uint64_t stream_id,
                         uint32_t *d_out, cudaStream_t s)
{
    const int sms = sm_count();
    const uint64_t k = s1 - s0;
    uint64_t want = (k + 256ull * kSampleUnroll - 1) / (256ull * kSampleUnroll);
    uint64_t cap = (uint64_t)sms * 16; // 16 blocks per SM: more random loads in flight
    const uint32_t blocks = (uint32_t)(want < cap ? (want < 1 ? 1 : want) : cap);
    k_sample<<<blocks, 256, 0, s>>>(t->buckets, t->n, t->hdr, s0, s1, (uint32_t)seed, (uint32_t)(seed >> 32),
                                    (uint32_t)stream_id, (uint32_t)(stream_id >> 32), d_out);
    return launch_err();
}

wrs_status read_status(const wrs_table *t, uint32_t *out)
{
    return read_back(t, out, &t->hdr->status, sizeof(uint32_t));
}

void destroy_log(OpLog *L)
{
    if (!L) return;
    for (int k = 0; k < L->nslots; ++k) cudaEventDestroy(L->slot_ev[k]);
    if (L->build_ev) cudaEventDestroy(L->build_ev);
    if (L->priv) cudaStreamDestroy(L->priv); // pending work still completes
    delete L;
}

} // namespace

extern "C" {

wrs_status wrs_table_create(uint64_t capacity_n, wrs_table **out)
{
    if (!out) return WRS_EINVAL;
    *out = nullptr;
    if (capacity_n == 0 || capacity_n >= (1ull << 32)) return WRS_EINVAL;
    wrs_table *t = new (std::nothrow) wrs_table();
    if (!t) return WRS_ENOMEM;
    std::memset(t, 0, sizeof(*t));
    t->log = new (std::nothrow) OpLog();
    if (!t->log) { delete t; return WRS_ENOMEM; }
    t->cap = capacity_n;
    t->ntiles_cap = (uint32_t)((capacity_n + kTile - 1) / kTile);
    t->host_status = -1;
    cudaGetDevice(&t->device);
    const Layout L = layout_for(t->ntiles_cap);
    cudaError_t e = cudaStreamCreateWithFlags(&t->log->priv, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t->log->build_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) { destroy_log(t->log); delete t; return cuda_err(e); }
    // stream-ordered allocations on the private stream, so that freeing the
    // table is stream-ordered too (cudaFreeAsync)
    cudaStream_t ps = t->log->priv;
    e = cudaMallocAsync(reinterpret_cast<void **>(&t->ws), L.total, ps);
    if (e != cudaSuccess) { destroy_log(t->log); delete t; return cuda_err(e); }
    e = cudaMallocAsync(reinterpret_cast<void **>(&t->buckets), capacity_n * sizeof(uint4), ps);
    if (e != cudaSuccess) {
        cudaFreeAsync(t->ws, ps);
        cudaStreamSynchronize(ps);
        destroy_log(t->log);
        delete t;
        return cuda_err(e);
    }
    t->hdr = reinterpret_cast<DevHeader *>(t->ws + L.hdr);
    t->part = reinterpret_cast<Partial *>(t->ws + L.part);
    t->agg = reinterpret_cast<TileSum *>(t->ws + L.agg);
    t->incl = reinterpret_cast<TileSum *>(t->ws + L.incl);
    t->cagg = reinterpret_cast<TileSum *>(t->ws + L.cagg);
    t->cincl = reinterpret_cast<TileSum *>(t->ws + L.cincl);
    t->flags = reinterpret_cast<uint32_t *>(t->ws + L.flags);
    t->split = reinterpret_cast<Split *>(t->ws + L.split);
    t->slist = reinterpret_cast<uint16_t *>(t->ws + L.slist);
    e = cudaMemsetAsync(t->ws, 0, L.total, ps);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ps);
    if (e != cudaSuccess) {
        cudaFreeAsync(t->ws, ps);
        cudaFreeAsync(t->buckets, ps);
        cudaStreamSynchronize(ps);
        destroy_log(t->log);
        delete t;
        return cuda_err(e);
    }
    // the memory is ready for every stream; the private stream is made again
    // on first need
    cudaStreamDestroy(ps);
    t->log->priv = nullptr;
    *out = t;
    return WRS_OK;
}

wrs_status wrs_table_build(wrs_table *t, const void *d_weights, uint64_t n, wrs_dtype dtype, void *stream)
{
    if (!t || !d_weights || n == 0 || n > t->cap) return WRS_EINVAL;
    if (dtype != WRS_U32 && dtype != WRS_F32) return WRS_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_weights) % 4) != 0) return WRS_EINVAL;
    return enqueue_build(t, d_weights, n, dtype, static_cast<cudaStream_t>(stream));
}

wrs_status wrs_table_build_opts(wrs_table *t, const void *d_weights, uint64_t n, wrs_dtype dtype,
                                const wrs_build_opts *opts, void *stream)
{
    if (!t || !d_weights || n == 0 || n > t->cap) return WRS_EINVAL;
    if (dtype != WRS_U32 && dtype != WRS_F32) return WRS_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_weights) % 4) != 0) return WRS_EINVAL;
    BuildOpts o;
    if (opts) {
        if (opts->flags != 0) return WRS_EINVAL;
        if (opts->tile != 0 && opts->tile != (uint32_t)kTile) return WRS_EINVAL;
        if (opts->window != 0 && opts->window != (uint32_t)kTile) return WRS_EINVAL;
        if (opts->acc != WRS_ACC_AUTO && opts->acc != WRS_ACC_U64 && opts->acc != WRS_ACC_U128) return WRS_EINVAL;
        const uint32_t ntiles = (uint32_t)((n + kTile - 1) / kTile);
        if (opts->splits > ntiles) return WRS_EINVAL;
        if (opts->splits) o.group = (ntiles + opts->splits - 1) / opts->splits;
        o.acc = opts->acc;
    }
    return enqueue_build(t, d_weights, n, dtype, static_cast<cudaStream_t>(stream), o);
}

wrs_status wrs_build(const void *d_weights, uint64_t n, wrs_dtype dtype, void *stream, wrs_table **out)
{
    if (!out) return WRS_EINVAL;
    *out = nullptr;
    wrs_table *t = nullptr;
    wrs_status st = wrs_table_create(n, &t);
    if (st != WRS_OK) return st;
    st = wrs_table_build(t, d_weights, n, dtype, stream);
    if (st != WRS_OK) { wrs_table_free(t); return st; }
    *out = t;
    return WRS_OK;
}

wrs_status wrs_sample(const wrs_table *t, uint64_t k, uint64_t seed, uint64_t stream_id, uint32_t *d_out,
                      void *stream)
{
    if (!t || t->n == 0) return WRS_EINVAL;
    if (k == 0) return WRS_OK;
    if (!d_out) return WRS_EINVAL;
    if (t->host_status > 0) return (wrs_status)t->host_status;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    wrs_status st = launch_sample(t, 0, k, seed, stream_id, d_out, s);
    if (st == WRS_OK) st = log_op(const_cast<wrs_table *>(t), s, false);
    return st;
}

wrs_status wrs_table_build_host(wrs_table *t, const void *h_weights, uint64_t n, wrs_dtype dtype, void *stream)
{
    if (!t || !h_weights || n == 0 || n > t->cap) return WRS_EINVAL;
    if (dtype != WRS_U32 && dtype != WRS_F32) return WRS_EINVAL;
    const uint64_t bytes = n * 4;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (t->stage_w_bytes < bytes) {
        if (t->stage_w) { // freed once every operation of the table that may read it is done
            wrs_status st = order_after_all(t);
            if (st != WRS_OK) return st;
            cudaFreeAsync(t->stage_w, t->log->priv);
            t->stage_w = nullptr;
            t->stage_w_bytes = 0;
        }
        cudaError_t e = cudaMallocAsync(&t->stage_w, bytes, s);
        if (e != cudaSuccess) return cuda_err(e);
        t->stage_w_bytes = bytes;
    }
    cudaError_t e = cudaMemcpyAsync(t->stage_w, h_weights, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_err(e);
    return enqueue_build(t, t->stage_w, n, dtype, s);
}

wrs_status wrs_sample_host(wrs_table *t, uint64_t k, uint64_t seed, uint64_t stream_id, uint32_t *h_out,
                           void *stream)
{
    if (!t || t->n == 0) return WRS_EINVAL;
    if (k == 0) return WRS_OK;
    if (!h_out) return WRS_EINVAL;
    if (t->host_status > 0) return (wrs_status)t->host_status;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (t->stage_out_cap < k) {
        if (t->stage_out) { // every earlier host-buffer sample has synchronised already
            cudaFreeAsync(t->stage_out, s);
            t->stage_out = nullptr;
            t->stage_out_cap = 0;
        }
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&t->stage_out), k * sizeof(uint32_t), s);
        if (e != cudaSuccess) return cuda_err(e);
        t->stage_out_cap = k;
    }
    if (!t->copy_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&t->copy_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t->copy_ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_err(e);
    }
    // sample in chunks; each chunk's copy to the host runs on copy_stream
    // while the next chunk is drawn
    const uint64_t chunk = 1ull << 25;
    for (uint64_t c0 = 0; c0 < k; c0 += chunk) {
        const uint64_t c1 = c0 + chunk < k ? c0 + chunk : k;
        wrs_status st = launch_sample(t, c0, c1, seed, stream_id, t->stage_out, s);
        if (st != WRS_OK) return st;
        cudaError_t e = cudaEventRecord(t->copy_ev, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(t->copy_stream, t->copy_ev, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_out + c0, t->stage_out + c0, (c1 - c0) * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                t->copy_stream);
        if (e != cudaSuccess) return cuda_err(e);
    }
    wrs_status st = log_op(t, s, false);
    if (st != WRS_OK) return st;
    cudaError_t e = cudaStreamSynchronize(t->copy_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return cuda_err(e);
}

wrs_status wrs_table_status(const wrs_table *t)
{
    if (!t) return WRS_EINVAL;
    if (t->n == 0) return WRS_EINVAL;
    uint32_t st = 0;
    wrs_status e = read_status(t, &st);
    if (e != WRS_OK) return e;
    const_cast<wrs_table *>(t)->host_status = (int)st;
    return (wrs_status)st;
}

wrs_status wrs_table_info_get(const wrs_table *t, wrs_table_info *info)
{
    if (!t || !info) return WRS_EINVAL;
    if (t->n == 0) return WRS_EINVAL;
    DevHeader h;
    const wrs_status st = read_back(t, &h, t->hdr, sizeof(h));
    if (st != WRS_OK) return st;
    info->n = t->n;
    info->q_lo = h.q_lo;
    info->q_hi = h.q_hi;
    info->beta = h.beta;
    info->shift = h.shift;
    info->qp = h.qp;
    info->n_light = h.n_light;
    info->light_max = h.light_max;
    info->status = (int32_t)h.status;
    const_cast<wrs_table *>(t)->host_status = (int)h.status;
    return WRS_OK;
}

int wrs_check_build(void) { return WRS_CHECK; }

wrs_status wrs_table_check_failures(const wrs_table *t, uint64_t *failures)
{
    if (!t || !failures || t->n == 0) return WRS_EINVAL;
    DevHeader h;
    const wrs_status st = read_back(t, &h, t->hdr, sizeof(h));
    if (st != WRS_OK) return st;
    *failures = h.pad[0];
    return WRS_OK;
}

const wrs_bucket *wrs_table_buckets(const wrs_table *t)
{
    return t ? reinterpret_cast<const wrs_bucket *>(t->buckets) : nullptr;
}

wrs_status wrs_table_download(const wrs_table *t, void *h_buckets, uint64_t bytes)
{
    if (!t || !h_buckets || t->n == 0 || bytes < t->n * sizeof(uint4)) return WRS_EINVAL;
    return read_back(t, h_buckets, t->buckets, t->n * sizeof(uint4));
}

wrs_status wrs_table_upload(wrs_table *t, const void *h_buckets, uint64_t n, uint64_t q_lo, uint64_t q_hi,
                            int32_t beta)
{
    if (!t || !h_buckets || n == 0 || n > t->cap) return WRS_EINVAL;
    if ((q_lo | q_hi) == 0 || (q_hi >> 31) != 0) return WRS_EINVAL;
    DevHeader h;
    std::memset(&h, 0, sizeof(h));
    unsigned __int128 Q = ((unsigned __int128)q_hi << 64) | q_lo;
    int bits = 0;
    for (unsigned __int128 v = Q; v; v >>= 1) ++bits;
    int shift = bits > 64 ? bits - 64 : 0;
    h.status = 0;
    h.beta = beta;
    h.shift = (uint32_t)shift;
    h.q_lo = q_lo;
    h.q_hi = q_hi;
    h.qp = (uint64_t)(Q >> shift);
    h.n = n;
    // after every operation of the table (samples may still read the
    // buckets), on the private stream; synchronous for the caller
    wrs_status st = order_after_all(t);
    if (st != WRS_OK) return st;
    cudaStream_t ps = t->log->priv;
    cudaError_t e = cudaMemcpyAsync(t->buckets, h_buckets, n * sizeof(uint4), cudaMemcpyHostToDevice, ps);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t->hdr, &h, sizeof(h), cudaMemcpyHostToDevice, ps);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ps);
    if (e != cudaSuccess) return cuda_err(e);
    st = log_op(t, ps, true);
    if (st != WRS_OK) return st;
    t->n = n;
    t->host_status = 0;
    t->pp_n = 0;
    return WRS_OK;
}

wrs_status wrs_table_set_timing(wrs_table *t, int enable)
{
    if (!t) return WRS_EINVAL;
    if (enable && !t->timing) {
        for (int i = 0; i <= kStages; ++i) {
            cudaError_t e = cudaEventCreate(&t->ev[i]);
            if (e != cudaSuccess) {
                for (int j = 0; j < i; ++j) cudaEventDestroy(t->ev[j]);
                return cuda_err(e);
            }
        }
        t->timing = 1;
    } else if (!enable && t->timing) {
        for (int i = 0; i <= kStages; ++i) cudaEventDestroy(t->ev[i]); // pending records still complete
        t->timing = 0;
        t->timed_build = 0;
    }
    return WRS_OK;
}

wrs_status wrs_table_stage_ms(const wrs_table *t, float *ms, uint32_t count)
{
    if (!t || !ms || count == 0 || count > (uint32_t)kStages) return WRS_EINVAL;
    if (!t->timing || !t->timed_build) return WRS_EINVAL;
    cudaError_t e = cudaEventSynchronize(t->ev[kStages]);
    for (uint32_t i = 0; e == cudaSuccess && i < count; ++i) e = cudaEventElapsedTime(&ms[i], t->ev[i], t->ev[i + 1]);
    return cuda_err(e);
}

void wrs_table_free(wrs_table *t)
{
    if (!t) return;
    // stream-ordered: the memory is released on the private stream once every
    // tracked operation of the table has completed; the host does not wait
    const wrs_status st = order_after_all(t);
    cudaStream_t ps = t->log->priv;
    if (st != WRS_OK) cudaStreamSynchronize(ps);
    if (t->timing)
        for (int i = 0; i <= kStages; ++i) cudaEventDestroy(t->ev[i]);
    if (t->copy_ev) cudaEventRecord(t->copy_ev, t->copy_stream);
    if (t->copy_ev) cudaStreamWaitEvent(ps, t->copy_ev, 0);
    cudaFreeAsync(t->ws, ps);
    cudaFreeAsync(t->buckets, ps);
    if (t->stage_w) cudaFreeAsync(t->stage_w, ps);
    if (t->stage_out) cudaFreeAsync(t->stage_out, ps);
    if (t->pp_ws) cudaFreeAsync(t->pp_ws, ps);
    if (t->copy_stream) cudaStreamDestroy(t->copy_stream);
    if (t->copy_ev) cudaEventDestroy(t->copy_ev);
    destroy_log(t->log);
    delete t;
}

const char *wrs_status_str(wrs_status s)
{
    switch (s) {
    case WRS_OK: return "ok";
    case WRS_EINVAL: return "invalid argument or weights";
    case WRS_ENOMEM: return "out of memory";
    case WRS_EOVERFLOW: return "exact weight sum exceeds 95 bits";
    case WRS_ETIMEOUT: return "bounded device wait ran out";
    case WRS_EDEVICE: return "CUDA runtime error";
    case WRS_EINTERNAL: return "internal invariant failed";
    }
    return "unknown status";
}

uint32_t wrs_set_wait_limit(uint32_t polls)
{
    if (polls == 0) polls = 1;
    return g_wait_limit.exchange(polls);
}

void wrs_debug_skip_publish(int64_t tile)
{
    g_skip_tile.store(tile);
}

} // extern "C"

// ---------------------------------------------------------------------------
// Build without any allocation (wrs_build_noalloc).
//
// Some callers cannot call cudaMalloc: a real-time or embedded process whose
// device memory budget is fixed at start-up, or a host framework that owns
// all device memory through its own pool and forbids allocations behind its
// back.  For them, the build's scratch (per-block
// partial sums, tile sums and prefixes, look-back flags, split results,
// sparse member lists) lives in one file-scope device array sized for
// WRS_NOALLOC_MAX_N weights; the caller passes the weights, the output
// buckets and the output header.  Every GPU that loads the library holds
// this array until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr uint64_t kNaMaxN = WRS_NOALLOC_MAX_N;
constexpr uint32_t kNaTiles = (uint32_t)((kNaMaxN + kTile - 1) / kTile);
constexpr uint32_t kNaChunks = (kNaTiles + kScanChunk - 1) / kScanChunk;
constexpr uint64_t na_up(uint64_t x) { return (x + 255) / 256 * 256; }
constexpr uint64_t kNaPart = 0;
constexpr uint64_t kNaAgg = kNaPart + na_up(kMaxParts * sizeof(Partial));
constexpr uint64_t kNaIncl = kNaAgg + na_up((uint64_t)kNaTiles * sizeof(TileSum));
constexpr uint64_t kNaCagg = kNaIncl + na_up((uint64_t)kNaTiles * sizeof(TileSum));
constexpr uint64_t kNaCincl = kNaCagg + na_up((uint64_t)kNaChunks * sizeof(TileSum));
constexpr uint64_t kNaFlags = kNaCincl + na_up((uint64_t)kNaChunks * sizeof(TileSum));
constexpr uint64_t kNaSplit = kNaFlags + na_up((uint64_t)kNaChunks * sizeof(uint32_t));
constexpr uint64_t kNaSlist = kNaSplit + na_up((uint64_t)kNaTiles * sizeof(Split));
constexpr uint64_t kNaBytes = kNaSlist + na_up((uint64_t)kNaTiles * kSparse * sizeof(uint16_t));

// Zero at module load.  Every call clears the look-back flags on its stream
// before the scan and publishes with generation 1, so nothing on the launch
// path depends on host state that changes from call to call.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

constexpr uint32_t kNaEpoch = 1;

struct NoallocDevice {
    std::atomic<unsigned char *> scratch{nullptr}; // device address of g_noalloc_scratch on this device
    std::mutex init;                               // first-call set-up, once per device
};
NoallocDevice g_noalloc[64];

static_assert(sizeof(DevHeader) <= WRS_DEVICE_HEADER_BYTES, "device header does not fit");
static_assert(offsetof(DevHeader, status) == offsetof(wrs_device_header, status), "layout");
static_assert(offsetof(DevHeader, tile_counter) == offsetof(wrs_device_header, tile_counter), "layout");
static_assert(offsetof(DevHeader, f32) == offsetof(wrs_device_header, f32), "layout");
static_assert(offsetof(DevHeader, beta) == offsetof(wrs_device_header, beta), "layout");
static_assert(offsetof(DevHeader, shift) == offsetof(wrs_device_header, shift), "layout");
static_assert(offsetof(DevHeader, q_lo) == offsetof(wrs_device_header, q_lo), "layout");
static_assert(offsetof(DevHeader, q_hi) == offsetof(wrs_device_header, q_hi), "layout");
static_assert(offsetof(DevHeader, qp) == offsetof(wrs_device_header, qp), "layout");
static_assert(offsetof(DevHeader, light_max) == offsetof(wrs_device_header, light_max), "layout");
static_assert(offsetof(DevHeader, n) == offsetof(wrs_device_header, n), "layout");
static_assert(offsetof(DevHeader, n_light) == offsetof(wrs_device_header, n_light), "layout");
static_assert(sizeof(wrs_device_header) == WRS_DEVICE_HEADER_BYTES, "layout");

} // namespace

extern "C" wrs_status wrs_build_noalloc(const void *d_weights, uint64_t n, wrs_dtype dtype, void *d_buckets,
                                        void *d_header, void *stream)
{
    if (!d_weights || !d_buckets || !d_header || n == 0) return WRS_EINVAL;
    if (n > kNaMaxN) return WRS_EINVAL; // beyond the static scratch: use wrs_table_create/wrs_table_build
    if (dtype != WRS_U32 && dtype != WRS_F32) return WRS_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_weights) % 4) != 0) return WRS_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_buckets) % 16) != 0 || (reinterpret_cast<uintptr_t>(d_header) % 16) != 0)
        return WRS_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return WRS_EDEVICE;
    NoallocDevice &D = g_noalloc[dev];
    unsigned char *scratch = D.scratch.load(std::memory_order_acquire);
    if (!scratch) {
        // once per device, with that device current: the array's device address
        std::lock_guard<std::mutex> lock(D.init);
        scratch = D.scratch.load(std::memory_order_relaxed);
        if (!scratch) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return WRS_EDEVICE;
            const wrs_status st = set_kernel_attributes();
            if (st != WRS_OK) return st;
            scratch = static_cast<unsigned char *>(ptr);
            D.scratch.store(scratch, std::memory_order_release);
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint32_t *w = static_cast<const uint32_t *>(d_weights);
    const int vec = (reinterpret_cast<uintptr_t>(w) % 16) == 0;
    const uint32_t ntiles = (uint32_t)((n + kTile - 1) / kTile);
    const uint32_t nchunks = (ntiles + kScanChunk - 1) / kScanChunk;
    const uint32_t f32 = dtype == WRS_F32;
    DevHeader *hdr = static_cast<DevHeader *>(d_header);
    uint4 *buckets = static_cast<uint4 *>(d_buckets);
    Partial *part = reinterpret_cast<Partial *>(scratch + kNaPart);
    TileSum *agg = reinterpret_cast<TileSum *>(scratch + kNaAgg);
    TileSum *incl = reinterpret_cast<TileSum *>(scratch + kNaIncl);
    TileSum *cagg = reinterpret_cast<TileSum *>(scratch + kNaCagg);
    TileSum *cincl = reinterpret_cast<TileSum *>(scratch + kNaCincl);
    uint32_t *flags = reinterpret_cast<uint32_t *>(scratch + kNaFlags);
    Split *split = reinterpret_cast<Split *>(scratch + kNaSplit);
    uint16_t *slist = reinterpret_cast<uint16_t *>(scratch + kNaSlist);

    uint64_t want = (n + (uint64_t)kThreads * 16 - 1) / ((uint64_t)kThreads * 16);
    uint32_t nparts = (uint32_t)(want < 1 ? 1 : (want > kMaxParts ? kMaxParts : want));
    const uint32_t blocks_cap = (uint32_t)sm_count() * 8;
    if (nparts > blocks_cap) nparts = blocks_cap;
    const uint32_t cls_want = (ntiles + kWarps - 1) / kWarps; // one warp per tile
    uint32_t cls_blocks = blocks_cap < cls_want ? blocks_cap : cls_want;
    // the look-back flags start from zero on the stream, in stream order with
    // the scan that reads them
    if (cudaMemsetAsync(flags, 0, (size_t)nchunks * sizeof(uint32_t), s) != cudaSuccess) return WRS_EDEVICE;
    if (check_clear(buckets, n, s) != WRS_OK) return WRS_EDEVICE;

    if (f32) k_stats<1><<<nparts, kThreads, 0, s>>>(w, n, vec, part);
    else k_stats<0><<<nparts, kThreads, 0, s>>>(w, n, vec, part);
    k_stats_combine<<<1, kThreads, 0, s>>>(part, nparts, n, f32, hdr);
    if (f32) k_classify<1><<<cls_blocks, kThreads, 0, s>>>(w, n, vec, hdr, agg, slist, ntiles);
    else k_classify<0><<<cls_blocks, kThreads, 0, s>>>(w, n, vec, hdr, agg, slist, ntiles);
    k_tilescan<<<nchunks, kThreads, 0, s>>>(hdr, agg, cagg, cincl, incl, flags, ntiles, kNaEpoch,
                                            g_wait_limit.load(), kNone);
    k_split<<<(ntiles + kThreads - 1) / kThreads, kThreads, 0, s>>>(incl, ntiles, n, hdr, split);
    const uint32_t sweep_blocks = (ntiles + kSweepTiles - 1) / kSweepTiles;
    if (f32) k_sweep<1><<<sweep_blocks, kThreads, sizeof(SweepSmem), s>>>(w, n, vec, hdr, incl, split, slist, ntiles, buckets, kSweepTiles, 0);
    else k_sweep<0><<<sweep_blocks, kThreads, sizeof(SweepSmem), s>>>(w, n, vec, hdr, incl, split, slist, ntiles, buckets, kSweepTiles, 0);
    return launch_err();
}

#include "wrs_twolevel.cuh"
#include "wrs_batch.cuh"
#include "wrs_osnd.cuh"
#include "wrs_psaplus.cuh"
