// wrs_psaplus.cuh -- PSA+ builds (wrs_table_build_psa_plus of include/wrs.h).
// Included by wrs.cu only, after wrs_twolevel.cuh.
//
// Sec. 4.2 "Performance Optimization in Practice": every tile of 2048
// consecutive items (a PE's allotment) first runs Alg. 2 on its own items in
// the global units (capacity Q, item i weighs n q_i), stopping when the next
// light or the next heavy item would lie outside the tile; the items left
// over -- the heavy item current at the stop with its unassigned residual,
// every other unassigned item whole -- form, in index order, the input of
// Alg. 2 (= PSA) for the rest of the table.
//
// Phase 1 (k_pp_local, one block per tile): the tile's light keys D (prefix
// of deficits Q - n q) and heavy keys E (prefix of excesses n q - Q), local
// to the tile; with D_tot the tile's total deficit and E_last the last heavy
// key, either the lights run out first (E_last > D_tot: every light is
// packed, the heavies with E <= D_tot are packed, the next one stops with
// residual) or the last heavy is covered first (the lights with D < E_last
// are packed, every heavy but the last, which stops).  The packed items are
// one merge, as in the single table's sweep; the leftovers are staged per
// tile.  Phase 2: the leftovers are compacted (look-back scan of the tile
// counts), their global keys are written once (lights and heavies apart,
// look-back scan of per-tile sums), and one block per 2048 merge steps finds
// its start by a warp-cooperative co-rank search over those keys and walks.
#pragma once

namespace wrs {

// The table's status, read once for the whole block (every thread returns or
// none does, so no later barrier is left waiting).
__device__ __forceinline__ bool block_stopped(const DevHeader *hdr)
{
    __shared__ uint32_t s_st;
    if (threadIdx.x == 0) s_st = *(volatile const uint32_t *)&hdr->status;
    __syncthreads();
    return s_st != 0;
}

// ------------------------------------------------------------ phase 1
template <int F32>
__global__ void __launch_bounds__(kThreads, 3) k_pp_local(const uint32_t *__restrict__ w, uint64_t n, int vec,
                                                          DevHeader *hdr, uint4 *__restrict__ table,
                                                          uint64_t *__restrict__ lo_v, uint32_t *__restrict__ lo_idx,
                                                          TileSum *__restrict__ cnt_agg)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GroupSmem &S = *reinterpret_cast<GroupSmem *>(smem_raw);
    __shared__ uint32_t s_ab[2];
    __shared__ u128 s_res;
    if (block_stopped(hdr)) return;
    const uint32_t n32 = (uint32_t)n;
    const u128 Q = mk128(hdr->q_lo, hdr->q_hi);
    const uint32_t light_max = hdr->light_max, shift = hdr->shift;
    const int beta = hdr->beta;
    const uint64_t tile0 = (uint64_t)blockIdx.x * kTile;
    const uint64_t first = tile0 + (uint64_t)threadIdx.x * kItems;
    uint32_t x[kItems];
    load_items(w, n, vec, first, x);
    uint32_t lmask = 0, hmask = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        if (first + k < n) {
            if (x[k] <= light_max) lmask |= 1u << k; else hmask |= 1u << k;
        }
    }
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan_u32((uint32_t)__popc(lmask) | ((uint32_t)__popc(hmask) << 16), tot,
                                                 S.cnt);
    const uint32_t nl = tot & 0xFFFFu, nh = tot >> 16;
    const uint32_t l0 = ex & 0xFFFFu, h0 = ex >> 16;
    u128 sd = 0, se = 0;
    {
        uint32_t ls = l0, hs = h0;
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            if (!(((lmask | hmask) >> k) & 1u)) continue;
            const u128 nq = nq_of(x[k], F32, beta, n32);
            const uint16_t off = (uint16_t)(threadIdx.x * kItems + k);
            if ((lmask >> k) & 1u) {
                const u128 d = Q - nq;
                S.okey[swz(ls)] = d;
                S.ooff[ls] = off;
                sd += d;
                ++ls;
            } else {
                const u128 e = nq - Q;
                S.hkey[swz(hs)] = e;
                S.hoff[hs] = off;
                se += e;
                ++hs;
            }
        }
    }
    U2 sums;
    const U2 exs = block_exclusive_scan2(U2{sd, se}, sums, S.scan);
    {
        u128 kl = exs.a, ke = exs.b;
        for (uint32_t j = 0; j < (uint32_t)__popc(lmask); ++j) {
            const u128 d = S.okey[swz(l0 + j)];
            S.okey[swz(l0 + j)] = kl;
            kl += d;
        }
        for (uint32_t j = 0; j < (uint32_t)__popc(hmask); ++j) {
            ke += S.hkey[swz(h0 + j)];
            S.hkey[swz(h0 + j)] = ke;
        }
    }
    const u128 D_tot = sums.a;
    __syncthreads();
    // where the greedy pass stops: A lights and B heavies are packed
    if (threadIdx.x < 32) {
        uint32_t A = 0, B = 0;
        if (nh > 0) {
            const u128 E_last = S.hkey[swz(nh - 1)];
            if (E_last > D_tot) { A = nl; B = warp_search(S.hkey, 0, nh, D_tot, true); }
            else { A = warp_search(S.okey, 0, nl, E_last, false); B = nh - 1; }
        }
        if (threadIdx.x == 0) {
            s_ab[0] = A;
            s_ab[1] = B;
            if (B < nh) { // residual of the heavy item current at the stop
                const u128 DA = A < nl ? S.okey[swz(A)] : D_tot;
                s_res = S.hkey[swz(B)] - DA + Q;
            }
        }
    }
    __syncthreads();
    const uint32_t A = s_ab[0], B = s_ab[1];
    bool bad = false;
    // the packed items: lights [0, A) and heavies [0, B), one merge
    const uint32_t M = A + B;
    if (M > 0) {
        const uint32_t per = (M + kThreads - 1) / kThreads;
        const uint32_t d0 = threadIdx.x * per;
        if (d0 < M) {
            uint32_t lo = d0 > A ? d0 - A : 0, hi = d0 < B ? d0 : B;
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if (S.hkey[swz(mid - 1)] <= S.okey[swz(d0 - mid)]) lo = mid; else hi = mid - 1;
            }
            uint32_t j = lo, i = d0 - lo;
            const uint32_t steps = min(per, M - d0);
            u128 ej = j < nh ? S.hkey[swz(j)] : (u128)0;
            u128 di = i < nl ? S.okey[swz(i)] : D_tot;
            for (uint32_t st = 0; st < steps; ++st) {
                if ((j < B) && (i >= A || ej <= di)) { // heavy j: Q - (D_i - E_j), alias the next heavy (in the tile)
                    const u128 gap = di - ej;
                    if (gap > Q || j + 1 >= nh) bad = true;
                    const uint32_t me = (uint32_t)(tile0 + S.hoff[j]);
                    const uint32_t nx = (uint32_t)(tile0 + S.hoff[min(j + 1, nh - 1)]);
                    const uint32_t alias = gap == 0 ? me : nx;
                    const uint64_t thr = lo64((Q - gap) >> shift);
                    table[me] = make_uint4((uint32_t)thr, (uint32_t)(thr >> 32), alias, 0u);
                    ++j;
                    if (j < nh) ej = S.hkey[swz(j)];
                } else { // light i: its own weight, alias the current heavy
                    const u128 dn = i + 1 < nl ? S.okey[swz(i + 1)] : D_tot;
                    const u128 nq = Q - (dn - di);
                    const uint32_t me = (uint32_t)(tile0 + S.ooff[i]);
                    uint32_t alias = me;
                    if (nq != Q) {
                        if (j < nh) alias = (uint32_t)(tile0 + S.hoff[j]);
                        else bad = true;
                    }
                    const uint64_t thr = lo64(nq >> shift);
                    table[me] = make_uint4((uint32_t)thr, (uint32_t)(thr >> 32), alias, 0u);
                    ++i;
                    di = dn;
                }
            }
        }
    }
    // the leftovers, in index order: lights of rank >= A, heavies of rank >= B
    uint32_t left = 0;
    {
        uint32_t lr = l0, hr = h0;
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            if ((lmask >> k) & 1u) { if (lr >= A) left |= 1u << k; ++lr; }
            else if ((hmask >> k) & 1u) { if (hr >= B) left |= 1u << k; ++hr; }
        }
    }
    uint32_t ntot;
    uint32_t slot = block_exclusive_scan_u32((uint32_t)__popc(left), ntot, S.cnt);
    {
        uint32_t hr = h0;
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const bool is_h = (hmask >> k) & 1u;
            if ((left >> k) & 1u) {
                const u128 v = (is_h && hr == B) ? s_res : nq_of(x[k], F32, beta, n32);
                lo_v[2 * (tile0 + slot)] = lo64(v);
                lo_v[2 * (tile0 + slot) + 1] = hi64(v);
                lo_idx[tile0 + slot] = (uint32_t)(first + k);
                ++slot;
            }
            if (is_h) ++hr;
        }
    }
    if (threadIdx.x == 0) {
        TileSum a;
        a.l_lo = a.l_hi = a.h_lo = a.h_hi = 0;
        a.cl = ntot; a.nheavy = 0; a.first_heavy = kNone; a.pad = 0;
        tilesum_st(cnt_agg + blockIdx.x, a);
        atomicAdd(reinterpret_cast<unsigned long long *>(&hdr->n_light), (unsigned long long)nl);
    }
    if (bad) set_status(hdr, kEInternal);
}

// -------------------------------------------------------- compaction
// Tile t's leftovers (cnt_incl: inclusive prefix of the tiles' leftover
// counts) move to [prefix before t, prefix through t) of the compacted list.
__global__ void __launch_bounds__(kThreads) k_pp_compact(const uint64_t *__restrict__ lo_v,
                                                         const uint32_t *__restrict__ lo_idx,
                                                         const TileSum *__restrict__ cnt_incl,
                                                         uint64_t *__restrict__ cv, uint32_t *__restrict__ cidx,
                                                         const DevHeader *hdr)
{
    if (*(volatile const uint32_t *)&hdr->status) return;
    const uint32_t t = blockIdx.x;
    const uint32_t end = tilesum_ldcg(cnt_incl + t).cl;
    const uint32_t beg = t ? tilesum_ldcg(cnt_incl + t - 1).cl : 0u;
    const uint64_t src = (uint64_t)t * kTile;
    const uint4 *sv = reinterpret_cast<const uint4 *>(lo_v) + src;
    uint4 *dv = reinterpret_cast<uint4 *>(cv) + beg;
    for (uint32_t i = threadIdx.x; i < end - beg; i += kThreads) {
        dv[i] = __ldcs(sv + i);
        cidx[beg + i] = __ldcs(lo_idx + src + i);
    }
}

// Sets the leftover count m (from the scan of the tile counts) and rearms
// the look-back scan's dynamic tile ids.
__global__ void k_pp_reset(DevHeader *hdr, uint32_t *m_ptr, const TileSum *cnt_incl, uint32_t ntiles)
{
    if (threadIdx.x == 0) {
        hdr->tile_counter = 0;
        *m_ptr = tilesum_ldcg(cnt_incl + (ntiles - 1)).cl;
    }
}

// ------------------------------------------------------------ phase 2
// Per tile of 2048 of the compacted list: its light count and the sums of
// its lights' deficits Q - v and of its heavies' excesses v - Q (light iff
// v <= Q).  Tiles past the list write zeros, so the scan's last inclusive
// prefix holds the totals.
__global__ void __launch_bounds__(kThreads) k_pp_tiles(const uint64_t *__restrict__ cv, const uint32_t *m_ptr,
                                                       const DevHeader *hdr, TileSum *__restrict__ agg)
{
    __shared__ U2 s_scan[kWarps];
    __shared__ uint32_t s_cnt[kWarps];
    if (block_stopped(hdr)) return;
    const uint32_t m = *m_ptr;
    const uint64_t t0 = (uint64_t)blockIdx.x * kTile;
    const u128 Q = mk128(hdr->q_lo, hdr->q_hi);
    const uint4 *v4 = reinterpret_cast<const uint4 *>(cv);
    u128 sd = 0, se = 0;
    uint32_t cl = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const uint64_t i = t0 + (uint64_t)k * kThreads + threadIdx.x; // order is irrelevant for sums
        if (i < m) {
            const uint4 r = __ldg(v4 + i);
            const u128 v = mk128(r.x | ((uint64_t)r.y << 32), r.z | ((uint64_t)r.w << 32));
            if (v <= Q) { sd += Q - v; ++cl; } else se += v - Q;
        }
    }
    U2 tot;
    block_exclusive_scan2(U2{sd, se}, tot, s_scan);
    uint32_t ctot;
    block_exclusive_scan_u32(cl, ctot, s_cnt);
    if (threadIdx.x == 0) {
        TileSum a;
        a.l_lo = lo64(tot.a); a.l_hi = hi64(tot.a); a.h_lo = lo64(tot.b); a.h_hi = hi64(tot.b);
        a.cl = ctot; a.nheavy = 0; a.first_heavy = kNone; a.pad = 0;
        tilesum_st(agg + blockIdx.x, a);
    }
}

// Global keys of the leftovers, written once: the light of rank x at
// keys[x] with D = the deficits of the lights before it, the heavy of rank y
// at keys[NL + y] with E = the excesses of the heavies up to it (NL = the
// light count), each key's item index beside it in kidx.
__global__ void __launch_bounds__(kThreads) k_pp_keys(const uint64_t *__restrict__ cv,
                                                      const uint32_t *__restrict__ cidx, const uint32_t *m_ptr,
                                                      const DevHeader *hdr, const TileSum *__restrict__ incl,
                                                      uint32_t ntiles, uint64_t *__restrict__ keys,
                                                      uint32_t *__restrict__ kidx)
{
    __shared__ U2 s_scan[kWarps];
    __shared__ uint32_t s_cnt[kWarps];
    if (block_stopped(hdr)) return;
    const uint32_t m = *m_ptr;
    const uint64_t t0 = (uint64_t)blockIdx.x * kTile;
    if (t0 >= m) return;
    const u128 Q = mk128(hdr->q_lo, hdr->q_hi);
    const uint32_t NL = tilesum_ldcg(incl + (ntiles - 1)).cl;
    const TileSum before = load_prefix(incl, blockIdx.x);
    const uint32_t heavies_before = (uint32_t)t0 - before.cl;
    const uint64_t first = t0 + (uint64_t)threadIdx.x * kItems;
    const uint4 *v4 = reinterpret_cast<const uint4 *>(cv);
    u128 v[kItems];
    u128 sd = 0, se = 0;
    uint32_t cl = 0, ch = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        v[k] = 0;
        if (first + k < m) {
            const uint4 r = __ldg(v4 + first + k);
            v[k] = mk128(r.x | ((uint64_t)r.y << 32), r.z | ((uint64_t)r.w << 32));
            if (v[k] <= Q) { sd += Q - v[k]; ++cl; } else { se += v[k] - Q; ++ch; }
        }
    }
    U2 tot;
    const U2 ex = block_exclusive_scan2(U2{sd, se}, tot, s_scan);
    uint32_t ctot;
    const uint32_t cex = block_exclusive_scan_u32(cl | (ch << 16), ctot, s_cnt);
    u128 D = mk128(before.l_lo, before.l_hi) + ex.a, E = mk128(before.h_lo, before.h_hi) + ex.b;
    uint64_t lr = before.cl + (cex & 0xFFFFu), hr = (uint64_t)NL + heavies_before + (cex >> 16);
    uint4 *k4 = reinterpret_cast<uint4 *>(keys);
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        if (first + k >= m) continue;
        if (v[k] <= Q) {
            k4[lr] = make_uint4((uint32_t)lo64(D), (uint32_t)(lo64(D) >> 32), (uint32_t)hi64(D),
                                (uint32_t)(hi64(D) >> 32));
            kidx[lr] = cidx[first + k];
            D += Q - v[k];
            ++lr;
        } else {
            E += v[k] - Q;
            k4[hr] = make_uint4((uint32_t)lo64(E), (uint32_t)(lo64(E) >> 32), (uint32_t)hi64(E),
                                (uint32_t)(hi64(E) >> 32));
            kidx[hr] = cidx[first + k];
            ++hr;
        }
    }
}

__device__ __forceinline__ u128 pp_key(const uint64_t *keys, uint64_t i)
{
    const uint4 r = __ldcg(reinterpret_cast<const uint4 *>(keys) + i);
    return mk128(r.x | ((uint64_t)r.y << 32), r.z | ((uint64_t)r.w << 32));
}

struct PpSmem {
    u128 lkey[kTile + 8];   // keys D of the lights the block may reach (swizzled)
    u128 hkey[kTile + 8];   // keys E of the heavies it may reach (swizzled)
    uint32_t lidx[kTile + 1];
    uint32_t hidx[kTile + 2];
    uint32_t start[2];
};

// Block b walks merge steps [2048 b, 2048 (b + 1)) of the leftovers' lights
// (keys D) and heavies (keys E), a heavy before a light when E <= D: a
// light's bucket is its own v with the current heavy as alias; a heavy's is
// Q - (D_next - E) with D_next the key of the next light, and the next heavy
// as alias (itself when the bucket is full).  The block's first step is
// found by a co-rank search over the global keys, done by one warp: each
// round probes 32 evenly spaced candidates, so a list of m keys takes about
// log_32(m) rounds.
__global__ void __launch_bounds__(kThreads) k_pp_merge(const uint64_t *__restrict__ keys,
                                                       const uint32_t *__restrict__ kidx, const uint32_t *m_ptr,
                                                       DevHeader *hdr, const TileSum *__restrict__ incl,
                                                       uint32_t ntiles, uint4 *__restrict__ table)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PpSmem &S = *reinterpret_cast<PpSmem *>(smem_raw);
    if (block_stopped(hdr)) return;
    const uint32_t m = *m_ptr;
    const uint64_t d_begin = (uint64_t)blockIdx.x * kTile;
    if (d_begin >= m) return;
    const uint32_t steps_total = (uint32_t)min((uint64_t)kTile, (uint64_t)m - d_begin);
    const u128 Q = mk128(hdr->q_lo, hdr->q_hi);
    const uint32_t shift = hdr->shift;
    const TileSum last = tilesum_ldcg(incl + (ntiles - 1));
    const uint32_t NL = last.cl, NH = m - last.cl;
    const u128 D_tot = mk128(last.l_lo, last.l_hi);
    const uint64_t *lkeys = keys, *hkeys = keys + 2 * (uint64_t)NL;
    // co-rank of step d: the number j of heavies among the first d merged
    // items, the largest j in [max(0, d - NL), min(d, NH)] with j = its lower
    // end or heavy j-1 before light d-j (E[j-1] <= D[d-j]); the predicate
    // holds for every j up to the answer and for none after it
    if (threadIdx.x < 32) {
        const uint32_t lane = threadIdx.x;
        const uint64_t d = d_begin;
        uint64_t lo = d > NL ? d - NL : 0, hi = d < NH ? d : NH;
        while (lo < hi) {
            const uint64_t step = (hi - lo + 31) / 32;
            const uint64_t p = lo + 1 + step * lane;
            bool ok = false;
            if (p <= hi) ok = (d - p >= NL) || pp_key(hkeys, p - 1) <= pp_key(lkeys, d - p);
            const uint32_t cnt = (uint32_t)__popc(__ballot_sync(0xFFFFFFFFu, ok));
            if (cnt == 0) break;
            const uint64_t nhi = lo + step * cnt; // the first failing probe, minus one
            lo = lo + 1 + step * (cnt - 1);
            hi = nhi < hi ? nhi : hi;
        }
        if (lane == 0) { S.start[0] = (uint32_t)(d - lo); S.start[1] = (uint32_t)lo; }
    }
    __syncthreads();
    const uint32_t i0 = S.start[0], j0 = S.start[1];
    // the block consumes at most steps_total keys of either kind; one more of
    // each is read as the "next" key
    const uint32_t la = (uint32_t)min((uint64_t)steps_total + 1, (uint64_t)(NL - i0));
    const uint32_t hb = (uint32_t)min((uint64_t)steps_total + 1, (uint64_t)(NH - j0));
    for (uint32_t t = threadIdx.x; t < la; t += kThreads) {
        S.lkey[swz(t)] = pp_key(lkeys, (uint64_t)i0 + t);
        S.lidx[t] = kidx[(uint64_t)i0 + t];
    }
    for (uint32_t t = threadIdx.x; t < hb; t += kThreads) {
        S.hkey[swz(t)] = pp_key(hkeys, (uint64_t)j0 + t);
        S.hidx[t] = kidx[(uint64_t)NL + j0 + t];
    }
    if (threadIdx.x == 0) S.hidx[hb] = ((uint64_t)j0 + hb < NH) ? kidx[(uint64_t)NL + j0 + hb] : kNone;
    __syncthreads();
    // the block's steps, split evenly over the threads by a local co-rank
    // search (light i of the block is global light i0 + i; past the loaded
    // lights there is none left, la = NL - i0 then)
    const uint32_t per = (steps_total + kThreads - 1) / kThreads;
    const uint32_t d0 = threadIdx.x * per;
    bool bad = false;
    if (d0 < steps_total) {
        uint32_t lo = d0 > la ? d0 - la : 0, hi = d0 < hb ? d0 : hb;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (S.hkey[swz(mid - 1)] <= S.lkey[swz(d0 - mid)]) lo = mid; else hi = mid - 1;
        }
        uint32_t j = lo, i = d0 - lo;
        const uint32_t steps = min(per, steps_total - d0);
        for (uint32_t st = 0; st < steps; ++st) {
            const u128 di = i < la ? S.lkey[swz(i)] : D_tot;
            if (j < hb && (i >= la || S.hkey[swz(j)] <= di)) { // heavy j
                const u128 gap = di - S.hkey[swz(j)];
                const uint32_t me = S.hidx[j], nx = S.hidx[j + 1];
                if (gap > Q || (nx == kNone && gap != 0)) bad = true;
                const uint32_t alias = (nx == kNone || gap == 0) ? me : nx;
                const uint64_t thr = lo64((Q - gap) >> shift);
                table[me] = make_uint4((uint32_t)thr, (uint32_t)(thr >> 32), alias, 0u);
                ++j;
            } else { // light i
                if (i >= la) { bad = true; break; }
                const u128 dn = (i + 1 < la) ? S.lkey[swz(i + 1)]
                                             : ((uint64_t)i0 + i + 1 < NL ? pp_key(lkeys, (uint64_t)i0 + i + 1) : D_tot);
                const u128 v = Q - (dn - di);
                const uint32_t me = S.lidx[i];
                uint32_t alias = me;
                if (v != Q) {
                    if ((uint64_t)j0 + j < NH) alias = j < hb ? S.hidx[j] : kidx[(uint64_t)NL + j0 + j];
                    else bad = true;
                }
                const uint64_t thr = lo64(v >> shift);
                table[me] = make_uint4((uint32_t)thr, (uint32_t)(thr >> 32), alias, 0u);
                ++i;
            }
        }
    }
    if (bad) set_status(hdr, kEInternal);
}

} // namespace wrs

// ---------------------------------------------------------------- host
namespace {

bool g_pp_attr_done[64];

wrs_status psa_plus_attributes()
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return WRS_EDEVICE;
    if (g_pp_attr_done[dev]) return WRS_OK;
    const int g = (int)sizeof(GroupSmem), p = (int)sizeof(PpSmem);
    cudaError_t e = cudaFuncSetAttribute(k_pp_local<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, g);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pp_local<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, g);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pp_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, p);
    if (e != cudaSuccess) return WRS_EDEVICE;
    g_pp_attr_done[dev] = true;
    return WRS_OK;
}

// PSA+ scratch of a table, 40 bytes per weight of capacity: the per-tile
// leftovers (value, index), the compacted list (value, index) -- the global
// keys reuse the first pair -- and the leftover count.
struct PpLayout {
    uint64_t lo_v, lo_idx, cv, cidx, m, total;
};

PpLayout pp_layout(uint64_t cap)
{
    PpLayout L;
    uint64_t o = 0;
    L.lo_v = o; o = align_up(o + cap * 16, 256);
    L.lo_idx = o; o = align_up(o + cap * 4, 256);
    L.cv = o; o = align_up(o + cap * 16, 256);
    L.cidx = o; o = align_up(o + cap * 4, 256);
    L.m = o; o = align_up(o + 16, 256);
    L.total = o;
    return L;
}

} // namespace

extern "C" {

wrs_status wrs_table_build_psa_plus(wrs_table *t, const void *d_weights, uint64_t n, wrs_dtype dtype, void *stream)
{
    if (!t || !d_weights || n == 0 || n > t->cap) return WRS_EINVAL;
    if (dtype != WRS_U32 && dtype != WRS_F32) return WRS_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_weights) % 4) != 0) return WRS_EINVAL;
    wrs_status st = psa_plus_attributes();
    if (st != WRS_OK) return st;
    const PpLayout L = pp_layout(t->cap);
    if (!t->pp_ws) {
        cudaError_t e = cudaMalloc(&t->pp_ws, L.total);
        if (e != cudaSuccess) { t->pp_ws = nullptr; return cuda_err(e); }
    }
    uint64_t *lo_v = reinterpret_cast<uint64_t *>(t->pp_ws + L.lo_v);
    uint32_t *lo_idx = reinterpret_cast<uint32_t *>(t->pp_ws + L.lo_idx);
    uint64_t *cv = reinterpret_cast<uint64_t *>(t->pp_ws + L.cv);
    uint32_t *cidx = reinterpret_cast<uint32_t *>(t->pp_ws + L.cidx);
    uint32_t *m = reinterpret_cast<uint32_t *>(t->pp_ws + L.m);

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint32_t *w = static_cast<const uint32_t *>(d_weights);
    const int vec = (reinterpret_cast<uintptr_t>(w) % 16) == 0;
    const uint32_t f32 = dtype == WRS_F32;
    const uint32_t ntiles = (uint32_t)((n + kTile - 1) / kTile);
    const uint32_t nchunks = (ntiles + kScanChunk - 1) / kScanChunk;
    uint64_t want = (n + (uint64_t)kThreads * 16 - 1) / ((uint64_t)kThreads * 16);
    uint32_t nparts = (uint32_t)(want < 1 ? 1 : (want > kMaxParts ? kMaxParts : want));
    const uint32_t blocks_cap = (uint32_t)sm_count() * 8;
    if (nparts > blocks_cap) nparts = blocks_cap;
    const uint32_t wait_limit = g_wait_limit.load();
    uint32_t epoch[2];
    for (int i = 0; i < 2; ++i) {
        t->epoch = t->epoch + 1;
        if (t->epoch >= (1u << 30)) t->epoch = 1;
        epoch[i] = t->epoch;
    }

    // Q, beta, light_max (the weight-total pass of PSA)
    if (f32) k_stats<1><<<nparts, kThreads, 0, s>>>(w, n, vec, t->part);
    else k_stats<0><<<nparts, kThreads, 0, s>>>(w, n, vec, t->part);
    k_stats_combine<<<1, kThreads, 0, s>>>(t->part, nparts, n, f32, t->hdr);
    // phase 1: greedy per tile; leftover counts into agg
    if (f32) k_pp_local<1><<<ntiles, kThreads, sizeof(GroupSmem), s>>>(w, n, vec, t->hdr, t->buckets, lo_v, lo_idx, t->agg);
    else k_pp_local<0><<<ntiles, kThreads, sizeof(GroupSmem), s>>>(w, n, vec, t->hdr, t->buckets, lo_v, lo_idx, t->agg);
    k_tilescan<<<nchunks, kThreads, 0, s>>>(t->hdr, t->agg, t->cagg, t->cincl, t->incl, t->flags, ntiles, epoch[0],
                                            wait_limit, kNone);
    k_pp_compact<<<ntiles, kThreads, 0, s>>>(lo_v, lo_idx, t->incl, cv, cidx, t->hdr);
    k_pp_reset<<<1, 32, 0, s>>>(t->hdr, m, t->incl, ntiles);
    // phase 2: Alg. 2 on the leftovers (their keys overwrite lo_v / lo_idx)
    k_pp_tiles<<<ntiles, kThreads, 0, s>>>(cv, m, t->hdr, t->agg);
    k_tilescan<<<nchunks, kThreads, 0, s>>>(t->hdr, t->agg, t->cagg, t->cincl, t->incl, t->flags, ntiles, epoch[1],
                                            wait_limit, kNone);
    k_pp_keys<<<ntiles, kThreads, 0, s>>>(cv, cidx, m, t->hdr, t->incl, ntiles, lo_v, lo_idx);
    k_pp_merge<<<ntiles, kThreads, sizeof(PpSmem), s>>>(lo_v, lo_idx, m, t->hdr, t->incl, ntiles, t->buckets);
    st = launch_err();
    if (st == WRS_OK) {
        t->n = n;
        t->host_status = -1;
        t->timed_build = 0;
        t->pp_n = n;
    }
    return st;
}

wrs_status wrs_table_psa_plus_leftovers(const wrs_table *t, uint64_t *n_left)
{
    if (!t || !n_left || !t->pp_ws || t->pp_n == 0 || t->pp_n != t->n) return WRS_EINVAL;
    const PpLayout L = pp_layout(t->cap);
    uint32_t m = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&m, t->pp_ws + L.m, sizeof(m), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(e);
    *n_left = m;
    return WRS_OK;
}

} // extern "C"
