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
// k_pp_local (one block per tile): the tile's light keys D (prefix of
// deficits Q - n q) and heavy keys E (prefix of excesses n q - Q), local to
// the tile; with D_tot the tile's total deficit and E_last its last heavy key,
// either the lights run out first (E_last > D_tot: every light is packed, the
// heavies with E <= D_tot are packed, the next one stops with its residual)
// or the last heavy is covered first (the lights with D < E_last are packed,
// every heavy but the last, which stops).  The packed items are one merge, as
// in the single table's sweep.  The leftovers get keys local to the tile
// (light iff v <= Q; deficits Q - v, excesses v - Q) in the tile's staging
// slots, and the tile's sums and counts.  k_pp_scan1/k_pp_scan2 scan those
// over the tiles, k_pp_keys adds the prefixes and moves every key to its
// global rank (lights, then heavies), k_pp_starts finds where each block of
// merge steps begins (co-rank search, one warp per block), and k_pp_merge
// walks them.
#pragma once

namespace wrs {

// Leftover sums of tiles: l = deficits of the lights (v <= Q), h = excesses
// of the heavies, cl / nheavy = their counts (TileSum's fields).
__device__ __forceinline__ void pp_add(TileSum &a, const TileSum &b)
{
    const u128 l = mk128(a.l_lo, a.l_hi) + mk128(b.l_lo, b.l_hi);
    const u128 h = mk128(a.h_lo, a.h_hi) + mk128(b.h_lo, b.h_hi);
    a.l_lo = lo64(l); a.l_hi = hi64(l); a.h_lo = lo64(h); a.h_hi = hi64(h);
    a.cl += b.cl;
    a.nheavy += b.nheavy;
}

__device__ __forceinline__ TileSum pp_zero()
{
    TileSum z;
    z.l_lo = z.l_hi = z.h_lo = z.h_hi = 0;
    z.cl = 0; z.nheavy = 0; z.first_heavy = kNone; z.pad = 0;
    return z;
}

__device__ __forceinline__ void st_key(uint4 *p, u128 k)
{
    *p = make_uint4((uint32_t)lo64(k), (uint32_t)(lo64(k) >> 32), (uint32_t)hi64(k), (uint32_t)(hi64(k) >> 32));
}

__device__ __forceinline__ u128 ld_key(const uint4 *p)
{
    const uint4 r = __ldcg(p);
    return mk128(r.x | ((uint64_t)r.y << 32), r.z | ((uint64_t)r.w << 32));
}

// ------------------------------------------------------------ phase 1
template <int F32>
__global__ void __launch_bounds__(kThreads, 3) k_pp_local(const uint32_t *__restrict__ w, uint64_t n, int vec,
                                                          DevHeader *hdr, uint4 *__restrict__ table,
                                                          TileSum *__restrict__ tsum, uint4 *__restrict__ skeys,
                                                          uint32_t *__restrict__ sidx)
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
    const uint32_t tile = blockIdx.x;
    const uint64_t tile0 = (uint64_t)tile * kTile;
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
    // The leftovers: lights of rank >= A, heavies of rank > B, and heavy B
    // (when there is one) with its residual; in the second phase an item is
    // light iff its value v <= Q.  Their sums and their keys local to the
    // tile follow from the tile's own keys: the leftover lights' deficits are
    // D - D_A, the leftover heavies' excesses E - E_B, and heavy B adds
    // Q - res to the lights after it or res - Q before the heavies.
    const bool hasB = B < nh;
    const u128 res = hasB ? s_res : (u128)0;
    const bool Bl = hasB && res <= Q, Bh = hasB && res > Q;
    const uint32_t offB = hasB ? S.hoff[B] : 0xFFFFFFFFu;
    const u128 DA = A < nl ? S.okey[swz(A)] : D_tot;
    const u128 EB = hasB ? S.hkey[swz(B)] : (u128)0;
    const uint32_t ncl = (nl - A) + (Bl ? 1u : 0u);
    const uint32_t nch = hasB ? (nh - B - 1) + (Bh ? 1u : 0u) : 0u;
    if (threadIdx.x == 0) {
        const u128 lsum = (D_tot - DA) + (Bl ? Q - res : (u128)0);
        const u128 hsum = hasB ? (S.hkey[swz(nh - 1)] - EB) + (Bh ? res - Q : (u128)0) : (u128)0;
        TileSum a;
        a.l_lo = lo64(lsum); a.l_hi = hi64(lsum); a.h_lo = lo64(hsum); a.h_hi = hi64(hsum);
        a.cl = ncl; a.nheavy = nch; a.first_heavy = kNone; a.pad = 0;
        tilesum_st(tsum + tile, a);
        atomicAdd(reinterpret_cast<unsigned long long *>(&hdr->n_light), (unsigned long long)nl);
    }
    // the packed items, lights [0, A) and heavies [0, B), as one merge
    const uint32_t M = A + B;
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
                put_bucket(table, me, thr, alias, n, hdr);
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
                put_bucket(table, me, thr, alias, n, hdr);
                ++i;
                di = dn;
            }
        }
    }
    // the leftovers' keys local to the tile, in its staging slots: lights
    // first (D = deficits of the tile's leftover lights before), then heavies
    // (E = excesses up to and including)
    {
        uint32_t lr = l0, hr = h0;
        const uint64_t hbase = tile0 + ncl;
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const uint32_t off = threadIdx.x * kItems + k;
            if ((lmask >> k) & 1u) {
                if (lr >= A) {
                    const bool after = Bl && offB < off;
                    const uint64_t pos = tile0 + (lr - A) + (after ? 1u : 0u);
                    st_key(skeys + pos, S.okey[swz(lr)] - DA + (after ? Q - res : (u128)0));
                    sidx[pos] = (uint32_t)(first + k);
                }
                ++lr;
            } else if ((hmask >> k) & 1u) {
                if (hr == B) {
                    if (Bl) { // lr = the lights before it
                        const u128 Dk = lr < nl ? S.okey[swz(lr)] : D_tot;
                        const uint64_t pos = tile0 + (lr > A ? lr - A : 0u);
                        st_key(skeys + pos, lr > A ? Dk - DA : (u128)0);
                        sidx[pos] = (uint32_t)(first + k);
                    } else {
                        st_key(skeys + hbase, res - Q);
                        sidx[hbase] = (uint32_t)(first + k);
                    }
                } else if (hr > B) {
                    const uint64_t pos = hbase + (hr - B - 1) + (Bh ? 1u : 0u);
                    st_key(skeys + pos, S.hkey[swz(hr)] - EB + (Bh ? res - Q : (u128)0));
                    sidx[pos] = (uint32_t)(first + k);
                }
                ++hr;
            }
        }
    }
    if (bad) set_status(hdr, kEInternal);
}

// ------------------------------------------------------- tile scan
// Exclusive prefix of the tiles' leftover sums and counts, in two levels:
// k_pp_scan1 scans 2048 tiles per block (tpre[t] = prefix within the block,
// bsum[b] = the block's total); k_pp_scan2 (one block) turns bsum into
// exclusive block prefixes and writes the grand total to tot.  n < 2^32
// gives at most 2^21 tiles, so at most 1024 blocks.
__device__ __forceinline__ void pp_scan_block(TileSum (&v)[kItems], TileSum &total)
{
    __shared__ U2 s_scan[kWarps];
    __shared__ uint32_t s_c1[kWarps], s_c2[kWarps];
    TileSum sum = pp_zero();
#pragma unroll
    for (int k = 0; k < kItems; ++k) pp_add(sum, v[k]);
    U2 tot;
    const U2 ex = block_exclusive_scan2(U2{mk128(sum.l_lo, sum.l_hi), mk128(sum.h_lo, sum.h_hi)}, tot, s_scan);
    uint32_t t1, t2;
    const uint32_t e1 = block_exclusive_scan_u32(sum.cl, t1, s_c1);
    const uint32_t e2 = block_exclusive_scan_u32(sum.nheavy, t2, s_c2);
    TileSum run;
    run.l_lo = lo64(ex.a); run.l_hi = hi64(ex.a); run.h_lo = lo64(ex.b); run.h_hi = hi64(ex.b);
    run.cl = e1; run.nheavy = e2; run.first_heavy = kNone; run.pad = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) { // v[k] becomes its exclusive prefix
        const TileSum own = v[k];
        v[k] = run;
        pp_add(run, own);
    }
    total.l_lo = lo64(tot.a); total.l_hi = hi64(tot.a); total.h_lo = lo64(tot.b); total.h_hi = hi64(tot.b);
    total.cl = t1; total.nheavy = t2; total.first_heavy = kNone; total.pad = 0;
}

__global__ void __launch_bounds__(kThreads) k_pp_scan1(const TileSum *__restrict__ tsum, uint32_t ntiles,
                                                       const DevHeader *hdr, TileSum *__restrict__ tpre,
                                                       TileSum *__restrict__ bsum)
{
    if (block_stopped(hdr)) return;
    const uint64_t t0 = (uint64_t)blockIdx.x * kTile + (uint64_t)threadIdx.x * kItems;
    TileSum v[kItems];
#pragma unroll
    for (int k = 0; k < kItems; ++k) v[k] = t0 + k < ntiles ? tilesum_ldcg(tsum + t0 + k) : pp_zero();
    TileSum total;
    pp_scan_block(v, total);
#pragma unroll
    for (int k = 0; k < kItems; ++k)
        if (t0 + k < ntiles) tilesum_st(tpre + t0 + k, v[k]);
    if (threadIdx.x == 0) tilesum_st(bsum + blockIdx.x, total);
}

__global__ void __launch_bounds__(kThreads) k_pp_scan2(TileSum *bsum, uint32_t nblocks, const DevHeader *hdr,
                                                       TileSum *tot, uint32_t *m_out)
{
    if (block_stopped(hdr)) return;
    const uint32_t b0 = threadIdx.x * kItems;
    TileSum v[kItems];
#pragma unroll
    for (int k = 0; k < kItems; ++k) v[k] = b0 + k < nblocks ? tilesum_ldcg(bsum + b0 + k) : pp_zero();
    TileSum total;
    pp_scan_block(v, total);
#pragma unroll
    for (int k = 0; k < kItems; ++k)
        if (b0 + k < nblocks) tilesum_st(bsum + b0 + k, v[k]);
    if (threadIdx.x == 0) {
        tilesum_st(tot, total);
        *m_out = total.cl + total.nheavy;
    }
}

// Tile t's staged keys plus the prefixes before the tile, moved to their
// global ranks: light x of the tile to keys[L_before + x], heavy y to
// keys[NL + H_before + y].  One warp per tile; coalesced on both sides.
__global__ void __launch_bounds__(kThreads) k_pp_keys(const uint4 *__restrict__ skeys,
                                                      const uint32_t *__restrict__ sidx,
                                                      const TileSum *__restrict__ tsum,
                                                      const TileSum *__restrict__ tpre,
                                                      const TileSum *__restrict__ bsum, const TileSum *tot,
                                                      uint32_t ntiles, const DevHeader *hdr,
                                                      uint4 *__restrict__ keys, uint32_t *__restrict__ kidx)
{
    if (*(volatile const uint32_t *)&hdr->status) return; // no barrier in this kernel
    const uint32_t t = blockIdx.x * kWarps + (threadIdx.x >> 5);
    if (t >= ntiles) return;
    const uint32_t lane = threadIdx.x & 31;
    const TileSum own = tilesum_ldcg(tsum + t);
    const uint32_t cnt = own.cl + own.nheavy;
    if (cnt == 0) return;
    TileSum pre = tilesum_ldcg(bsum + t / kTile);
    pp_add(pre, tilesum_ldcg(tpre + t));
    const uint32_t NL = tilesum_ldcg(tot).cl;
    const u128 D0 = mk128(pre.l_lo, pre.l_hi), E0 = mk128(pre.h_lo, pre.h_hi);
    const uint64_t src = (uint64_t)t * kTile;
    for (uint32_t x = lane; x < cnt; x += 32) {
        const u128 k = ld_key(skeys + src + x);
        const uint32_t idx = __ldcs(sidx + src + x);
        uint64_t dst;
        u128 key;
        if (x < own.cl) { dst = (uint64_t)pre.cl + x; key = D0 + k; }
        else { dst = (uint64_t)NL + pre.nheavy + (x - own.cl); key = E0 + k; }
        st_key(keys + dst, key);
        kidx[dst] = idx;
    }
}

// ------------------------------------------------------------ phase 2
// Totals of the leftovers: NL lights, NH heavies, D_tot deficits.
struct PpTotals {
    uint32_t NL, NH;
    u128 D_tot;
};

__device__ __forceinline__ PpTotals pp_totals(const TileSum *tot)
{
    const TileSum last = tilesum_ldcg(tot);
    PpTotals t;
    t.NL = last.cl;
    t.NH = last.nheavy;
    t.D_tot = mk128(last.l_lo, last.l_hi);
    return t;
}

constexpr uint32_t kMergeSteps = 1024; // merge steps per block of k_pp_merge

// Where merge block b starts: the number j of heavies among the first d =
// 1024 b merged items, the largest j in [max(0, d - NL), min(d, NH)] that is
// its lower end or has heavy j-1 before light d-j (E[j-1] <= D[d-j]).  The
// predicate holds for every j up to the answer and for none after it.  One
// warp per block: each round probes 32 evenly spaced candidates, so m keys
// take about log_32(m) rounds.  starts[b] = (lights, heavies) before it.
__global__ void __launch_bounds__(kThreads) k_pp_starts(const uint4 *__restrict__ keys, const DevHeader *hdr,
                                                        const TileSum *tot, uint2 *__restrict__ starts)
{
    if (*(volatile const uint32_t *)&hdr->status) return; // no barrier in this kernel
    const PpTotals T = pp_totals(tot);
    const uint64_t m = (uint64_t)T.NL + T.NH;
    const uint4 *lkeys = keys, *hkeys = keys + T.NL;
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t b = (uint64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const uint64_t d = b * kMergeSteps;
    if (d >= m) return;
    uint64_t lo = d > T.NL ? d - T.NL : 0, hi = d < T.NH ? d : T.NH;
    while (lo < hi) {
        const uint64_t step = (hi - lo + 31) / 32;
        const uint64_t p = lo + 1 + step * lane;
        bool ok = false;
        if (p <= hi) ok = (d - p >= T.NL) || ld_key(hkeys + (p - 1)) <= ld_key(lkeys + (d - p));
        const uint32_t cnt = (uint32_t)__popc(__ballot_sync(0xFFFFFFFFu, ok));
        if (cnt == 0) break;
        const uint64_t nhi = lo + step * cnt; // the first failing probe, minus one
        lo = lo + 1 + step * (cnt - 1);
        hi = nhi < hi ? nhi : hi;
    }
    if (lane == 0) starts[b] = make_uint2((uint32_t)(d - lo), (uint32_t)lo);
}

struct PpSmem {
    u128 lkey[kMergeSteps + 8];   // keys D of the lights the block may reach (swizzled)
    u128 hkey[kMergeSteps + 8];   // keys E of the heavies it may reach (swizzled)
    uint32_t lidx[kMergeSteps + 1];
    uint32_t hidx[kMergeSteps + 2];
};

// Block b walks merge steps [1024 b, 1024 (b + 1)) of the leftovers' lights
// (keys D) and heavies (keys E), a heavy before a light when E <= D: a
// light's bucket is its own v with the current heavy as alias; a heavy's is
// Q - (D_next - E) with D_next the key of the next light, and the next heavy
// as alias (itself when the bucket is full).
__global__ void __launch_bounds__(kThreads) k_pp_merge(const uint4 *__restrict__ keys,
                                                       const uint32_t *__restrict__ kidx, DevHeader *hdr,
                                                       const TileSum *tot, const uint2 *__restrict__ starts,
                                                       uint4 *__restrict__ table)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PpSmem &S = *reinterpret_cast<PpSmem *>(smem_raw);
    if (block_stopped(hdr)) return;
    const PpTotals T = pp_totals(tot);
    const uint64_t m = (uint64_t)T.NL + T.NH;
    const uint64_t d_begin = (uint64_t)blockIdx.x * kMergeSteps;
    if (d_begin >= m) return;
    const uint4 *lkeys = keys, *hkeys = keys + T.NL;
    const uint32_t *lidx = kidx, *hidx = kidx + T.NL;
    const uint32_t steps_total = (uint32_t)min((uint64_t)kMergeSteps, m - d_begin);
    const u128 Q = mk128(hdr->q_lo, hdr->q_hi);
    const uint32_t shift = hdr->shift;
    const uint2 st0 = starts[blockIdx.x];
    const uint32_t i0 = st0.x, j0 = st0.y;
    // the block consumes the keys up to the next block's start; one more of
    // each kind is read as the "next" key
    uint32_t i1 = T.NL, j1 = T.NH;
    if (d_begin + kMergeSteps < m) {
        const uint2 st1 = starts[blockIdx.x + 1];
        i1 = st1.x;
        j1 = st1.y;
    }
    const uint32_t la = min(i1 - i0 + 1, T.NL - i0);
    const uint32_t hb = min(j1 - j0 + 1, T.NH - j0);
    for (uint32_t t = threadIdx.x; t < la; t += kThreads) {
        S.lkey[swz(t)] = ld_key(lkeys + (uint64_t)i0 + t);
        S.lidx[t] = lidx[(uint64_t)i0 + t];
    }
    for (uint32_t t = threadIdx.x; t < hb; t += kThreads) {
        S.hkey[swz(t)] = ld_key(hkeys + (uint64_t)j0 + t);
        S.hidx[t] = hidx[(uint64_t)j0 + t];
    }
    if (threadIdx.x == 0) S.hidx[hb] = ((uint64_t)j0 + hb < T.NH) ? hidx[(uint64_t)j0 + hb] : kNone;
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
            const u128 di = i < la ? S.lkey[swz(i)] : T.D_tot;
            if (j < hb && (i >= la || S.hkey[swz(j)] <= di)) { // heavy j
                const u128 gap = di - S.hkey[swz(j)];
                const uint32_t me = S.hidx[j], nx = S.hidx[j + 1];
                if (gap > Q || (nx == kNone && gap != 0)) bad = true;
                const uint32_t alias = (nx == kNone || gap == 0) ? me : nx;
                const uint64_t thr = lo64((Q - gap) >> shift);
                put_bucket(table, me, thr, alias, hdr->n, hdr);
                ++j;
            } else { // light i
                if (i >= la) { bad = true; break; }
                const u128 dn = (i + 1 < la) ? S.lkey[swz(i + 1)]
                                             : ((uint64_t)i0 + i + 1 < T.NL ? ld_key(lkeys + (uint64_t)i0 + i + 1)
                                                                            : T.D_tot);
                const u128 v = Q - (dn - di);
                const uint32_t me = S.lidx[i];
                uint32_t alias = me;
                if (v != Q) {
                    if ((uint64_t)j0 + j < T.NH) alias = j < hb ? S.hidx[j] : hidx[(uint64_t)j0 + j];
                    else bad = true;
                }
                const uint64_t thr = lo64(v >> shift);
                put_bucket(table, me, thr, alias, hdr->n, hdr);
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

// PSA+ scratch of a table, about 40 bytes per weight of capacity: staged
// keys and item indices of the leftovers (tile by tile), the same at their
// global ranks, per-tile leftover sums and their prefixes, block sums, the
// totals, merge-block starts and the leftover count.
struct PpLayout {
    uint64_t skeys, sidx, keys, kidx, tsum, tpre, bsum, tot, starts, m, total;
};

PpLayout pp_layout(uint64_t cap)
{
    const uint64_t ntiles = (cap + kTile - 1) / kTile;
    const uint64_t nblocks = (ntiles + kTile - 1) / kTile;
    const uint64_t nmerge = (cap + kMergeSteps - 1) / kMergeSteps;
    PpLayout L;
    uint64_t o = 0;
    L.skeys = o; o = align_up(o + ntiles * kTile * 16, 256);
    L.sidx = o; o = align_up(o + ntiles * kTile * 4, 256);
    L.keys = o; o = align_up(o + cap * 16, 256);
    L.kidx = o; o = align_up(o + cap * 4, 256);
    L.tsum = o; o = align_up(o + ntiles * sizeof(TileSum), 256);
    L.tpre = o; o = align_up(o + ntiles * sizeof(TileSum), 256);
    L.bsum = o; o = align_up(o + nblocks * sizeof(TileSum), 256);
    L.tot = o; o = align_up(o + sizeof(TileSum), 256);
    L.starts = o; o = align_up(o + nmerge * sizeof(uint2), 256);
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
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&t->pp_ws), L.total,
                                        static_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) {
            t->pp_ws = nullptr;
            return cuda_err(e);
        }
    }
    uint8_t *ws = t->pp_ws;
    uint4 *skeys = reinterpret_cast<uint4 *>(ws + L.skeys);
    uint32_t *sidx = reinterpret_cast<uint32_t *>(ws + L.sidx);
    uint4 *keys = reinterpret_cast<uint4 *>(ws + L.keys);
    uint32_t *kidx = reinterpret_cast<uint32_t *>(ws + L.kidx);
    TileSum *tsum = reinterpret_cast<TileSum *>(ws + L.tsum);
    TileSum *tpre = reinterpret_cast<TileSum *>(ws + L.tpre);
    TileSum *bsum = reinterpret_cast<TileSum *>(ws + L.bsum);
    TileSum *tot = reinterpret_cast<TileSum *>(ws + L.tot);
    uint2 *starts = reinterpret_cast<uint2 *>(ws + L.starts);
    uint32_t *m = reinterpret_cast<uint32_t *>(ws + L.m);

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint32_t *w = static_cast<const uint32_t *>(d_weights);
    const int vec = (reinterpret_cast<uintptr_t>(w) % 16) == 0;
    const uint32_t f32 = dtype == WRS_F32;
    const uint32_t ntiles = (uint32_t)((n + kTile - 1) / kTile);
    const uint32_t nblocks = (ntiles + kTile - 1) / kTile;
    const uint32_t nmerge = (uint32_t)((n + kMergeSteps - 1) / kMergeSteps);
    uint64_t want = (n + (uint64_t)kThreads * 16 - 1) / ((uint64_t)kThreads * 16);
    uint32_t nparts = (uint32_t)(want < 1 ? 1 : (want > kMaxParts ? kMaxParts : want));
    const uint32_t blocks_cap = (uint32_t)sm_count() * 8;
    if (nparts > blocks_cap) nparts = blocks_cap;

    st = check_clear(t->buckets, n, s);
    if (st != WRS_OK) return st;
    // Q, beta, light_max (the weight-total pass of PSA)
    if (f32) k_stats<1><<<nparts, kThreads, 0, s>>>(w, n, vec, t->part);
    else k_stats<0><<<nparts, kThreads, 0, s>>>(w, n, vec, t->part);
    k_stats_combine<<<1, kThreads, 0, s>>>(t->part, nparts, n, f32, t->hdr);
    // phase 1; the leftovers' local keys and per-tile sums
    const size_t gs = sizeof(GroupSmem);
    if (f32) k_pp_local<1><<<ntiles, kThreads, gs, s>>>(w, n, vec, t->hdr, t->buckets, tsum, skeys, sidx);
    else k_pp_local<0><<<ntiles, kThreads, gs, s>>>(w, n, vec, t->hdr, t->buckets, tsum, skeys, sidx);
    // phase 2: Alg. 2 on the leftovers
    k_pp_scan1<<<nblocks, kThreads, 0, s>>>(tsum, ntiles, t->hdr, tpre, bsum);
    k_pp_scan2<<<1, kThreads, 0, s>>>(bsum, nblocks, t->hdr, tot, m);
    k_pp_keys<<<(ntiles + kWarps - 1) / kWarps, kThreads, 0, s>>>(skeys, sidx, tsum, tpre, bsum, tot, ntiles, t->hdr,
                                                                 keys, kidx);
    k_pp_starts<<<(nmerge + kWarps - 1) / kWarps, kThreads, 0, s>>>(keys, t->hdr, tot, starts);
    k_pp_merge<<<nmerge, kThreads, sizeof(PpSmem), s>>>(keys, kidx, t->hdr, tot, starts, t->buckets);
    st = launch_err();
    if (st == WRS_OK) st = log_op(t, s, true);
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
    const wrs_status st = read_back(t, &m, t->pp_ws + L.m, sizeof(m));
    if (st != WRS_OK) return st;
    *n_left = m;
    return WRS_OK;
}

} // extern "C"
