// The binary32-clock window of RL 32-wide ZGB cells per warp with each
// lane's rows held in shared memory: zgbm_window (fskmc_zgb32x4.cuh) with
// the same classes, draws, clock, member numbering and events, so it gives
// the same lattices, but a lane's RL rows (empty and A masks) sit in shared
// memory instead of registers. A row is then reached by an index known only
// at run time for the price of a load, and after each event the lane
// recounts only the row pairs whose members the event changed (at most two)
// instead of all RL / 2, and changes only the rows the event changed.
#pragma once
#include <cuda_runtime.h>

#include "fskmc_device.cuh"
#include "fskmc_internal.h"
#include "fskmc_zgb32.cuh"
#include "fskmc_zgb32x4.cuh"
#include "philox.cuh"

namespace fskmc {

namespace {

// Shared memory per warp: the RL cells' constants, each lane's bond masks of
// the two pair classes per row pair ({H0, H1, V0, V1}), and each lane's RL
// rows ({empty, A} per row).
__host__ __device__ constexpr int zgbs_warp_smem(int RL)
{
    return RL * (int)sizeof(Zgb32Const) + 2 * 32 * (RL / 2) * 16 + RL * 32 * 8;
}

// The windows of RL cells (zgbm_shape_ok) by one warp, as zgbm_window: group
// g runs the cell at `at` (`valid` false for a group without a cell) of
// replica R in the byte lattice src (== dst), all of the same window. wsm:
// zgbs_warp_smem(RL) bytes of 16-byte aligned shared memory. Returns this
// group's events; *bad_out is set if a rank search found no member (never,
// unless the counts and masks disagree) or a window ran away.
template <int RL, bool PERSIST>
__device__ uint32_t zgbs_window(uint8_t *wsm, const Replica &R, const CellGeom &G, const CellAt &at, bool valid,
                                int colour, uint32_t w, double hwin, uint64_t seed, const uint8_t *src, uint8_t *dst,
                                int lane, bool *bad_out)
{
    static_assert(RL == 4 || RL == 8, "4 or 8 cells per warp");
    constexpr unsigned FULLW = 0xffffffffu;
    constexpr int W = 32 / RL, NP = RL / 2;  // lanes per cell, row pairs per lane
    const int qy = G.qy, nrl = qy / RL;      // lanes holding the cell's rows
    const int l = lane & (W - 1), gb = lane & ~(W - 1);
    const unsigned gmask = ((1u << W) - 1u) << gb;
    const bool ew = colour == 0;
    const bool row = valid && l < nrl, first = l == 0, last = l == nrl - 1;
    Zgb32Const *Cw = reinterpret_cast<Zgb32Const *>(wsm) + lane / W;
    uint4 *bq = reinterpret_cast<uint4 *>(wsm + RL * sizeof(Zgb32Const));  // [class - 1][row pair][lane]
    // [row][lane]: {empty mask, A mask}; lane-contiguous, so a warp's access
    // to one row index per lane is free of bank conflicts whatever the rows
    uint2 *rows = reinterpret_cast<uint2 *>(wsm + RL * sizeof(Zgb32Const) + 2 * 32 * NP * 16);

    // The lane's rows and their halo sites, loaded from global memory and
    // stored to shared memory; local lane 0 also keeps the halo row above the
    // cell, the last row lane the one below (eH, aH). hx: bit r (8 + r) set
    // if row r's left halo site is empty (holds A), bit 16 + r (24 + r) if
    // its right halo site is.
    uint32_t eH = 0u, aH = 0u, hx = 0u;
    {
        uint32_t e[RL], a[RL];
#pragma unroll
        for (int r = 0; r < RL; ++r) { e[r] = 0u; a[r] = 0u; }
        if (row) {
            const int lx = at.lx, ly = at.ly, X0 = at.X0, Y0 = at.Y0;
            const int gxl = X0 > 0 ? X0 - 1 : lx - 1, gxr = X0 + 32 < lx ? X0 + 32 : 0;
#pragma unroll
            for (int r = 0; r < RL; ++r) {
                const uint8_t *p = src + (int64_t)(Y0 + RL * l + r) * lx;
                const uint4 u0 = zgbq_ld16<PERSIST>(p + X0), u1 = zgbq_ld16<PERSIST>(p + X0 + 16);
                const uint8_t sl = ld_site<PERSIST>(p + gxl), sr = ld_site<PERSIST>(p + gxr);
                zgbq_masks(u0, u1, e[r], a[r]);
                hx |= ((uint32_t)(sl == 0) | ((uint32_t)(sl == 1) << 8) | ((uint32_t)(sr == 0) << 16) |
                       ((uint32_t)(sr == 1) << 24)) << r;
            }
            if (first || last) {
                const int hy = first ? (Y0 > 0 ? Y0 - 1 : ly - 1) : (Y0 + qy < ly ? Y0 + qy : 0);
                const uint8_t *p = src + (int64_t)hy * lx + X0;
                zgbq_masks(zgbq_ld16<PERSIST>(p), zgbq_ld16<PERSIST>(p + 16), eH, aH);
            }
        }
#pragma unroll
        for (int r = 0; r < RL; ++r) rows[r * 32 + lane] = make_uint2(e[r], a[r]);
    }
    if (valid && l == 0) {
        Cw->rq[0] = R.rq[0];
        Cw->rq[1] = 2ull * R.rq[1];
        Cw->rq[2] = 2ull * R.rq[2];
        Cw->rq[3] = R.rq[3];
        Cw->seed = seed;
        Cw->dst = dst;
        Cw->qscale = R.qscale;
        Cw->hf = (float)hwin;
        Cw->ctr3 = R.rep | (TAG_EVENT << 24);
        Cw->w = w;
        Cw->m = at.m;
        Cw->X0 = at.X0;
        Cw->Y0 = at.Y0;
        Cw->lx = at.lx;
        Cw->ly = at.ly;
    }
    __syncwarp();
    const volatile Zgb32Const &C = *Cw;

    // The lane's classes. pc: its count of class k in row pair p (each below
    // 256) at bit 8 (NP k + p) % 32 of word NP k / 4; s03, s12: its totals of
    // classes 0 and 3, 1 and 2, packed (each below 2^16); bq: its bond masks
    // per pair; lb1, lb2: its rows' left cross bonds (bit r: row r's); n1,
    // n2: its top-halo bonds (local lane 0). eB, aB: the row below the lane's
    // last row (the next lane's row 0, or the bottom halo row in the last row
    // lane; a group's last lane, if it holds no rows, reads its own).
    uint32_t pc[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) pc[i] = 0u;
    uint32_t s03 = 0u, s12 = 0u, lb1 = 0u, lb2 = 0u, n1 = 0u, n2 = 0u, eB = 0u, aB = 0u;
    auto load_below = [&]() {
        const uint2 v = rows[lane + (l + 1 < W ? 1 : 0)];
        eB = last ? eH : v.x;
        aB = last ? aH : v.y;
    };
    // (Re)count row pair p: its rows 2p, 2p + 1, the row below them and the
    // halo sites of its rows.
    auto pair_update = [&](int p) {
        p &= NP - 1;
        const uint2 r0 = rows[(2 * p) * 32 + lane], r1 = rows[(2 * p + 1) * 32 + lane];
        const uint2 r2 = rows[min(2 * p + 2, RL - 1) * 32 + lane];
        const uint32_t be = p < NP - 1 ? r2.x : eB, ba = p < NP - 1 ? r2.y : aB;
        ZgbmPair B1, B2;
        zgbm_pair_bonds(p == NP - 1 && last, p == 0 && first, ew, r0.x, r0.y, r1.x, r1.y, be, ba, eH, aH,
                        hx >> (16 + 2 * p), hx >> (24 + 2 * p), B1, B2);
        // the rows' left cross bonds (E windows): site 0 and the left halo site
        const uint32_t c0e = (r0.x & 1u) | ((r1.x & 1u) << 1), c0a = (r0.y & 1u) | ((r1.y & 1u) << 1);
        const uint32_t hle = (hx >> (2 * p)) & 3u, hla = (hx >> (8 + 2 * p)) & 3u;
        const uint32_t L1 = ew ? hle & c0e : 0u, L2 = ew ? (hla ^ c0a) & ~(hle | c0e) & 3u : 0u;
        bq[32 * p + lane] = make_uint4(B1.H0, B1.H1, B1.V0, B1.V1);  // lane-contiguous: no bank conflicts
        bq[32 * NP + 32 * p + lane] = make_uint4(B2.H0, B2.H1, B2.V0, B2.V1);
        lb1 = (lb1 & ~(3u << (2 * p))) | (L1 << (2 * p));
        lb2 = (lb2 & ~(3u << (2 * p))) | (L2 << (2 * p));
        uint32_t c1 = __popc(B1.H0) + __popc(B1.H1) + __popc(B1.V0) + __popc(B1.V1) + __popc(L1);
        uint32_t c2 = __popc(B2.H0) + __popc(B2.H1) + __popc(B2.V0) + __popc(B2.V1) + __popc(L2);
        if (p == 0) {  // the top-halo bonds (zero unless local lane 0 in an O window)
            n1 = B1.N;
            n2 = B2.N;
            c1 += __popc(n1);
            c2 += __popc(n2);
        }
        const uint32_t cn[4] = {(uint32_t)(__popc(r0.x) + __popc(r1.x)), c1, c2,
                                (uint32_t)(__popc(r0.y) + __popc(r1.y))};
        uint32_t d[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int wi = k * NP / 4, sh = (8 * (k * NP + p)) % 32;
            d[k] = cn[k] - ((pc[wi] >> sh) & 0xFFu);  // modulo 2^32: the packed sums stay exact
            pc[wi] += d[k] << sh;
        }
        s03 += d[0] + (d[3] << 16);
        s12 += d[1] + (d[2] << 16);
    };
    load_below();
#pragma unroll
    for (int p = 0; p < NP; ++p) pair_update(p);

    float tauf = 0.0f, rlf = 0.0f;
    uint32_t rw2 = 0u, rw3 = 0u, ev = 0u;
    bool live = valid, bad = false;
    while (__any_sync(FULLW, live)) {
        uint32_t n[4];
        {  // the four totals as two packed sums (each below 2^16)
            const uint32_t t03 = __reduce_add_sync(gmask, s03), t12 = __reduce_add_sync(gmask, s12);
            n[0] = t03 & 0xFFFFu; n[3] = t03 >> 16; n[1] = t12 & 0xFFFFu; n[2] = t12 >> 16;
        }
        const uint64_t P0 = (uint64_t)n[0] * C.rq[0], P1 = P0 + (uint64_t)n[1] * C.rq[1];
        const uint64_t P2 = P1 + (uint64_t)n[2] * C.rq[2], lami = P2 + (uint64_t)n[3] * C.rq[3];
        if (lami == 0ull) live = false;
        if (live && ev >= MAX_EVENTS_PER_WINDOW) {
            bad = true;
            live = false;
        }
        if ((ev & (uint32_t)(W - 1)) == 0u && live) {  // W events' draws at once, one Philox block per lane
            const u32x4 o = draw(C.seed, ev + (uint32_t)l, C.w, C.m, C.ctr3);
            rlf = -__logf(__fmul_rn(__uint2float_rn((o.x >> 8) + 1u), 0x1p-24f));
            rw2 = o.z;
            rw3 = o.w;
        }
        const int sl = (int)(ev & (uint32_t)(W - 1));
        const uint32_t w2 = __shfl_sync(FULLW, rw2, sl, W), w3 = __shfl_sync(FULLW, rw3, sl, W);
        // class: the first k with (w2 lambda) >> 32 < P_k (exact integers),
        // member j of it, and this lane's count of that class
        const uint64_t t = (uint64_t)w2 * (lami >> 32) + (((uint64_t)w2 * (lami & 0xffffffffull)) >> 32);
        const int k = t < P0 ? 0 : (t < P1 ? 1 : (t < P2 ? 2 : 3));
        const uint32_t nk = k == 0 ? n[0] : (k == 1 ? n[1] : (k == 2 ? n[2] : n[3]));
        const uint32_t j = (uint32_t)(((uint64_t)w3 * (uint64_t)nk) >> 32);
        const int c = (int)(k == 0 ? s03 & 0xFFFFu : (k == 1 ? s12 & 0xFFFFu : (k == 2 ? s12 >> 16 : s03 >> 16)));
        // the clock: the event happens if it falls within the window
        const float lg = __shfl_sync(FULLW, rlf, sl, W);
        if (live) {
            const float lamf = __fmul_rn(u64_to_float_rz(lami), C.qscale);
            const float end = __fadd_rn(tauf, __fdividef(lg, lamf));
            if (end >= C.hf) live = false;
            else tauf = end;
        }
        if (!__any_sync(FULLW, live)) break;  // every window ended at this draw
        // the owner of member j: a prefix scan of the cell's counts, then the
        // bit in the owner's masks
        int incl = c;
#pragma unroll
        for (int off = 1; off < W; off <<= 1) {
            const int v = __shfl_up_sync(FULLW, incl, off, W);
            if (l >= off) incl += v;
        }
        const uint32_t hit = (__ballot_sync(FULLW, live && (uint32_t)incl > j) & gmask) >> gb;
        if (live && hit == 0u) {
            bad = true;
            live = false;
        }
        const int owner = hit ? __ffs(hit) - 1 : 0;
        // kind: 0 site, 1 horizontal bond, 2 vertical bond between rows rr and
        // rr + 1 of the lane, 3 vertical bond below its last row, 4 left cross
        // bond, 5 top-halo bond; rr: the row of the lane
        int code = 0;
        if (live && l == owner) {
            int r = (int)j - (incl - c);
            // the row pair that holds the lane's member r, from the pair
            // counts, then the member among the pair's entries
            uint32_t pk = 0u;
#pragma unroll
            for (int i = 0; i < NP; ++i)
                if (k * NP / 4 == i) pk = pc[i];
            pk >>= 8 * (k * NP) % 32;
            int p = 0;
#pragma unroll
            for (int q = 0; q < NP - 1; ++q) {
                const int cq = (int)((pk >> (8 * q)) & 0xFFu);
                if (p == q && r >= cq) {
                    r -= cq;
                    p = q + 1;
                }
            }
            // a site class's entries: the pair's two rows; a pair class's: row
            // 2p's horizontal bonds, the vertical bonds below it, its left
            // cross bond, for p = 0 the top-halo bonds, then row 2p + 1's
            // horizontal, vertical and left cross bonds
            const bool site = k == 0 || k == 3;
            const uint2 q0 = rows[(2 * p) * 32 + lane], q1 = rows[(2 * p + 1) * 32 + lane];
            const uint32_t s0 = k == 0 ? q0.x : q0.y, s1 = k == 0 ? q1.x : q1.y;
            const uint4 qv = bq[(site ? 0 : k - 1) * 32 * NP + 32 * p + lane];
            const uint32_t lb = k == 2 ? lb2 : lb1, nb = k == 2 ? n2 : n1;
            const uint32_t ms[7] = {site ? s0 : qv.x, site ? 0u : qv.z, site ? 0u : (lb >> (2 * p)) & 1u,
                                    (site || p != 0) ? 0u : nb, site ? s1 : qv.y, site ? 0u : qv.w,
                                    site ? 0u : (lb >> (2 * p + 1)) & 1u};
            uint32_t msk = 0u;
            int u0 = 0;
            bool found = false;
#pragma unroll
            for (int u = 0; u < 7; ++u) {
                const int cq = __popc(ms[u]);
                if (!found) {
                    if (r < cq) { msk = ms[u]; u0 = u; found = true; }
                    else r -= cq;
                }
            }
            const int rr = 2 * p + (u0 >= 4 ? 1 : 0);
            const int kind = site ? 0 : (u0 == 1 || u0 == 5 ? ((u0 == 5 && p == NP - 1) ? 3 : 2)
                                                           : (u0 == 2 || u0 == 6 ? 4 : (u0 == 3 ? 5 : 1)));
            code = (kind << 8) | (rr << 5) | select_bit(msk, r);
        }
        code = __shfl_sync(FULLW, code, owner, W);
        int dA = 0, dB = 0;  // the row pairs to recount (pair 0, unchanged, if none)
        if (live) {
            const int kind = code >> 8, rr = (code >> 5) & 7, x = code & 31;
            const uint32_t bit = 1u << x;
            // the changed sites' new state: A (class 0, adsorption), empty
            // (class 3, desorption; class 2, the reaction) or B (class 1, B2
            // adsorption: neither mask)
            const uint32_t setE = k >= 2 ? ~0u : 0u, setA = k == 0 ? ~0u : 0u;
            // this lane's changed sites: mA in its row r1, mB in row r1 + 1
            int r1 = -2;
            uint32_t mA = 0u, mB = 0u;
            if (l == owner) {
                // the sites of the member's row rr (a site; both ends of a
                // horizontal bond; the site of a cross or top-halo bond; the
                // upper end of a vertical one) and, for a vertical bond within
                // the lane, of row rr + 1; and the halo sites the bond changes
                r1 = rr;
                mA = kind == 1 ? (bit | (x < 31 ? bit << 1 : 0u)) : (kind == 4 ? 1u : bit);
                mB = kind == 2 ? bit : 0u;
                // a bond's ends become empty or B
                const uint32_t hm = (kind == 1 && x == 31) ? 1u << (16 + rr) : (kind == 4 ? 1u << rr : 0u);
                hx = (hx & ~(hm * 0x101u)) | (hm & setE);
                if (kind == 5 || (kind == 3 && last)) {
                    eH = (eH & ~bit) | (bit & setE);
                    aH &= ~bit;
                }
                // the pairs whose members change: pair p reads rows 2p, 2p + 1,
                // 2p + 2 (the next lane's row 0 for the last pair) and the halo
                // sites of its rows
                dA = rr >> 1;
                dB = (rr & 1) ? (kind == 2 ? (rr + 1) >> 1 : dA) : (rr >= 2 ? (rr >> 1) - 1 : dA);
            } else if (kind == 3 && owner != nrl - 1 && l == owner + 1) {
                // the lower end of a vertical bond below the owner's last row
                // (unless the owner holds the cell's last row: the bottom halo
                // row, changed above); its pair 0 changes
                r1 = -1;
                mB = bit;
            } else if (rr == 0 && kind != 3 && l == owner - 1) {
                dA = NP - 1;  // the owner's row 0 is this lane's row below
                dB = NP - 1;
            }
            if (r1 >= 0) {
                uint2 &v = rows[(r1 & (RL - 1)) * 32 + lane];
                v.x = (v.x & ~mA) | (mA & setE);
                v.y = (v.y & ~mA) | (mA & setA);
            }
            if (mB) {
                uint2 &v = rows[((r1 + 1) & (RL - 1)) * 32 + lane];
                v.x = (v.x & ~mB) | (mB & setE);
                v.y = (v.y & ~mB) | (mB & setA);
            }
            ++ev;
        }
        // the rows' changes before the row below is read; the row below is
        // read before the next event changes it
        __syncwarp();
        load_below();
        pair_update(dA);
        pair_update(dB);
        __syncwarp();
    }

    // Write back: the cell's rows, and the owned halo ends (the halo columns
    // in E windows, the halo rows in O windows)
    if (row) {
        uint8_t *const out = C.dst;
        const int lx = C.lx, ly = C.ly, X0 = C.X0, Y0 = C.Y0;
        const int y0 = Y0 + RL * l;
#pragma unroll
        for (int r = 0; r < RL; ++r) {
            const uint2 v = rows[r * 32 + lane];
            zgb_store_row(out + (int64_t)(y0 + r) * lx + X0, v.x, v.y);
        }
        if (ew) {
            const int gxl = X0 > 0 ? X0 - 1 : lx - 1, gxr = X0 + 32 < lx ? X0 + 32 : 0;
#pragma unroll
            for (int r = 0; r < RL; ++r) {
                const uint32_t h = hx >> r;
                out[(int64_t)(y0 + r) * lx + gxl] = (uint8_t)((h & 1u) ? 0 : ((h & 0x100u) ? 1 : 2));
                out[(int64_t)(y0 + r) * lx + gxr] = (uint8_t)((h & 0x10000u) ? 0 : ((h & 0x1000000u) ? 1 : 2));
            }
        } else {
            if (first) zgb_store_row(out + (int64_t)(Y0 > 0 ? Y0 - 1 : ly - 1) * lx + X0, eH, aH);
            if (last) zgb_store_row(out + (int64_t)(Y0 + qy < ly ? Y0 + qy : 0) * lx + X0, eH, aH);
        }
    }
    if (bad) *bad_out = true;
    return ev;
}

}  // namespace

}  // namespace fskmc
