// The binary32-clock window of four 32-wide ZGB cells per warp, held in
// registers: group g = lane / 8 of the warp runs cell g, and its local lane
// l = lane % 8 owns rows 4l .. 4l + 3 of that cell.
//
// This is zgb32x2_window (fskmc_zgb32x2.cuh) with four rows per lane and
// four cells per warp: the same classes from bit masks (each pair of rows
// through zgbp_bonds), the same undirected bonds at twice the directed
// rate, the same draws (event e of a cell draws Philox counter e), the same
// fixed-point class sums, binary32 clock and member numbering (row by row),
// so it gives the lattices of the one- and two-cell kernels. The four cells
// step in lockstep, one event each per iteration, until all four windows
// have ended; the steps one lane does for a whole cell are issued once for
// four cells. The rows are loaded from global memory straight into
// registers (no shared-memory staging), so the shared memory a warp holds is
// only the cells' constants and the lanes' bond masks.
#pragma once
#include <cuda_runtime.h>

#include "fskmc_device.cuh"
#include "fskmc_internal.h"
#include "fskmc_zgb32.cuh"
#include "fskmc_zgb32x2.cuh"
#include "philox.cuh"

namespace fskmc {

namespace {

// Four cells per warp: rows in multiples of 4, 8 <= qy <= 32.
__host__ __device__ constexpr bool zgbq_shape_ok(int qx, int qy)
{
    return qx == 32 && qy >= 8 && qy <= 32 && (qy & 3) == 0;
}

// Shared memory per warp: the four cells' constants, then each lane's bond
// masks of the two pair classes for its two row pairs ({H0, H1, V0, V1} per
// pair) and {L, N}.
__host__ __device__ constexpr int zgbq_warp_smem()
{
    return 4 * (int)sizeof(Zgb32Const) + 2 * 32 * 32 + 2 * 32 * 8;
}

// Empty / A masks of the 32 sites of a row held as two 16-byte words
// (states 0, 1, 2; see zgb_row_masks).
__device__ __forceinline__ void zgbq_masks(const uint4 u0, const uint4 u1, uint32_t &e, uint32_t &a)
{
    const uint32_t v[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
    e = 0u;
    a = 0u;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t ta = v[k] & 0x01010101u;
        const uint32_t te = ~(v[k] | (v[k] >> 1)) & 0x01010101u;
        e |= ((te * 0x00204081u) >> 21 & 0xFu) << (4 * k);
        a |= ((ta * 0x00204081u) >> 21 & 0xFu) << (4 * k);
    }
}

template <bool PERSIST>
__device__ __forceinline__ uint4 zgbq_ld16(const uint8_t *p)
{
    const uint4 *q = reinterpret_cast<const uint4 *>(p);
    if (PERSIST) return __ldcg(q);
    return *q;
}

// A site's halo code: bit 0 empty, bit 1 A (B neither).
__device__ __forceinline__ uint32_t zgbq_hcode(uint8_t s)
{
    return (uint32_t)(s == 0) | ((uint32_t)(s == 1) << 1);
}


// The windows of four cells (qx == 32, qy a multiple of 4 in 8..32) by one
// warp: group g runs the cell at `at` (its own; `valid` false for a group
// without a cell) of replica R in the byte lattice src (== dst: ZGB updates
// in place), all four of the same window. wsm: zgbq_warp_smem() bytes of
// 16-byte aligned shared memory. Returns this group's events; *bad_out is
// set if a rank search found no member (never, unless the counts and masks
// disagree) or a window ran away.
template <bool PERSIST>
__device__ uint32_t zgb32x4_window(uint8_t *wsm, const Replica &R, const CellGeom &G, const CellAt &at, bool valid,
                                   int colour, uint32_t w, double hwin, uint64_t seed, const uint8_t *src,
                                   uint8_t *dst, int lane, bool *bad_out)
{
    constexpr unsigned FULLW = 0xffffffffu;
    const int qy = G.qy, nrl = qy >> 2;  // lanes holding the cell's rows
    const int l = lane & 7, gb = lane & 24;
    const unsigned gmask = 0xFFu << gb;
    const bool ew = colour == 0;
    const bool row = valid && l < nrl, first = l == 0, last = l == nrl - 1;
    Zgb32Const *Cw = reinterpret_cast<Zgb32Const *>(wsm) + (lane >> 3);
    uint4 *bq = reinterpret_cast<uint4 *>(wsm + 4 * sizeof(Zgb32Const));           // [class - 1][lane][row pair]
    uint2 *bln = reinterpret_cast<uint2 *>(wsm + 4 * sizeof(Zgb32Const) + 2048);   // [class - 1][lane]

    // The lane's rows 4l .. 4l + 3 and their halo sites, loaded from global
    // memory into registers; local lane 0 also the halo row above the cell,
    // the last row lane the one below (qy >= 8: two different lanes). hl,
    // hr: row r's left / right halo site at bits 2r (empty), 2r + 1 (A).
    uint32_t e[4] = {0u, 0u, 0u, 0u}, a[4] = {0u, 0u, 0u, 0u}, eH = 0u, aH = 0u, hl = 0u, hr = 0u;
    if (row) {
        const int lx = at.lx, ly = at.ly, X0 = at.X0, Y0 = at.Y0;
        const int gxl = X0 > 0 ? X0 - 1 : lx - 1, gxr = X0 + 32 < lx ? X0 + 32 : 0;
        uint4 u[8];
        uint8_t hL[4], hR[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const uint8_t *p = src + (int64_t)(Y0 + 4 * l + r) * lx;
            u[2 * r] = zgbq_ld16<PERSIST>(p + X0);
            u[2 * r + 1] = zgbq_ld16<PERSIST>(p + X0 + 16);
            hL[r] = ld_site<PERSIST>(p + gxl);
            hR[r] = ld_site<PERSIST>(p + gxr);
        }
        uint4 h0 = make_uint4(0u, 0u, 0u, 0u), h1 = h0;
        if (first || last) {
            const int hy = first ? (Y0 > 0 ? Y0 - 1 : ly - 1) : (Y0 + qy < ly ? Y0 + qy : 0);
            const uint8_t *p = src + (int64_t)hy * lx + X0;
            h0 = zgbq_ld16<PERSIST>(p);
            h1 = zgbq_ld16<PERSIST>(p + 16);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            zgbq_masks(u[2 * r], u[2 * r + 1], e[r], a[r]);
            hl |= zgbq_hcode(hL[r]) << (2 * r);
            hr |= zgbq_hcode(hR[r]) << (2 * r);
        }
        if (first || last) zgbq_masks(h0, h1, eH, aH);
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

    float tauf = 0.0f, rlf = 0.0f;
    uint32_t rw2 = 0u, rw3 = 0u, ev = 0u;
    bool live = valid, bad = false;
    while (__any_sync(FULLW, live)) {
        // this cell's classes: each lane's member counts (its two row pairs
        // through zgbp_bonds), the totals and the fixed-point rate sums
        uint32_t eB = __shfl_down_sync(FULLW, e[0], 1, 8), aB = __shfl_down_sync(FULLW, a[0], 1, 8);
        if (last) { eB = eH; aB = aH; }
        int cl[4];
        cl[0] = __popc(e[0]) + __popc(e[1]) + __popc(e[2]) + __popc(e[3]);
        cl[3] = __popc(a[0]) + __popc(a[1]) + __popc(a[2]) + __popc(a[3]);
        {
            const ZgbPairBonds B10 = zgbp_bonds(1, false, first, ew, e[0], a[0], e[1], a[1], e[2], a[2], eH, aH, hl, hr);
            const ZgbPairBonds B11 =
                zgbp_bonds(1, last, false, ew, e[2], a[2], e[3], a[3], eB, aB, eH, aH, hl >> 4, hr >> 4);
            const ZgbPairBonds B20 = zgbp_bonds(2, false, first, ew, e[0], a[0], e[1], a[1], e[2], a[2], eH, aH, hl, hr);
            const ZgbPairBonds B21 =
                zgbp_bonds(2, last, false, ew, e[2], a[2], e[3], a[3], eB, aB, eH, aH, hl >> 4, hr >> 4);
            cl[1] = zgbp_bond_count(B10) + zgbp_bond_count(B11);
            cl[2] = zgbp_bond_count(B20) + zgbp_bond_count(B21);
            bq[2 * lane] = make_uint4(B10.H0, B10.H1, B10.V0, B10.V1);
            bq[2 * lane + 1] = make_uint4(B11.H0, B11.H1, B11.V0, B11.V1);
            bq[64 + 2 * lane] = make_uint4(B20.H0, B20.H1, B20.V0, B20.V1);
            bq[64 + 2 * lane + 1] = make_uint4(B21.H0, B21.H1, B21.V0, B21.V1);
            bln[lane] = make_uint2(B10.L | (B11.L << 2), B10.N);
            bln[32 + lane] = make_uint2(B20.L | (B21.L << 2), B20.N);
        }
        uint32_t n[4];
        {  // the four totals as two packed sums (each below 2^16)
            const uint32_t s03 = __reduce_add_sync(gmask, (uint32_t)cl[0] | ((uint32_t)cl[3] << 16));
            const uint32_t s12 = __reduce_add_sync(gmask, (uint32_t)cl[1] | ((uint32_t)cl[2] << 16));
            n[0] = s03 & 0xFFFFu; n[3] = s03 >> 16; n[1] = s12 & 0xFFFFu; n[2] = s12 >> 16;
        }
        const uint64_t P0 = (uint64_t)n[0] * C.rq[0], P1 = P0 + (uint64_t)n[1] * C.rq[1];
        const uint64_t P2 = P1 + (uint64_t)n[2] * C.rq[2], lami = P2 + (uint64_t)n[3] * C.rq[3];
        if (lami == 0ull) live = false;
        if (live && ev >= MAX_EVENTS_PER_WINDOW) {
            bad = true;
            live = false;
        }
        if ((ev & 7u) == 0u && live) {  // 8 events' draws at once, one Philox block per lane
            const u32x4 o = draw(C.seed, ev + (uint32_t)l, C.w, C.m, C.ctr3);
            rlf = -__logf(__fmul_rn(__uint2float_rn((o.x >> 8) + 1u), 0x1p-24f));
            rw2 = o.z;
            rw3 = o.w;
        }
        const int sl = (int)(ev & 7u);
        const uint32_t w2 = __shfl_sync(FULLW, rw2, sl, 8), w3 = __shfl_sync(FULLW, rw3, sl, 8);
        // class: the first k with (w2 lambda) >> 32 < P_k (exact integers),
        // member j of it, and this lane's count of that class
        const uint64_t t = (uint64_t)w2 * (lami >> 32) + (((uint64_t)w2 * (lami & 0xffffffffull)) >> 32);
        const int k = t < P0 ? 0 : (t < P1 ? 1 : (t < P2 ? 2 : 3));
        const uint32_t nk = k == 0 ? n[0] : (k == 1 ? n[1] : (k == 2 ? n[2] : n[3]));
        const uint32_t j = (uint32_t)(((uint64_t)w3 * (uint64_t)nk) >> 32);
        const int c = k == 0 ? cl[0] : (k == 1 ? cl[1] : (k == 2 ? cl[2] : cl[3]));
        // the clock: the event happens if it falls within the window
        const float lg = __shfl_sync(FULLW, rlf, sl, 8);
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
        for (int off = 1; off < 8; off <<= 1) {
            const int v = __shfl_up_sync(FULLW, incl, off, 8);
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
        // bond, 5 top-halo bond; rr: the row of the lane (0..3)
        int code = 0;
        if (live && l == owner) {
            int r = (int)j - (incl - c);
            uint32_t msk;
            int kind, rr;
            if (k == 0 || k == 3) {
                const uint32_t m[4] = {k == 0 ? e[0] : a[0], k == 0 ? e[1] : a[1], k == 0 ? e[2] : a[2],
                                       k == 0 ? e[3] : a[3]};
                kind = 0;
                msk = m[0];
                rr = 0;
                bool found = false;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int cq = __popc(m[q]);
                    if (!found) {
                        if (r < cq) { msk = m[q]; rr = q; found = true; }
                        else r -= cq;
                    }
                }
            } else {
                // the lane's members of class k as counted above, row by row:
                // each row's horizontal bonds, the vertical bonds below it, its
                // left cross bond, and for row 0 the top-halo bonds
                const uint4 q0 = bq[(k - 1) * 64 + 2 * lane], q1 = bq[(k - 1) * 64 + 2 * lane + 1];
                const uint2 ln = bln[(k - 1) * 32 + lane];
                const uint32_t ms[13] = {q0.x, q0.z, ln.x & 1u, ln.y, q0.y, q0.w, (ln.x >> 1) & 1u,
                                         q1.x, q1.z, (ln.x >> 2) & 1u, q1.y, q1.w, (ln.x >> 3) & 1u};
                constexpr int kd[13] = {1, 2, 4, 5, 1, 2, 4, 1, 2, 4, 1, 3, 4};
                constexpr int rw[13] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3};
                msk = ms[0];
                kind = 1;
                rr = 0;
                bool found = false;
#pragma unroll
                for (int q = 0; q < 13; ++q) {
                    const int cq = __popc(ms[q]);
                    if (!found) {
                        if (r < cq) { msk = ms[q]; kind = kd[q]; rr = rw[q]; found = true; }
                        else r -= cq;
                    }
                }
            }
            code = (kind << 7) | (rr << 5) | select_bit(msk, r);
        }
        code = __shfl_sync(FULLW, code, owner, 8);
        if (live) {
            const int kind = code >> 7, rr = (code >> 5) & 3, x = code & 31;
            const uint32_t bit = 1u << x;
            if (kind == 0) {
                if (l == owner) {
                    // A adsorbs on an empty site (class 0) or desorbs (class 3)
                    const bool toA = k == 0;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const uint32_t m = rr == q ? bit : 0u;
                        e[q] = toA ? (e[q] & ~m) : (e[q] | m);
                        a[q] = toA ? (a[q] | m) : (a[q] & ~m);
                    }
                }
            } else {
                // B2 adsorption makes both ends B, the reaction both ends empty
                const bool toB = k == 1;
                const uint32_t hrc = (kind == 1 && x == 31) ? 3u << (2 * rr) : 0u;
                const uint32_t hlc = kind == 4 ? 3u << (2 * rr) : 0u;
                const bool hrow = kind == 5 || (kind == 3 && last);
                const uint32_t hval = toB ? 0u : 0x55u;  // empty: bit 2r of a pair; B: neither
                if (l == owner) {
                    // the sites of the member's row rr (both ends of a horizontal
                    // bond, the site of a cross or top-halo bond, the upper end
                    // of a vertical one) and, for a vertical bond within the
                    // lane, of row rr + 1
                    const uint32_t mA = kind == 1 ? (bit | (x < 31 ? bit << 1 : 0u)) : (kind == 4 ? 1u : bit);
                    const uint32_t mB = kind == 2 ? bit : 0u;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const uint32_t m = (rr == q ? mA : 0u) | (rr + 1 == q ? mB : 0u);
                        e[q] = toB ? (e[q] & ~m) : (e[q] | m);
                        a[q] &= ~m;
                    }
                    hr = (hr & ~hrc) | (hval & hrc);
                    hl = (hl & ~hlc) | (hval & hlc);
                    if (hrow) { eH = toB ? (eH & ~bit) : (eH | bit); aH &= ~bit; }
                }
                // the lower end of a vertical bond below the owner's last row,
                // unless the owner holds the cell's last row (the bottom halo row,
                // changed above)
                if (kind == 3 && owner != nrl - 1 && l == owner + 1) {
                    e[0] = toB ? (e[0] & ~bit) : (e[0] | bit);
                    a[0] &= ~bit;
                }
            }
            ++ev;
        }
    }

    // Write back: the cell's rows, and the owned halo ends (the halo columns
    // in E windows, the halo rows in O windows)
    if (row) {
        uint8_t *const out = C.dst;
        const int lx = C.lx, ly = C.ly, X0 = C.X0, Y0 = C.Y0;
        const int y0 = Y0 + 4 * l;
#pragma unroll
        for (int r = 0; r < 4; ++r) zgb_store_row(out + (int64_t)(y0 + r) * lx + X0, e[r], a[r]);
        if (ew) {
            const int gxl = X0 > 0 ? X0 - 1 : lx - 1, gxr = X0 + 32 < lx ? X0 + 32 : 0;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const uint32_t cl2 = hl >> (2 * r), cr2 = hr >> (2 * r);
                out[(int64_t)(y0 + r) * lx + gxl] = (uint8_t)((cl2 & 1u) ? 0 : ((cl2 & 2u) ? 1 : 2));
                out[(int64_t)(y0 + r) * lx + gxr] = (uint8_t)((cr2 & 1u) ? 0 : ((cr2 & 2u) ? 1 : 2));
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
