// The binary32-clock window of two 32-wide ZGB cells per warp, held in
// registers: half h = lane / 16 of the warp runs cell h, and its local lane
// l = lane % 16 owns rows 2l and 2l + 1 of that cell.
//
// This is zgb32_window (fskmc_zgb32.cuh) with two rows per lane: the same
// classes from bit masks, the same undirected bonds at twice the directed
// rate, the same draws, fixed-point class sums and binary32 clock, one
// cell's events in order. The two cells step in lockstep, one event each
// per iteration, until both windows have ended; what is shared is the
// instruction stream, so the steps that one lane of a cell does for the
// whole cell (the class and member draw, the clock, the member's position)
// are issued once for two cells. A cell whose window has ended idles until
// the other's ends.
//
// Members of a pair class, numbered as the one-row window numbers them: row
// by row, and within a row y its horizontal bonds ((x, y)-(x+1, y); x = 31
// is the cross bond to the right halo, owned in E windows), the vertical
// bonds below it ((x, y)-(x, y+1); for the cell's last row the cross bonds
// to the bottom halo, owned in O windows), its left cross bond (E windows)
// and, for row 0, the vertical cross bonds to the top halo (O windows). With
// the same draws per event, both windows take the same events: the two
// kernels give identical lattices.
#pragma once
#include <cuda_runtime.h>

#include "fskmc_device.cuh"
#include "fskmc_internal.h"
#include "fskmc_zgb32.cuh"
#include "philox.cuh"

namespace fskmc {

namespace {

// Shared memory one half-warp's cell needs: the staged box rows and the
// per-window constants.
__host__ __device__ constexpr int zgbp_half_smem(int qy)
{
    return 64 * (qy + 2) + (int)sizeof(Zgb32Const);
}

// Shared memory per warp: both halves' cells, then each lane's bond masks of
// the two pair classes as counted in the current event ({H0, H1, V0, V1}
// and {L, N} per class and lane), which the owner of the drawn member reads
// back instead of recomputing them.
__host__ __device__ constexpr int zgbp_warp_smem(int qy)
{
    return 2 * zgbp_half_smem(qy) + 2 * 32 * 16 + 2 * 32 * 8;
}

// Two cells per warp: rows of even count 4 <= qy <= 32.
__host__ __device__ constexpr bool zgbp_shape_ok(int qx, int qy)
{
    return qx == 32 && qy >= 4 && qy <= 32 && (qy & 1) == 0;
}

// A lane's members of pair class k, by kind. e0, a0 / e1, a1: empty and A
// masks of rows 2l and 2l + 1; eB, aB: the row below row 2l + 1 (the
// bottom halo row in the last row lane); eN, aN: the top halo row (read in
// local lane 0 only); hl, hr: the left and right halo sites of the two rows,
// bit 2r set if row r's site is empty, bit 2r + 1 if it holds A. Lanes
// beyond the cell's rows hold all-zero masks and so have no members.
struct ZgbPairBonds {
    uint32_t H0, H1, V0, V1, L, N;  // L: bit r = row r's left cross bond
};

__device__ __forceinline__ ZgbPairBonds zgbp_bonds(int k, bool last, bool first, bool ew, uint32_t e0,
                                                   uint32_t a0, uint32_t e1, uint32_t a1, uint32_t eB,
                                                   uint32_t aB, uint32_t eN, uint32_t aN, uint32_t hl,
                                                   uint32_t hr)
{
    // right neighbours of every site of a row: site 31's is the right halo site
    const uint32_t eR0 = __funnelshift_r(e0, hr, 1), aR0 = __funnelshift_r(a0, hr >> 1, 1);
    const uint32_t eR1 = __funnelshift_r(e1, hr >> 2, 1), aR1 = __funnelshift_r(a1, hr >> 3, 1);
    const uint32_t ownH = ew ? ~0u : 0x7FFFFFFFu;           // bond 31 crosses to the right halo
    const uint32_t ownV1 = (!last || !ew) ? ~0u : 0u;       // the last row's bonds cross to the bottom halo
    const uint32_t ownN = (first && !ew) ? ~0u : 0u;        // local lane 0: bonds to the top halo
    const uint32_t ownL = ew ? 3u : 0u;
    ZgbPairBonds B;
    if (k == 1) {
        B.H0 = e0 & eR0 & ownH;
        B.H1 = e1 & eR1 & ownH;
        B.V0 = e0 & e1;
        B.V1 = e1 & eB & ownV1;
        B.L = ((hl & e0 & 1u) | ((hl >> 1) & (e1 << 1) & 2u)) & ownL;
        B.N = eN & e0 & ownN;
    } else {
        const uint32_t b0 = ~(e0 | a0), b1 = ~(e1 | a1);
        const uint32_t bR0 = ~(eR0 | aR0), bR1 = ~(eR1 | aR1), bB = ~(eB | aB), bN = ~(eN | aN);
        B.H0 = ((a0 & bR0) | (b0 & aR0)) & ownH;
        B.H1 = ((a1 & bR1) | (b1 & aR1)) & ownH;
        B.V0 = (a0 & b1) | (b0 & a1);
        B.V1 = ((a1 & bB) | (b1 & aB)) & ownV1;
        // left halo site of row r: A if bit 2r + 1, B if neither bit
        const uint32_t hla = ((hl >> 1) & 1u) | ((hl >> 2) & 2u);
        const uint32_t hlb = (~(hl | (hl >> 1)) & 1u) | (~((hl >> 1) | (hl >> 2)) & 2u);
        const uint32_t s0a = a0 & 1u, s0b = b0 & 1u, s1a = (a1 & 1u) << 1, s1b = (b1 & 1u) << 1;
        B.L = ((hla & (s0b | s1b)) | (hlb & (s0a | s1a))) & ownL;
        B.N = ((aN & b0) | (bN & a0)) & ownN;
    }
    return B;
}

__device__ __forceinline__ int zgbp_bond_count(const ZgbPairBonds &B)
{
    return __popc(B.H0) + __popc(B.H1) + __popc(B.V0) + __popc(B.V1) + __popc(B.L) + __popc(B.N);
}


// The windows of two cells (qx == 32, even 4 <= qy <= 32) by one warp: half
// h runs the cell at `at` (its own; `valid` false for a half without a
// cell) of replica R in the byte lattice src (== dst: ZGB updates in
// place). wsm: zgbp_warp_smem(qy) bytes of 16-byte aligned shared
// memory. Returns this half's events; *bad_out is set if a rank search found
// no member (never, unless the counts and masks disagree) or a window ran
// away.
template <bool PERSIST>
__device__ uint32_t zgb32x2_window(uint8_t *wsm, const Replica &R, const CellGeom &G, const CellAt &at,
                                   bool valid, int colour, uint32_t w, double hwin, uint64_t seed,
                                   const uint8_t *src, uint8_t *dst, int lane, bool *bad_out)
{
    constexpr unsigned FULLW = 0xffffffffu;
    const int qy = G.qy, BH = qy + 2;
    const int l = lane & 15, seg = lane & 16;
    const unsigned hmask = seg ? 0xFFFF0000u : 0x0000FFFFu;
    const bool ew = colour == 0;
    const bool row = valid && l < (qy >> 1), first = l == 0, last = l == (qy >> 1) - 1;
    uint8_t *raw = wsm + (seg ? zgbp_half_smem(qy) : 0);
    uint4 *bq = reinterpret_cast<uint4 *>(wsm + 2 * zgbp_half_smem(qy));     // [class - 1][lane]
    uint2 *bln = reinterpret_cast<uint2 *>(wsm + 2 * zgbp_half_smem(qy) + 1024);

    // Stage each half's box rows (the rows above and below its cell too) as
    // four aligned 16-byte chunks: the 16 sites left of the cell, its 32, the
    // 16 right of it.
    if (valid) {
        const int lx = at.lx, ly = at.ly, X0 = at.X0, Y0 = at.Y0;
        const int xl = X0 >= 16 ? X0 - 16 : X0 - 16 + lx;
        const int xr = X0 + 32 < lx ? X0 + 32 : X0 + 32 - lx;
        for (int i = l; i < 4 * BH; i += 16) {
            const int by = i >> 2, part = i & 3;
            int gy = Y0 - 1 + by;
            gy += (gy < 0) ? ly : 0; gy -= (gy >= ly) ? ly : 0;
            const int gx = part == 0 ? xl : (part == 3 ? xr : X0 + 16 * (part - 1));
            cp_async16(raw + by * 64 + 16 * part, src + (int64_t)gy * lx + gx);
        }
    }
    Zgb32Const *Cw = reinterpret_cast<Zgb32Const *>(raw + 64 * BH);
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
    cp_async_wait_all();
    __syncwarp();
    const volatile Zgb32Const &C = *Cw;
    // local lane l: rows 2l and 2l + 1 (box rows 2l + 1, 2l + 2) and their
    // halo sites; (eH, aH): in local lane 0 the top halo row, in the last
    // row lane the bottom halo row (qy >= 4: two different lanes)
    uint32_t e0 = 0u, a0 = 0u, e1 = 0u, a1 = 0u, eH = 0u, aH = 0u, hl = 0u, hr = 0u;
    if (row) {
        const uint8_t *r0 = raw + (2 * l + 1) * 64 + 16, *r1 = r0 + 64;
        zgb_row_masks(r0, e0, a0);
        zgb_row_masks(r1, e1, a1);
        hl = (uint32_t)(r0[-1] == 0) | ((uint32_t)(r0[-1] == 1) << 1) | ((uint32_t)(r1[-1] == 0) << 2) |
             ((uint32_t)(r1[-1] == 1) << 3);
        hr = (uint32_t)(r0[32] == 0) | ((uint32_t)(r0[32] == 1) << 1) | ((uint32_t)(r1[32] == 0) << 2) |
             ((uint32_t)(r1[32] == 1) << 3);
        if (first) zgb_row_masks(raw + 16, eH, aH);
        if (last) zgb_row_masks(raw + (qy + 1) * 64 + 16, eH, aH);
    }

    float tauf = 0.0f, rlf = 0.0f;
    uint32_t rw2 = 0u, rw3 = 0u, ev = 0u, it = 0u;
    bool live = valid, bad = false;
    while (__any_sync(FULLW, live)) {
        // this half's classes: each lane's member counts, the totals and the
        // fixed-point rate sums
        uint32_t eB = __shfl_down_sync(FULLW, e0, 1, 16), aB = __shfl_down_sync(FULLW, a0, 1, 16);
        if (last) { eB = eH; aB = aH; }
        int cl[4];
        cl[0] = __popc(e0) + __popc(e1);
        cl[3] = __popc(a0) + __popc(a1);
        {
            const ZgbPairBonds B1 = zgbp_bonds(1, last, first, ew, e0, a0, e1, a1, eB, aB, eH, aH, hl, hr);
            const ZgbPairBonds B2 = zgbp_bonds(2, last, first, ew, e0, a0, e1, a1, eB, aB, eH, aH, hl, hr);
            cl[1] = zgbp_bond_count(B1);
            cl[2] = zgbp_bond_count(B2);
            bq[lane] = make_uint4(B1.H0, B1.H1, B1.V0, B1.V1);
            bq[32 + lane] = make_uint4(B2.H0, B2.H1, B2.V0, B2.V1);
            bln[lane] = make_uint2(B1.L, B1.N);
            bln[32 + lane] = make_uint2(B2.L, B2.N);
        }
        uint32_t n[4];
        {  // the four totals as two packed sums (each below 2^16)
            const uint32_t s03 = __reduce_add_sync(hmask, (uint32_t)cl[0] | ((uint32_t)cl[3] << 16));
            const uint32_t s12 = __reduce_add_sync(hmask, (uint32_t)cl[1] | ((uint32_t)cl[2] << 16));
            n[0] = s03 & 0xFFFFu; n[3] = s03 >> 16; n[1] = s12 & 0xFFFFu; n[2] = s12 >> 16;
        }
        const uint64_t P0 = (uint64_t)n[0] * C.rq[0], P1 = P0 + (uint64_t)n[1] * C.rq[1];
        const uint64_t P2 = P1 + (uint64_t)n[2] * C.rq[2], lami = P2 + (uint64_t)n[3] * C.rq[3];
        if (lami == 0ull) live = false;
        if (live && ev >= MAX_EVENTS_PER_WINDOW) {
            bad = true;
            live = false;
        }
        if ((it & 15u) == 0u && valid) {  // 16 events' draws at once, one Philox block per lane
            const u32x4 o = draw(C.seed, it + (uint32_t)l, C.w, C.m, C.ctr3);
            rlf = -__logf(__fmul_rn(__uint2float_rn((o.x >> 8) + 1u), 0x1p-24f));
            rw2 = o.z;
            rw3 = o.w;
        }
        const int sl = (int)(it & 15u);
        const uint32_t w2 = __shfl_sync(FULLW, rw2, sl, 16), w3 = __shfl_sync(FULLW, rw3, sl, 16);
        // class: the first k with (w2 lambda) >> 32 < P_k (exact integers),
        // member j of it, and this lane's count of that class
        const uint64_t t = (uint64_t)w2 * (lami >> 32) + (((uint64_t)w2 * (lami & 0xffffffffull)) >> 32);
        const int k = t < P0 ? 0 : (t < P1 ? 1 : (t < P2 ? 2 : 3));
        const uint32_t nk = k == 0 ? n[0] : (k == 1 ? n[1] : (k == 2 ? n[2] : n[3]));
        const uint32_t j = (uint32_t)(((uint64_t)w3 * (uint64_t)nk) >> 32);
        const int c = k == 0 ? cl[0] : (k == 1 ? cl[1] : (k == 2 ? cl[2] : cl[3]));
        // the clock: the event happens if it falls within the window
        const float lg = __shfl_sync(FULLW, rlf, sl, 16);
        if (live) {
            const float lamf = __fmul_rn(u64_to_float_rz(lami), C.qscale);
            const float end = __fadd_rn(tauf, __fdividef(lg, lamf));
            if (end >= C.hf) live = false;
            else tauf = end;
        }
        if (!__any_sync(FULLW, live)) break;  // both windows ended at this draw
        // the owner of member j: a prefix scan of the half's counts, then the
        // bit in the owner's masks
        int incl = c;
#pragma unroll
        for (int off = 1; off < 16; off <<= 1) {
            const int v = __shfl_up_sync(FULLW, incl, off, 16);
            if (l >= off) incl += v;
        }
        const uint32_t hit = (__ballot_sync(FULLW, live && (uint32_t)incl > j) & hmask) >> seg;
        if (live && hit == 0u) {
            bad = true;
            live = false;
        }
        const int owner = hit ? __ffs(hit) - 1 : 0;
        // kind: 0 site, 1 horizontal bond, 2 vertical bond within the lane,
        // 3 vertical bond below it, 4 left cross bond, 5 top-halo bond; rr:
        // which of the lane's two rows (kinds 0, 1, 4)
        int code = 0;
        if (live && l == owner) {
            int r = (int)j - (incl - c);
            uint32_t msk;
            int kind, rr;
            if (k == 0 || k == 3) {
                const uint32_t m0 = k == 0 ? e0 : a0, m1 = k == 0 ? e1 : a1;
                const int p0 = __popc(m0);
                kind = 0;
                rr = r >= p0 ? 1 : 0;
                msk = rr ? m1 : m0;
                r -= rr ? p0 : 0;
            } else {
                // this lane's members of class k as counted above: row 2l's
                // (its horizontal bonds, the vertical bonds below it, its left
                // cross bond, the top-halo bonds), then row 2l + 1's -- the
                // one-row window's numbering row by row
                const uint4 q = bq[(k - 1) * 32 + lane];
                const uint2 ln = bln[(k - 1) * 32 + lane];
                const uint32_t L0 = ln.x & 1u, L1 = (ln.x >> 1) & 1u;
                const int cH0 = __popc(q.x), cV0 = __popc(q.z), cN = __popc(ln.y), cH1 = __popc(q.y);
                const int cV1 = __popc(q.w);
                msk = q.x; kind = 1; rr = 0;
                if (r >= cH0) {
                    r -= cH0; msk = q.z; kind = 2;
                    if (r >= cV0) {
                        r -= cV0; msk = L0; kind = 4;
                        if (r >= (int)L0) {
                            r -= (int)L0; msk = ln.y; kind = 5;
                            if (r >= cN) {
                                r -= cN; msk = q.y; kind = 1; rr = 1;
                                if (r >= cH1) {
                                    r -= cH1; msk = q.w; kind = 3;
                                    if (r >= cV1) { r -= cV1; msk = L1; kind = 4; }
                                }
                            }
                        }
                    }
                }
            }
            code = (kind << 6) | (rr << 5) | select_bit(msk, r);
        }
        code = __shfl_sync(FULLW, code, owner, 16);
        if (live) {
            const int kind = code >> 6, rr = (code >> 5) & 1, x = code & 31;
            const uint32_t bit = 1u << x;
            if (kind == 0) {
                if (l == owner) {
                    // A adsorbs on an empty site (class 0) or desorbs (class 3)
                    const uint32_t m0 = rr ? 0u : bit, m1 = rr ? bit : 0u;
                    if (k == 0) { e0 &= ~m0; a0 |= m0; e1 &= ~m1; a1 |= m1; }
                    else { a0 &= ~m0; e0 |= m0; a1 &= ~m1; e1 |= m1; }
                }
            } else {
                // B2 adsorption makes both ends B, the reaction both ends empty
                const bool toB = k == 1;
                uint32_t m0 = 0u, m1 = 0u, hrc = 0u, hlc = 0u;  // sites of rows 0 / 1, halo bit pairs
                bool hrow = false;                               // the top / bottom halo row's bit x
                if (kind == 1) {
                    const uint32_t m = bit | (x < 31 ? bit << 1 : 0u);
                    if (rr) m1 = m; else m0 = m;
                    if (x == 31) hrc = 3u << (2 * rr);
                } else if (kind == 2) {
                    m0 = bit;
                    m1 = bit;
                } else if (kind == 3) {
                    m1 = bit;
                    hrow = last;
                } else if (kind == 4) {
                    if (rr) m1 = 1u; else m0 = 1u;
                    hlc = 3u << (2 * rr);
                } else {
                    m0 = bit;
                    hrow = true;
                }
                const uint32_t hval = toB ? 0u : 0x5u;  // empty: bit 2r of the pair; B: neither
                if (l == owner) {
                    e0 = toB ? (e0 & ~m0) : (e0 | m0);
                    a0 &= ~m0;
                    e1 = toB ? (e1 & ~m1) : (e1 | m1);
                    a1 &= ~m1;
                    hr = (hr & ~hrc) | (hval & hrc);
                    hl = (hl & ~hlc) | (hval & hlc);
                    if (hrow) { eH = toB ? (eH & ~bit) : (eH | bit); aH &= ~bit; }
                }
                // the lower end of a vertical bond below the owner's second
                // row, unless the owner holds the cell's last row (then it is
                // the bottom halo row, changed above)
                if (kind == 3 && owner != (qy >> 1) - 1 && l == owner + 1) {
                    e0 = toB ? (e0 & ~bit) : (e0 | bit);
                    a0 &= ~bit;
                }
            }
            ++ev;
        }
        ++it;
    }

    // Write back: the cell's rows, and the owned halo ends (the halo columns
    // in E windows, the halo rows in O windows)
    if (row) {
        uint8_t *const out = C.dst;
        const int lx = C.lx, ly = C.ly, X0 = C.X0, Y0 = C.Y0;
        const int y0 = Y0 + 2 * l;
        zgb_store_row(out + (int64_t)y0 * lx + X0, e0, a0);
        zgb_store_row(out + (int64_t)(y0 + 1) * lx + X0, e1, a1);
        if (ew) {
            const int gxl = X0 > 0 ? X0 - 1 : lx - 1, gxr = X0 + 32 < lx ? X0 + 32 : 0;
            const auto st = [](uint32_t h2) { return (uint8_t)((h2 & 1u) ? 0 : ((h2 & 2u) ? 1 : 2)); };
            out[(int64_t)y0 * lx + gxl] = st(hl);
            out[(int64_t)y0 * lx + gxr] = st(hr);
            out[(int64_t)(y0 + 1) * lx + gxl] = st(hl >> 2);
            out[(int64_t)(y0 + 1) * lx + gxr] = st(hr >> 2);
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
