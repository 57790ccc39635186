// The binary32-clock window of RL 32-wide ZGB cells per warp (RL = 4 or 8),
// held in registers: group g = lane / W of the warp (W = 32 / RL lanes)
// runs cell g, and its local lane l = lane % W owns rows RL l .. RL l + RL - 1
// of that cell.
//
// This is zgb32x2_window (fskmc_zgb32x2.cuh) with RL rows per lane and RL
// cells per warp: the same classes from bit masks (each pair of rows through
// zgbm_pair_bonds), the same undirected bonds at twice the directed rate, the
// same draws (event e of a cell draws Philox counter e), the same fixed-point
// class sums, binary32 clock and member numbering (row by row), so it gives
// the lattices of the one- and two-cell kernels. The cells step in lockstep,
// one event each per iteration, until all their windows have ended; the
// steps one lane does for a whole cell are issued once for RL cells. The
// rows are loaded from global memory straight into registers (no
// shared-memory staging), so the shared memory a warp holds is only the
// cells' constants and the lanes' bond masks.
#pragma once
#include <cuda_runtime.h>

#include "fskmc_device.cuh"
#include "fskmc_internal.h"
#include "fskmc_zgb32.cuh"
#include "fskmc_zgb32x2.cuh"
#include "philox.cuh"

namespace fskmc {

namespace {

// RL cells per warp: rows a multiple of RL, 2 RL <= qy <= 32 (a cell's first
// and last row lanes differ).
__host__ __device__ constexpr bool zgbm_shape_ok(int RL, int qx, int qy)
{
    return qx == 32 && qy >= 2 * RL && qy <= 32 && qy % RL == 0;
}

// Shared memory per warp: the RL cells' constants, then each lane's bond
// masks of the two pair classes for its RL / 2 row pairs ({H0, H1, V0, V1}
// per pair) and {L, N}.
__host__ __device__ constexpr int zgbm_warp_smem(int RL)
{
    return RL * (int)sizeof(Zgb32Const) + 2 * 32 * (RL / 2) * 16 + 2 * 32 * 8;
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

// A lane's members of the two pair classes in its rows r, r + 1 (empty
// masks e0, e1, A masks a0, a1), except the left cross bonds: the
// horizontal bonds of each row (bond 31 to the right halo site, owned in E
// windows), the vertical bonds between the two rows and below row r + 1
// (eB, aB: the row below; crossing to the bottom halo in the cell's last
// row, owned in O windows), and for the cell's row 0 the vertical bonds to
// the top halo row eN, aN (O windows). hre, hra: bit 0 (1) set if the right
// halo site of row r (r + 1) is empty / holds A. B2 adsorption takes an
// empty-empty bond; the reaction an A-B bond, i.e. one end A and neither
// end empty.
struct ZgbmPair {
    uint32_t H0, H1, V0, V1, N;
};

__device__ __forceinline__ void zgbm_pair_bonds(bool last, bool first, bool ew, uint32_t e0, uint32_t a0, uint32_t e1,
                                                uint32_t a1, uint32_t eB, uint32_t aB, uint32_t eN, uint32_t aN,
                                                uint32_t hre, uint32_t hra, ZgbmPair &B1, ZgbmPair &B2)
{
    // right neighbours of every site of a row: site 31's is the right halo site
    const uint32_t eR0 = __funnelshift_r(e0, hre, 1), aR0 = __funnelshift_r(a0, hra, 1);
    const uint32_t eR1 = __funnelshift_r(e1, hre >> 1, 1), aR1 = __funnelshift_r(a1, hra >> 1, 1);
    const uint32_t ownH = ew ? ~0u : 0x7FFFFFFFu;
    const uint32_t ownV1 = (!last || !ew) ? ~0u : 0u;
    const uint32_t ownN = (first && !ew) ? ~0u : 0u;
    B1.H0 = e0 & eR0 & ownH;
    B1.H1 = e1 & eR1 & ownH;
    B1.V0 = e0 & e1;
    B1.V1 = e1 & eB & ownV1;
    B1.N = eN & e0 & ownN;
    B2.H0 = (a0 ^ aR0) & ~(e0 | eR0) & ownH;
    B2.H1 = (a1 ^ aR1) & ~(e1 | eR1) & ownH;
    B2.V0 = (a0 ^ a1) & ~(e0 | e1);
    B2.V1 = (a1 ^ aB) & ~(e1 | eB) & ownV1;
    B2.N = (aN ^ a0) & ~(eN | e0) & ownN;
}


// The windows of RL cells (zgbm_shape_ok) by one warp: group g runs the cell
// at `at` (its own; `valid` false for a group without a cell) of replica R in
// the byte lattice src (== dst: ZGB updates in place), all of the same
// window. wsm: zgbm_warp_smem(RL) bytes of 16-byte aligned shared memory.
// Returns this group's events; *bad_out is set if a rank search found no
// member (never, unless the counts and masks disagree) or a window ran away.
template <int RL, bool PERSIST>
__device__ uint32_t zgbm_window(uint8_t *wsm, const Replica &R, const CellGeom &G, const CellAt &at, bool valid,
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
    uint2 *bln = reinterpret_cast<uint2 *>(wsm + RL * sizeof(Zgb32Const) + 2 * 32 * NP * 16);  // [class - 1][lane]

    // The lane's rows and their halo sites, loaded from global memory into
    // registers; local lane 0 also the halo row above the cell, the last row
    // lane the one below. hx: bit r (8 + r) set if row r's left halo site is
    // empty (holds A), bit 16 + r (24 + r) if its right halo site is.
    uint32_t e[RL], a[RL], eH = 0u, aH = 0u, hx = 0u;
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
        // this cell's classes: each lane's member counts (its row pairs
        // through zgbm_pair_bonds, its rows' left cross bonds), the totals and
        // the fixed-point rate sums
        uint32_t eB = __shfl_down_sync(FULLW, e[0], 1, W), aB = __shfl_down_sync(FULLW, a[0], 1, W);
        if (last) { eB = eH; aB = aH; }
        // the left cross bonds of the lane's rows (owned in E windows), bit r
        // for row r: its site 0 (gathered into ce, ca) and left halo site
        uint32_t ce = 0u, ca = 0u;
#pragma unroll
        for (int r = 0; r < RL; ++r) {
            ce = __funnelshift_r(ce, e[r], 1);
            ca = __funnelshift_r(ca, a[r], 1);
        }
        ce >>= 32 - RL;
        ca >>= 32 - RL;
        const uint32_t ownL = ew ? 0xFFu : 0u, hle = hx & 0xFFu, hla = (hx >> 8) & 0xFFu;
        const uint32_t lbits1 = hle & ce & ownL, lbits2 = (hla ^ ca) & ~(hle | ce) & ownL;
        // cl: the lane's member count of each class; pc: its count of class
        // k in row pair p (each below 256) at bit 8 (NP k + p) of the NP words
        int cl[4] = {0, 0, 0, 0};
        uint32_t pc[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) pc[i] = 0u;
        uint32_t n1 = 0u, n2 = 0u;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const int s0 = __popc(e[2 * p]) + __popc(e[2 * p + 1]), s3 = __popc(a[2 * p]) + __popc(a[2 * p + 1]);
            cl[0] += s0;
            cl[3] += s3;
            pc[0] += (uint32_t)s0 << (8 * p);
            pc[3 * NP / 4] += (uint32_t)s3 << (8 * (3 * NP + p) % 32);
        }
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            // rows 2p, 2p + 1; the row below is the lane's row 2p + 2, or the
            // next lane's row 0 (the bottom halo row in the last row lane)
            const uint32_t be = p < NP - 1 ? e[2 * p + 2] : eB, ba = p < NP - 1 ? a[2 * p + 2] : aB;
            ZgbmPair B1, B2;
            zgbm_pair_bonds(p == NP - 1 && last, p == 0 && first, ew, e[2 * p], a[2 * p], e[2 * p + 1], a[2 * p + 1],
                            be, ba, eH, aH, hx >> (16 + 2 * p), hx >> (24 + 2 * p), B1, B2);
            int c1 = __popc(B1.H0) + __popc(B1.H1) + __popc(B1.V0) + __popc(B1.V1) + __popc((lbits1 >> (2 * p)) & 3u);
            int c2 = __popc(B2.H0) + __popc(B2.H1) + __popc(B2.V0) + __popc(B2.V1) + __popc((lbits2 >> (2 * p)) & 3u);
            if (p == 0) {
                n1 = B1.N;
                n2 = B2.N;
                c1 += __popc(n1);
                c2 += __popc(n2);
            }
            cl[1] += c1;
            cl[2] += c2;
            pc[NP / 4] += (uint32_t)c1 << (8 * (NP + p) % 32);
            pc[2 * NP / 4] += (uint32_t)c2 << (8 * (2 * NP + p) % 32);
            bq[32 * p + lane] = make_uint4(B1.H0, B1.H1, B1.V0, B1.V1);  // lane-contiguous: no bank conflicts
            bq[32 * NP + 32 * p + lane] = make_uint4(B2.H0, B2.H1, B2.V0, B2.V1);
        }
        bln[lane] = make_uint2(lbits1, n1);
        bln[32 + lane] = make_uint2(lbits2, n2);
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
        const int c = k == 0 ? cl[0] : (k == 1 ? cl[1] : (k == 2 ? cl[2] : cl[3]));
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
            uint32_t s0 = 0u, s1 = 0u;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                if (p == q) {
                    s0 = k == 0 ? e[2 * q] : a[2 * q];
                    s1 = k == 0 ? e[2 * q + 1] : a[2 * q + 1];
                }
            }
            const int kb = site ? 0 : k - 1;
            const uint4 qv = bq[kb * 32 * NP + 32 * p + lane];
            const uint2 ln = bln[kb * 32 + lane];
            const uint32_t ms[7] = {site ? s0 : qv.x, site ? 0u : qv.z, site ? 0u : (ln.x >> (2 * p)) & 1u,
                                    (site || p != 0) ? 0u : ln.y, site ? s1 : qv.y, site ? 0u : qv.w,
                                    site ? 0u : (ln.x >> (2 * p + 1)) & 1u};
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
            } else if (kind == 3 && owner != nrl - 1 && l == owner + 1) {
                // the lower end of a vertical bond below the owner's last row
                // (unless the owner holds the cell's last row: the bottom halo
                // row, changed above)
                r1 = -1;
                mB = bit;
            }
#pragma unroll
            for (int q = 0; q < RL; ++q) {
                const uint32_t m = (r1 == q ? mA : 0u) | (r1 + 1 == q ? mB : 0u);
                e[q] = (e[q] & ~m) | (m & setE);
                a[q] = (a[q] & ~m) | (m & setA);
            }
            ++ev;
        }
    }

    // Write back: the cell's rows, and the owned halo ends (the halo columns
    // in E windows, the halo rows in O windows)
    if (row) {
        uint8_t *const out = C.dst;
        const int lx = C.lx, ly = C.ly, X0 = C.X0, Y0 = C.Y0;
        const int y0 = Y0 + RL * l;
#pragma unroll
        for (int r = 0; r < RL; ++r) zgb_store_row(out + (int64_t)(y0 + r) * lx + X0, e[r], a[r]);
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
