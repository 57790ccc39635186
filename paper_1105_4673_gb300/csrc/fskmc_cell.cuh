// One coarse cell's fractional window, one warp per cell (shared by the
// plain and persistent window kernels and the nested kernel).
//
// In a window of colour c and length h every cell of colour c runs its own
// serial SSA (Eqs. totalrate and skeleton) on its sites, reading neighbours
// outside its write set as they were when the window began (Section 2.2,
// Step 1 / Step 3). The cell's write set lives in shared memory for the whole
// window; the rate-class counts are exact integers kept incrementally; the
// chosen member is found by an integer rank search over per-lane membership
// bit masks (popcount, warp prefix scan, ballot).
#pragma once
#include <cuda/atomic>
#include <cuda_runtime.h>

#include "fskmc_device.cuh"
#include "fskmc_internal.h"
#include "philox.cuh"

namespace fskmc {

namespace {

struct Layout {
    int BW, BH, nsite, s, SW;
    int box_bytes, scls_bytes, sitemask_words, slotmask_words, rowmask_words;
    int bytes;
};

// 8x8 bit-matrix transpose (row r = byte r, column c = bit c) by three
// delta swaps.
__device__ __forceinline__ uint64_t transpose8(uint64_t x)
{
    uint64_t t;
    t = (x ^ (x >> 7)) & 0x00AA00AA00AA00AAull;
    x = x ^ t ^ (t << 7);
    t = (x ^ (x >> 14)) & 0x0000CCCC0000CCCCull;
    x = x ^ t ^ (t << 14);
    t = (x ^ (x >> 28)) & 0x00000000F0F0F0F0ull;
    x = x ^ t ^ (t << 28);
    return x;
}

// Per-site count n of occupied nearest neighbours (0..4) of a row of 32
// sites, from the occupancy masks of its four neighbours, as bit planes; eq[v]
// is the mask of sites with n == v.
__device__ __forceinline__ void count_eq(uint32_t up, uint32_t right, uint32_t down, uint32_t left,
                                         uint32_t eq[5])
{
    const uint32_t s1 = up ^ down, c1 = up & down, s2 = right ^ left, c2 = right & left;
    const uint32_t b0 = s1 ^ s2, k0 = s1 & s2;
    const uint32_t b1 = c1 ^ c2 ^ k0, b2 = (c1 & c2) | (k0 & (c1 ^ c2));
    eq[0] = ~b0 & ~b1 & ~b2;
    eq[1] = b0 & ~b1 & ~b2;
    eq[2] = ~b0 & b1 & ~b2;
    eq[3] = b0 & b1 & ~b2;
    eq[4] = ~b0 & ~b1 & b2;
}

// Slot-mask words of one lane from direction-major masks: D[d] bit t is slot
// (site t, d) of the lane's 32 sites; the canonical layout puts slot (t, d)
// at bit t*8 + d of the lane's 256-bit run (word t/4, byte t%4, bit d).
__device__ __forceinline__ void store_slot_words(const uint32_t D[8], uint32_t *words, int lane)
{
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        uint64_t m = 0;
#pragma unroll
        for (int d = 0; d < 8; ++d) m |= (uint64_t)((D[d] >> (8 * g)) & 0xFFu) << (8 * d);
        m = transpose8(m);
        words[(2 * g) * 32 + lane] = (uint32_t)m;
        words[(2 * g + 1) * 32 + lane] = (uint32_t)(m >> 32);
    }
}

// Per-warp shared memory: the cell and its halo (one byte per site), the
// class code of every own site, membership masks ([mask][word][lane]),
// then 16 class counts (int), 16 counts as binary64 and 16 fixed-point rates.
template <int MODEL>
__host__ __device__ inline Layout make_layout(int qx, int qy)
{
    using TR = Traits<MODEL>;
    Layout L;
    L.BW = qx + 2 * TR::HW;
    L.BH = qy + 2 * TR::HW;
    L.nsite = qx * qy;
    L.s = 32;                       // each lane owns one 32-site word of every site mask
    L.SW = TR::KB ? 8 : 0;          // and 8 words (32 sites x 8 slots) of every slot mask
    L.box_bytes = (L.BW * L.BH + 15) & ~15;
    L.scls_bytes = (L.nsite + 15) & ~15;
    L.sitemask_words = TR::KS * 32;
    L.slotmask_words = TR::KB * L.SW * 32;
    L.rowmask_words = MODEL == ZGB ? 3 * L.BH : (MODEL == DIFFUSION ? L.BH : 0);
    L.bytes = L.box_bytes + L.scls_bytes + 4 * (L.sitemask_words + L.slotmask_words) +
              4 * MAX_CLASSES + 8 * MAX_CLASSES + 8 * MAX_CLASSES + 4 * L.rowmask_words;
    L.bytes = (L.bytes + 15) & ~15;
    return L;
}

// Copy the sites of inactive cell (cx, cy) that no active cell writes in a
// window of colour col (ping-pong mode): columns 1..qx-2 of an O cell in E
// windows, rows 1..qy-2 of an E cell in O windows.
template <bool PERSIST>
__device__ void copy_unwritten(const uint8_t *src, uint8_t *dst, int lx, int ly, int qx, int qy,
                               int cx, int cy, int col, int lane)
{
    const int X0 = cx * qx, Y0 = cy * qy;
    if (qx == 32 && (lx & 31) == 0) {
        // 32-wide cells: one 32-byte row per lane (32-byte aligned), read as
        // two 16-byte words; E windows write its bytes 1..30 as aligned
        // 1-, 2-, 4- and 8-byte pieces, O windows rows 1..qy-2 whole
        const int r0 = col == 0 ? 0 : 1, r1 = col == 0 ? qy : qy - 1;
        for (int r = r0 + lane; r < r1; r += 32) {
            const int64_t o = (int64_t)(Y0 + r) * lx + X0;
            const uint4 *sp = reinterpret_cast<const uint4 *>(src + o);
            const uint4 a = PERSIST ? __ldcg(sp) : sp[0], b = PERSIST ? __ldcg(sp + 1) : sp[1];
            uint8_t *d = dst + o;
            if (col == 0) {
                d[1] = (uint8_t)(a.x >> 8);
                *reinterpret_cast<uint16_t *>(d + 2) = (uint16_t)(a.x >> 16);
                *reinterpret_cast<uint32_t *>(d + 4) = a.y;
                *reinterpret_cast<uint2 *>(d + 8) = make_uint2(a.z, a.w);
                *reinterpret_cast<uint2 *>(d + 16) = make_uint2(b.x, b.y);
                *reinterpret_cast<uint32_t *>(d + 24) = b.z;
                *reinterpret_cast<uint16_t *>(d + 28) = (uint16_t)b.w;
                d[30] = (uint8_t)(b.w >> 16);
            } else {
                reinterpret_cast<uint4 *>(d)[0] = a;
                reinterpret_cast<uint4 *>(d)[1] = b;
            }
        }
        return;
    }
    const int c0 = col == 0 ? 1 : 0, wdt = col == 0 ? qx - 2 : qx;  // columns c0 .. c0 + wdt - 1
    const int r0 = col == 0 ? 0 : 1, nrow = col == 0 ? qy : qy - 2;  // rows r0 .. r0 + nrow - 1
    if (wdt <= 0 || nrow <= 0) return;
    // walk the region in row-major steps of 32 without dividing by its width
    int r = r0, c = lane;
    while (c >= wdt) { c -= wdt; ++r; }
    for (int i = lane; i < wdt * nrow; i += 32) {
        const int64_t o = (int64_t)(Y0 + r) * lx + X0 + c0 + c;
        dst[o] = ld_site<PERSIST>(src + o);
        c += 32;
        while (c >= wdt) { c -= wdt; ++r; }
    }
}

// One cell's fractional window (Eqs. totalrate and skeleton run on the cell
// for the window length). Returns the number of events; *amb is set if an
// edge decision landed within about 1e-12 (relative) of the window end.
//
// CLK = double: the binary64 contract shared with the oracle -- lambda and
// the class thresholds P_k form the ordered fused multiply-add chain over
// the counts (as binary64) and the rates; the waiting time is
// -log(u_t)/lambda; comparisons of non-negative doubles are done on their
// bit patterns (same order, integer pipe).
// CLK = float: the rate-class sums are exact 64-bit fixed-point integers
// (counts times rates rounded to multiples of 2^-qshift), the class is the
// first k with (w2 * lambda_int) >> 32 < P_k, and only the window clock
// (lambda, waiting time, tau) is binary32 relative to the window start.
template <int MODEL, typename CLK, bool PERSIST, bool PACKED>
__device__ uint32_t cell_window(uint8_t *wsm, const Replica &R, const CellGeom &G, const CellAt &at,
                                int colour, uint32_t w, double hwin, bool screen, uint64_t seed,
                                const uint8_t *src, uint8_t *dst, int lane, bool *amb_out,
                                bool *bad_out, uint32_t *nexact_out)
{
    using TR = Traits<MODEL>;
    constexpr bool F64 = sizeof(CLK) == 8;
    constexpr int K = TR::K, HW = TR::HW, RR = TR::R;
    const int qx = G.qx, qy = G.qy;

    const Layout Lo = make_layout<MODEL>(qx, qy);
    uint8_t *box = wsm;
    uint8_t *scls = wsm + Lo.box_bytes;
    uint32_t *sitemask = reinterpret_cast<uint32_t *>(scls + Lo.scls_bytes);
    uint32_t *slotmask = sitemask + Lo.sitemask_words;
    int *cnt = reinterpret_cast<int *>(slotmask + Lo.slotmask_words);
    double *dcnt = reinterpret_cast<double *>(cnt + MAX_CLASSES);
    uint32_t *rowm = reinterpret_cast<uint32_t *>(dcnt + 2 * MAX_CLASSES);

    const int lx = at.lx, ly = at.ly;
    const uint32_t m = at.m;
    const int X0 = at.X0, Y0 = at.Y0;
    const int BW = Lo.BW, BH = Lo.BH, nsite = Lo.nsite;
    constexpr int SW = TR::KB ? 8 : 0;
    const int NL = (nsite + 31) >> 5;  // lanes that own sites

    // ZGB with 32-wide cells: rows are staged one per step so that warp
    // ballots give each row's state masks for the bit-parallel class build.
    const bool zrow = (MODEL == ZGB) && !PACKED && qx == 32;
    const bool drow = (MODEL == DIFFUSION) && qx == 32;
    if (drow || zrow) {
        // Every row of the box in flight at once: each row as four aligned
        // 16-byte chunks -- the 16 sites left of the cell, its 32 sites, the
        // 16 sites right of it -- copied asynchronously into a staging area
        // (the membership-mask region, not used yet), then read back one
        // site per lane for the box and the row ballots.
        // diffusion: halo columns x = -2, -1, 32, 33 in lanes 1..4; ZGB:
        // x = -1 in lane 1, x = 32 in lane 2
        const int hx = drow ? (lane <= 2 ? lane - 3 : 32 + (lane - 3)) : (lane == 1 ? -1 : 32);
        const bool hl = drow ? (lane >= 1 && lane <= 4) : (lane == 1 || lane == 2);
        uint8_t *raw = reinterpret_cast<uint8_t *>(sitemask);
        const int xl = X0 >= 16 ? X0 - 16 : X0 - 16 + lx;      // the chunk left of the cell
        const int xr = X0 + 32 < lx ? X0 + 32 : X0 + 32 - lx;  // and the one right of it
        for (int i = lane; i < 4 * BH; i += 32) {
            const int by = i >> 2, part = i & 3;
            int gy = Y0 - HW + by;
            gy += (gy < 0) ? ly : 0; gy -= (gy >= ly) ? ly : 0;
            const int gx = part == 0 ? xl : (part == 3 ? xr : X0 + 16 * (part - 1));
            cp_async16(raw + by * 64 + 16 * part, src + (int64_t)gy * lx + gx);
        }
        cp_async_wait_all();
        __syncwarp();
        for (int by = 0; by < BH; ++by) {
            const uint8_t *rr = raw + by * 64 + 16;  // rr[x]: site x of the row, -16 <= x < 48
            const uint32_t v = rr[lane];
            box[by * BW + HW + lane] = (uint8_t)v;
            if (hl) box[by * BW + HW + hx] = rr[hx];
            if (drow) {
                const uint32_t mo = __ballot_sync(0xffffffffu, v == 1u);
                if (lane == 0) rowm[by] = mo;
            } else {
                const uint32_t me = __ballot_sync(0xffffffffu, v == 0u);
                const uint32_t ma = __ballot_sync(0xffffffffu, v == 1u);
                const uint32_t mb = __ballot_sync(0xffffffffu, v == 2u);
                if (lane == 0) { rowm[by] = me; rowm[BH + by] = ma; rowm[2 * BH + by] = mb; }
            }
        }
    } else {
        // Stage the cell and its halo (periodic wrap) from the window-start
        // state; on the ring only the cell's own row (the rows above and
        // below are never read).
        constexpr bool ring = MODEL == ISING1D;
        // walk the box in row-major steps of 32 without dividing by its width
        int by = ring ? HW : 0, bx = lane;
        while (bx >= BW) { bx -= BW; ++by; }
        for (int i = lane; i < (ring ? BW : BW * BH); i += 32) {
            int gy = Y0 - HW + by, gx = X0 - HW + bx;
            gy += (gy < 0) ? ly : 0; gy -= (gy >= ly) ? ly : 0;
            gx += (gx < 0) ? lx : 0; gx -= (gx >= lx) ? lx : 0;
            const int bi = by * BW + bx;
            if (PACKED) {
                const uint32_t *w32 = reinterpret_cast<const uint32_t *>(src) + (int64_t)gy * (lx >> 5) + (gx >> 5);
                const uint32_t wv = PERSIST ? __ldcg(w32) : *w32;
                box[bi] = (uint8_t)((wv >> (gx & 31)) & 1u);
            } else {
                box[bi] = ld_site<PERSIST>(src + (int64_t)gy * lx + gx);
            }
            bx += 32;
            while (bx >= BW) { bx -= BW; ++by; }
        }
    }
    for (int i = lane; i < Lo.sitemask_words + Lo.slotmask_words; i += 32) sitemask[i] = 0u;
    if (lane < MAX_CLASSES) cnt[lane] = 0;
    __syncwarp();

    if (drow) {
        // Bit-parallel class build, one cell row per lane: every site's
        // occupied-neighbour count n comes from bit-sliced adders over the
        // neighbour rows; site classes are 5 sigma + n; a hop slot's class is
        // 10 + n(origin) when the origin is occupied and the target empty, its
        // origin being the site (outward) or the halo site (inward).
        if (lane < qy) {
            const int yb = lane + HW;
            const uint8_t *b0 = box + yb * BW + HW;          // this row, x = 0
            const uint8_t *bu = b0 - BW, *bd = b0 + BW;      // rows above and below
            const uint32_t o = rowm[yb], oN = rowm[yb - 1], oS = rowm[yb + 1];
            const uint32_t oNN = rowm[yb - 2], oSS = rowm[yb + 2];
            const uint32_t hl1 = b0[-1] == 1, hl2 = b0[-2] == 1, hr1 = b0[32] == 1, hr2 = b0[33] == 1;
            uint32_t oT[4];
            oT[0] = oN;
            oT[1] = (o >> 1) | (hr1 << 31);
            oT[2] = oS;
            oT[3] = (o << 1) | hl1;
            uint32_t eq[5];
            count_eq(oN, oT[1], oS, oT[3], eq);
            // the counts of the inward origins: the rows above / below the
            // cell (whole rows) and the halo sites left and right of this row
            uint32_t eqN[5], eqS[5];
            {
                const uint32_t rl = (oN << 1) | (uint32_t)(bu[-1] == 1), rr = (oN >> 1) | ((uint32_t)(bu[32] == 1) << 31);
                count_eq(oNN, rr, o, rl, eqN);
                const uint32_t sl = (oS << 1) | (uint32_t)(bd[-1] == 1), sr = (oS >> 1) | ((uint32_t)(bd[32] == 1) << 31);
                count_eq(o, sr, oSS, sl, eqS);
            }
            const int nW = (int)hl2 + (int)(o & 1u) + (bu[-1] == 1) + (bd[-1] == 1);  // origin x = -1
            const int nE = (int)(o >> 31) + (int)hr2 + (bu[32] == 1) + (bd[32] == 1);  // origin x = 32
            const bool ew = colour == 0;
            uint32_t own[8];
            own[0] = (lane > 0 || !ew) ? ~0u : 0u;
            own[1] = ew ? ~0u : 0x7FFFFFFFu;
            own[2] = (lane < qy - 1 || !ew) ? ~0u : 0u;
            own[3] = ew ? ~0u : 0xFFFFFFFEu;
            own[4] = (lane == 0 && !ew) ? ~0u : 0u;
            own[5] = ew ? 0x80000000u : 0u;
            own[6] = (lane == qy - 1 && !ew) ? ~0u : 0u;
            own[7] = ew ? 1u : 0u;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                uint32_t D[8];
#pragma unroll
                for (int d = 0; d < 4; ++d) D[d] = o & ~oT[d] & eq[c] & own[d];  // outward
                D[4] = ~o & oN & eqN[c] & own[4];                                  // from the row above
                D[5] = ~o & oT[1] & (nE == c ? 0x80000000u : 0u) & own[5];        // from x = 32
                D[6] = ~o & oS & eqS[c] & own[6];                                  // from the row below
                D[7] = ~o & oT[3] & (nW == c ? 1u : 0u) & own[7];                  // from x = -1
                store_slot_words(D, slotmask + (mask_of<MODEL>(10 + c) * SW) * 32, lane);
            }
#pragma unroll
            for (int n = 0; n < 5; ++n) {
                sitemask[n * 32 + lane] = ~o & eq[n];
                sitemask[(5 + n) * 32 + lane] = o & eq[n];
            }
            uint8_t *srow = scls + lane * 32;
#pragma unroll 8
            for (int t = 0; t < 32; ++t) {
                int n = 0;
#pragma unroll
                for (int v = 1; v < 5; ++v) n += ((eq[v] >> t) & 1u) * v;
                srow[t] = (uint8_t)(5 * ((o >> t) & 1u) + n);
            }
        }
        __syncwarp();
    } else if (zrow) {
        // Bit-parallel class build, one cell row per lane: site classes are
        // the row's empty / A masks; slot classes compare each site with its
        // neighbour in every direction (N, E, S, W outward, then inward), with
        // the ownership rule as masks, and are transposed into the canonical
        // site-major slot layout.
        if (lane < qy) {
            const int yb = lane + HW;
            const uint32_t e = rowm[yb], a = rowm[BH + yb], b = rowm[2 * BH + yb];
            const int hl = box[yb * BW], hr = box[yb * BW + BW - 1];
            uint32_t tE[4], tA[4], tB[4];
            tE[0] = rowm[yb - 1]; tA[0] = rowm[BH + yb - 1]; tB[0] = rowm[2 * BH + yb - 1];
            tE[2] = rowm[yb + 1]; tA[2] = rowm[BH + yb + 1]; tB[2] = rowm[2 * BH + yb + 1];
            tE[1] = (e >> 1) | ((uint32_t)(hr == 0) << 31);
            tA[1] = (a >> 1) | ((uint32_t)(hr == 1) << 31);
            tB[1] = (b >> 1) | ((uint32_t)(hr == 2) << 31);
            tE[3] = (e << 1) | (uint32_t)(hl == 0);
            tA[3] = (a << 1) | (uint32_t)(hl == 1);
            tB[3] = (b << 1) | (uint32_t)(hl == 2);
            const bool ew = colour == 0;  // horizontal cross bonds belong to E cells
            uint32_t own[8];
            own[0] = (lane > 0 || !ew) ? ~0u : 0u;
            own[1] = ew ? ~0u : 0x7FFFFFFFu;
            own[2] = (lane < qy - 1 || !ew) ? ~0u : 0u;
            own[3] = ew ? ~0u : 0xFFFFFFFEu;
            own[4] = (lane == 0 && !ew) ? ~0u : 0u;
            own[5] = ew ? 0x80000000u : 0u;
            own[6] = (lane == qy - 1 && !ew) ? ~0u : 0u;
            own[7] = ew ? 1u : 0u;
            uint32_t D1[8], D2[8];
#pragma unroll
            for (int d = 0; d < 8; ++d) {
                const int dir = d & 3;
                D1[d] = e & tE[dir] & own[d];                             // B2 adsorbs: both empty
                D2[d] = ((a & tB[dir]) | (b & tA[dir])) & own[d];         // A + B react
            }
            store_slot_words(D1, slotmask + (mask_of<MODEL>(1) * SW) * 32, lane);
            store_slot_words(D2, slotmask + (mask_of<MODEL>(2) * SW) * 32, lane);
            sitemask[mask_of<MODEL>(0) * 32 + lane] = e;
            sitemask[mask_of<MODEL>(3) * 32 + lane] = a;
            uint8_t *srow = scls + lane * 32;
#pragma unroll 8
            for (int t = 0; t < 32; ++t)
                srow[t] = ((e >> t) & 1u) ? 0 : (((a >> t) & 1u) ? 3 : 0xFF);
        }
        __syncwarp();
    } else {
        // Class build: each lane classifies its own run of 32 sites and their slots.
        const int i0 = lane * 32;
        for (int t = 0; t < 32; ++t) {
            int i = i0 + t;
            if (i >= nsite) break;
            int lly = (int)fdiv((uint32_t)i, G.fqx), llx = i - lly * qx;
            int p = (lly + HW) * BW + llx + HW;
            int k = site_class<MODEL>(box, BW, p);
            scls[i] = (uint8_t)k;
            if (k >= 0) sitemask[mask_of<MODEL>(k) * 32 + lane] |= 1u << t;
            if (TR::KB) {
    #pragma unroll
                for (int d = 0; d < 8; ++d) {
                    if (!slot_owned(llx, lly, d, qx, qy, colour)) continue;
                    int dir = d & 3;
                    int pn = p + dir_dy(dir) * BW + dir_dx(dir);
                    int kb = (d < 4) ? slot_class<MODEL>(box, BW, p, pn) : slot_class<MODEL>(box, BW, pn, p);
                    if (kb < 0) continue;
                    int bit = t * 8 + d;
                    slotmask[(mask_of<MODEL>(kb) * SW + (bit >> 5)) * 32 + lane] |= 1u << (bit & 31);
                }
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        int c = 0;
        if (is_slot<MODEL>(k)) {
            for (int wd = 0; wd < SW; ++wd) c += __popc(slotmask[(mask_of<MODEL>(k) * SW + wd) * 32 + lane]);
        } else {
            c = __popc(sitemask[mask_of<MODEL>(k) * 32 + lane]);
        }
        c = __reduce_add_sync(0xffffffffu, c);
        if (lane == 0) cnt[k] = c;
    }
    __syncwarp();

    // Per-lane class data: lane k < K holds class k's count and rate.
    double rk[K];  // binary64 rates (uniform)
#pragma unroll
    for (int k = 0; k < K; ++k) rk[k] = F64 ? R.r[k] : 0.0;
    const uint64_t rq_lane = lane < K ? R.rq[lane] : 0ull;
    const float qscale = R.qscale;

    const long long hbits = dbits(hwin);
    const float hf = (float)hwin;
    double tau = 0.0;
    float tauf = 0.0f;
    bool amb = false;
    uint32_t e = 0;
    uint32_t rw3 = 0;
    double rl = 0.0, ruc = 0.0;
    float rlf = 0.0f;
    uint32_t rw2 = 0;
    const uint32_t ctr3 = R.rep | (TAG_EVENT << 24);
    // Binary64 clock, plain kernel: window-edge decisions screened by a
    // binary32 estimate on an exact integer clock (edge_screen); the binary64
    // clock tau runs one draw batch (32 events) behind -- at each batch start
    // lane i divides event i's l by its lambda for the batch just ended, and
    // event i of the next batch adds that waiting time to tau, in event order
    // -- and decides the events the estimate cannot, after catching up a copy
    // of tau; once such an event is taken the window's remaining decisions
    // are taken the same way (with the screen off or a window length outside
    // its range: every decision). The persistent kernel, bound by issue and
    // occupancy, where the screen's registers cost more than its latency
    // saves, divides and adds in binary64 for every event before its class
    // choice.
    float sf = 0.0f;
    const bool screen_ok = !PERSIST && edge_screen_scale(hwin, screen, sf);
    uint64_t clk = 0, err = 0;
    double lam_mine = 1.0, lq_prev = 0.0;  // lane i: event i of the batch
    int ntaken_cur = 0, ntaken_prev = 0;   // events taken in this batch, in the previous one
    uint32_t nexact = 0;
    bool near_edge = false;

    for (;;) {
        // Counts of this state, one class per lane.
        const int n_lane = lane < K ? cnt[lane] : 0;
        double Pd[K];
        double lamd = 0.0;
        uint64_t P_lane = 0, lami = 0;
        if (F64) {
            if (lane < K) dcnt[lane] = (double)n_lane;  // one conversion per class, lane-parallel
            __syncwarp();
#pragma unroll
            for (int k = 0; k < K; ++k) {
                double nk = dcnt[k];
                if (dbits(nk) != 0) lamd = __fma_rn(nk, rk[k], lamd);  // fma(0, r, x) == x
                Pd[k] = lamd;
            }
            if (dbits(lamd) == 0) break;
        } else {
            // exact integer prefix sums over the classes (lanes 0..15)
            P_lane = (uint64_t)(uint32_t)n_lane * rq_lane;
#pragma unroll
            for (int off = 1; off < K; off <<= 1) {
                uint64_t v = __shfl_up_sync(0xffffffffu, P_lane, off);
                if (lane >= off) P_lane += v;
            }
            lami = __shfl_sync(0xffffffffu, P_lane, K - 1);
            if (lami == 0ull) break;
        }
        if (e >= MAX_EVENTS_PER_WINDOW) {  // cannot happen with sane rates; never loop unboundedly
            *bad_out = true;
            break;
        }
        if ((e & 31u) == 0u) {
            if (F64 && !PERSIST) {
                // binary64 waiting times of the batch just ended, one event per lane
                const bool mine = lane < ntaken_cur;
                lq_prev = div_rn(mine ? rl : 1.0, mine ? lam_mine : 1.0);
                ntaken_prev = ntaken_cur;
                ntaken_cur = 0;
            }
            // 32 events' draws at once, one Philox block per lane
            u32x4 o = draw(seed, e + (uint32_t)lane, w, (uint32_t)m, ctr3);
            if (F64) {
                uint64_t b = ((uint64_t)o.x << 21) | (uint64_t)(o.y >> 11);
                rl = neg_log_u53(b + 1ull);
                ruc = u53_scaled(2ull * o.z + 1ull, 33);  // (o.z + 1/2) 2^-32
                if (!PERSIST) rlf = __double2float_rz(rl);
            } else {
                rlf = -__logf(__fmul_rn(__uint2float_rn((o.x >> 8) + 1u), 0x1p-24f));
            }
            rw2 = o.z;
            rw3 = o.w;
        }
        const int src_lane = (int)(e & 31u);
        const uint32_t w3 = __shfl_sync(0xffffffffu, rw3, src_lane);
        int k;
        if (F64 && PERSIST) {
            const double l = __shfl_sync(0xffffffffu, rl, src_lane);
            const double uc = __shfl_sync(0xffffffffu, ruc, src_lane);
            const double end = __dadd_rn(tau, div_rn(l, lamd));
            const long long eb = dbits(end);
            if (llabs(eb - hbits) < 9008ll) amb = true;  // |end - h| below ~1e-12 h
            ++nexact;
            if (eb >= hbits) break;
            tau = end;
            const long long tb = dbits(__dmul_rn(uc, lamd));
            k = K - 1;
#pragma unroll
            for (int kk = K - 2; kk >= 0; --kk)
                if (tb < dbits(Pd[kk])) k = kk;
        } else if (F64) {
            {  // the binary64 clock, one batch behind
                const double v = __shfl_sync(0xffffffffu, lq_prev, src_lane);
                if (src_lane < ntaken_prev) tau = __dadd_rn(tau, v);
            }
            if (lane == src_lane) lam_mine = lamd;
            const double uc = __shfl_sync(0xffffffffu, ruc, src_lane);
            const float lf = __shfl_sync(0xffffffffu, rlf, src_lane);
            uint64_t Qs, Es;
            bool take, unsure;
            edge_screen(lf, lamd, sf, clk, err, screen_ok, near_edge, Qs, Es, take, unsure);
            const long long tb = dbits(__dmul_rn(uc, lamd));
            k = K - 1;
#pragma unroll
            for (int kk = K - 2; kk >= 0; --kk)
                if (tb < dbits(Pd[kk])) k = kk;
            if (unsure) {
                // binary64 decision: tau up to event e - 1 (the rest of the
                // previous batch, then this batch's events before e, all
                // taken), plus event e's waiting time
                double t = tau;
                for (int i = 1; i < 32; ++i) {
                    const double v = __shfl_sync(0xffffffffu, lq_prev, i);
                    if (i > src_lane && i < ntaken_prev) t = __dadd_rn(t, v);
                }
                const bool mine = lane <= src_lane;
                const double lqc = div_rn(mine ? rl : 1.0, mine ? lam_mine : 1.0);
                for (int i = 0; i < 31; ++i) {
                    const double v = __shfl_sync(0xffffffffu, lqc, i);
                    if (i < src_lane) t = __dadd_rn(t, v);
                }
                const double end = __dadd_rn(t, __shfl_sync(0xffffffffu, lqc, src_lane));
                const long long eb = dbits(end);
                if (llabs(eb - hbits) < 9008ll) amb = true;  // |end - h| below ~1e-12 h
                take = eb < hbits;
                near_edge = true;
                ++nexact;
            }
            if (!take) break;
            clk += Qs;
            err = Es;
            ++ntaken_cur;
        } else {
            const float l = __shfl_sync(0xffffffffu, rlf, src_lane);
            const uint32_t w2 = __shfl_sync(0xffffffffu, rw2, src_lane);
            const float lamf = __fmul_rn(u64_to_float_rz(lami), qscale);
            const float end = __fadd_rn(tauf, __fdividef(l, lamf));
            if (end >= hf) break;
            tauf = end;
            const uint64_t t = (uint64_t)w2 * (lami >> 32) + (((uint64_t)w2 * (lami & 0xffffffffull)) >> 32);
            const uint32_t hitc = __ballot_sync(0xffffffffu, lane < K && t < P_lane);
            k = __ffs(hitc) - 1;
        }
        const int nk = __shfl_sync(0xffffffffu, n_lane, k);
        const uint32_t j = (uint32_t)(((uint64_t)w3 * (uint64_t)(uint32_t)nk) >> 32);

        // Rank search: the j-th member of class k in canonical order.
        const bool slot = is_slot<MODEL>(k);
        const int mk = mask_of<MODEL>(k);
        int c = 0;
        if (slot) {
            for (int wd = 0; wd < SW; ++wd) c += __popc(slotmask[(mk * SW + wd) * 32 + lane]);
        } else {
            c = __popc(sitemask[mk * 32 + lane]);
        }
        int incl = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += v;
        }
        const uint32_t hit = __ballot_sync(0xffffffffu, (uint32_t)incl > j);
        if (hit == 0u) {  // counts and masks disagree: stop rather than write out of bounds
            *bad_out = true;
            break;
        }
        const int owner = __ffs(hit) - 1;
        int pick = 0;
        if (lane == owner) {
            int r = (int)j - (incl - c);
            if (slot) {
                for (int wd = 0; wd < SW; ++wd) {
                    uint32_t mw = slotmask[(mk * SW + wd) * 32 + lane];
                    int pc = __popc(mw);
                    if (r < pc) { pick = wd * 32 + select_bit(mw, r); break; }
                    r -= pc;
                }
            } else {
                pick = select_bit(sitemask[mk * 32 + lane], r);
            }
        }
        pick = __shfl_sync(0xffffffffu, pick, owner);
        int site, d = 0;
        if (slot) { site = owner * 32 + (pick >> 3); d = pick & 7; }
        else { site = owner * 32 + pick; }
        const int sy = (int)fdiv((uint32_t)site, G.fqx), sx = site - sy * qx;
        int ox = sx, oy = sy, tx = sx, ty = sy;
        if (slot) {
            int dir = d & 3;
            if (d < 4) { tx += dir_dx(dir); ty += dir_dy(dir); }
            else { ox += dir_dx(dir); oy += dir_dy(dir); }
        }
        const int po = (oy + HW) * BW + ox + HW, pt = (ty + HW) * BW + tx + HW;
        if (is_spin_flip<MODEL>()) {
            // Spin flip at (sx, sy): its class k = S sigma + n becomes k -+ S,
            // and each neighbour inside the cell changes n by +-1. The new
            // classes follow from the old ones; no lattice reads needed.
            // S = 5 with neighbours N, E, S, W (lanes 1..4); on the ring
            // S = 3 with neighbours E, W (lanes 1, 2).
            constexpr int SK = MODEL == ISING1D ? 3 : 5;
            const int sold = k >= SK;
            if (lane == 0) box[po] = (uint8_t)(1 - sold);
            if (lane < SK) {
                int ux = sx, uy = sy;
                if (MODEL == ISING1D) { ux += lane == 1 ? 1 : (lane == 2 ? -1 : 0); }
                else if (lane > 0) { ux += dir_dx(lane - 1); uy += dir_dy(lane - 1); }
                if (ux >= 0 && ux < qx && uy >= 0 && uy < qy) {
                    const int i = uy * qx + ux;
                    int kold, knew;
                    if (lane == 0) { kold = k; knew = sold ? k - SK : k + SK; }
                    else { kold = (int8_t)scls[i]; knew = kold + (sold ? -1 : 1); }
                    scls[i] = (uint8_t)knew;
                    const int own = i >> 5;
                    const uint32_t bit = 1u << (i & 31);
                    atomicAnd(&sitemask[kold * 32 + own], ~bit);
                    atomicOr(&sitemask[knew * 32 + own], bit);
                    atomicSub(&cnt[kold], 1);
                    atomicAdd(&cnt[knew], 1);
                }
            }
        } else {
            // Apply the event (the update sigma -> sigma^{x,omega}).
            if (lane == 0) {
                if (is_spin_flip<MODEL>()) {
                    box[po] ^= 1;
                } else if (MODEL == DIFFUSION) {
                    if (k < 10) box[po] ^= 1;
                    else { box[po] = 0; box[pt] = 1; }
                } else {
                    if (k == 0) box[po] = 1;
                    else if (k == 3) box[po] = 0;
                    else if (k == 1) { box[po] = 2; box[pt] = 2; }
                    else { box[po] = 0; box[pt] = 0; }
                }
            }
            __syncwarp();

            if (MODEL == ZGB) {
                // ZGB: a site's class depends only on its own state and a
                // slot's only on the states of its two ends, so only the
                // changed sites' classes and the slots with an end at a changed
                // site can change. Lanes 0-7 take the origin's four directions
                // (the two directed slots between it and that neighbour), lanes
                // 8-15 the target's (pair events; the bond between the two is
                // left to the origin's lanes), lanes 16 and 17 the two sites'
                // own classes.
                const int grp = lane < 8 ? 0 : (lane < 16 ? 1 : 2);
                const bool use_t = grp == 1 || lane == 17;
                const int cxl = use_t ? tx : ox, cyl = use_t ? ty : oy;  // the changed site
                const bool c_in = cxl >= 0 && cxl < qx && cyl >= 0 && cyl < qy;
                const bool live = grp == 0 || lane == 16 || (slot && (grp == 1 || lane == 17));
                if (grp == 2) {
                    if (live && c_in) {
                        const int i = cyl * qx + cxl;
                        const int knew = site_class<MODEL>(box, BW, (cyl + HW) * BW + cxl + HW);
                        const int kold = (int8_t)scls[i];
                        if (knew != kold) {
                            scls[i] = (uint8_t)knew;
                            const uint32_t bit = 1u << (i & 31);
                            if (kold >= 0) {
                                atomicAnd(&sitemask[mask_of<MODEL>(kold) * 32 + (i >> 5)], ~bit);
                                atomicSub(&cnt[kold], 1);
                            }
                            if (knew >= 0) {
                                atomicOr(&sitemask[mask_of<MODEL>(knew) * 32 + (i >> 5)], bit);
                                atomicAdd(&cnt[knew], 1);
                            }
                        }
                    }
                } else if (live) {
                    const int dir = (lane & 7) >> 1, half = lane & 1;
                    const int nx = cxl + dir_dx(dir), ny = cyl + dir_dy(dir);
                    const bool n_in = nx >= 0 && nx < qx && ny >= 0 && ny < qy;
                    const int opp = dir ^ 2;
                    // the directed slot (member site s, slot d): outward s -> s+dir(d)
                    // for d < 4, inward s+dir(d-4) -> s for d >= 4
                    int sx_, sy_, d;
                    bool any = true;
                    if (grp == 1 && nx == ox && ny == oy) any = false;  // the pair's own bond
                    if (c_in) {
                        if (half == 0) { sx_ = cxl; sy_ = cyl; d = dir; }
                        else if (n_in) { sx_ = nx; sy_ = ny; d = opp; }
                        else { sx_ = cxl; sy_ = cyl; d = 4 + dir; }
                    } else {
                        any = any && n_in;
                        sx_ = nx; sy_ = ny; d = half == 0 ? opp : 4 + opp;
                    }
                    if (any && slot_owned(sx_, sy_, d, qx, qy, colour)) {
                        const int i = sy_ * qx + sx_;
                        const int pu = (sy_ + HW) * BW + sx_ + HW;
                        const int dd = d & 3;
                        const int pn = pu + dir_dy(dd) * BW + dir_dx(dd);
                        const int kn = d < 4 ? slot_class<MODEL>(box, BW, pu, pn) : slot_class<MODEL>(box, BW, pn, pu);
                        const int bitpos = (i & 31) * 8 + d;
                        const int wofs = (bitpos >> 5) * 32 + (i >> 5);
                        const uint32_t bit = 1u << (bitpos & 31);
                        int ko = -1;
#pragma unroll
                        for (int mbk = 0; mbk < TR::KB; ++mbk)
                            if (slotmask[mbk * SW * 32 + wofs] & bit) ko = slot_class_of_mask<MODEL>(mbk);
                        if (kn != ko) {
                            if (ko >= 0) {
                                atomicAnd(&slotmask[mask_of<MODEL>(ko) * SW * 32 + wofs], ~bit);
                                atomicSub(&cnt[ko], 1);
                            }
                            if (kn >= 0) {
                                atomicOr(&slotmask[mask_of<MODEL>(kn) * SW * 32 + wofs], bit);
                                atomicAdd(&cnt[kn], 1);
                            }
                        }
                    }
                }
            } else {
            // Refresh the classes of every own site within RR of the changed
            // sites, one site per lane (fixed region widths: 4 for RR = 1; 6 or
            // 5 for RR = 2 depending on the pair's orientation).
            {
                const int x0 = min(ox, tx) - RR, y0 = min(oy, ty) - RR;
                const int x1 = max(ox, tx) + RR, y1 = max(oy, ty) + RR;
                int ux, uy;
                if (RR == 1) {
                    ux = x0 + (lane & 3);
                    uy = y0 + (lane >> 2);
                } else if (oy != ty) {
                    ux = x0 + lane % 5;
                    uy = y0 + lane / 5;
                } else {
                    ux = x0 + lane % 6;
                    uy = y0 + lane / 6;
                }
                if (ux <= x1 && uy <= y1 && ux >= 0 && ux < qx && uy >= 0 && uy < qy) {
                    const int i = uy * qx + ux;
                    const int own = i >> 5, tt = i & 31;
                    const int pu = (uy + HW) * BW + ux + HW;
                    const int knew = site_class<MODEL>(box, BW, pu);
                    const int kold = (int8_t)scls[i];
                    if (knew != kold) {
                        scls[i] = (uint8_t)knew;
                        const uint32_t bit = 1u << tt;
                        if (kold >= 0) {
                            atomicAnd(&sitemask[mask_of<MODEL>(kold) * 32 + own], ~bit);
                            atomicSub(&cnt[kold], 1);
                        }
                        if (knew >= 0) {
                            atomicOr(&sitemask[mask_of<MODEL>(knew) * 32 + own], bit);
                            atomicAdd(&cnt[knew], 1);
                        }
                    }
                    if (TR::KB) {
    #pragma unroll
                        for (int dd = 0; dd < 8; ++dd) {
                            if (!slot_owned(ux, uy, dd, qx, qy, colour)) continue;
                            const int dir = dd & 3;
                            const int pn = pu + dir_dy(dir) * BW + dir_dx(dir);
                            const int kn = (dd < 4) ? slot_class<MODEL>(box, BW, pu, pn)
                                                    : slot_class<MODEL>(box, BW, pn, pu);
                            const int bitpos = tt * 8 + dd;
                            const int wofs = (bitpos >> 5) * 32 + own;
                            const uint32_t bit = 1u << (bitpos & 31);
                            int ko = -1;
    #pragma unroll
                            for (int mb = 0; mb < TR::KB; ++mb)
                                if (slotmask[mb * SW * 32 + wofs] & bit) ko = slot_class_of_mask<MODEL>(mb);
                            if (kn == ko) continue;
                            if (ko >= 0) {
                                atomicAnd(&slotmask[mask_of<MODEL>(ko) * SW * 32 + wofs], ~bit);
                                atomicSub(&cnt[ko], 1);
                            }
                            if (kn >= 0) {
                                atomicOr(&slotmask[mask_of<MODEL>(kn) * SW * 32 + wofs], bit);
                                atomicAdd(&cnt[kn], 1);
                            }
                        }
                    }
                }
            }
            }
        }
        __syncwarp();
        ++e;
    }

    // Write back the write set: own sites, plus the halo ends of owned cross
    // bonds for the two-site models (columns in E windows, rows in O windows).
    if (PACKED) {
        // one (row, word) pair per lane; a word shared with other cells
        // (cells narrower than 32 sites) is updated with atomics on this
        // cell's bits only
        uint32_t *dst32 = reinterpret_cast<uint32_t *>(dst);
        const int wa = X0 >> 5, nwr = ((X0 + qx - 1) >> 5) - wa + 1;
        for (int t = lane; t < qy * nwr; t += 32) {
            const int row = t / nwr, wi = wa + (t - row * nwr);
            const uint8_t *brow = box + (row + HW) * BW + HW - X0;
            uint32_t *drow = dst32 + (int64_t)(Y0 + row) * (lx >> 5);
            const int xs = max(X0, wi << 5), xe = min(X0 + qx, (wi + 1) << 5);
            uint32_t mask = 0u, bits = 0u;
            for (int xx = xs; xx < xe; ++xx) {
                const uint32_t b = 1u << (xx & 31);
                mask |= b;
                if (brow[xx]) bits |= b;
            }
            if (mask == 0xffffffffu) {
                drow[wi] = bits;
            } else {
                atomicAnd(drow + wi, ~mask);
                atomicOr(drow + wi, bits);
            }
        }
    } else if (zrow) {
        // 32-wide ZGB cells: lane L writes row L in two 16-byte stores, its
        // bytes rebuilt from the row's own-site class masks (empty = class 0,
        // A = class 3, B = neither), which the events keep current
        if (lane < qy) {
            const uint32_t am = sitemask[mask_of<MODEL>(3) * 32 + lane];
            const uint32_t bm = ~(sitemask[mask_of<MODEL>(0) * 32 + lane] | am);
            uint32_t wv[8];
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                // 4 mask bits -> 4 bytes of 0/1 (bit k to bit 8k by one multiply)
                const uint32_t ea = (((am >> (4 * g)) & 0xFu) * 0x00204081u) & 0x01010101u;
                const uint32_t eb = (((bm >> (4 * g)) & 0xFu) * 0x00204081u) & 0x01010101u;
                wv[g] = ea + 2u * eb;
            }
            uint4 *d = reinterpret_cast<uint4 *>(dst + (int64_t)(Y0 + lane) * lx + X0);
            d[0] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
            d[1] = make_uint4(wv[4], wv[5], wv[6], wv[7]);
        }
    } else {
        for (int i = lane; i < nsite; i += 32) {
            int lly = (int)fdiv((uint32_t)i, G.fqx), llx = i - lly * qx;
            dst[(int64_t)(Y0 + lly) * lx + X0 + llx] = box[(lly + HW) * BW + llx + HW];
        }
    }
    if (TR::KB) {
        if (colour == 0) {
            for (int i = lane; i < 2 * qy; i += 32) {
                int lly = i >> 1, side = i & 1;
                int bx = side ? HW + qx : HW - 1;
                int gx = side ? (X0 + qx) % lx : (X0 - 1 + lx) % lx;
                dst[(int64_t)(Y0 + lly) * lx + gx] = box[(lly + HW) * BW + bx];
            }
        } else {
            for (int i = lane; i < 2 * qx; i += 32) {
                int llx = i >> 1, side = i & 1;
                int by = side ? HW + qy : HW - 1;
                int gy = side ? (Y0 + qy) % ly : (Y0 - 1 + ly) % ly;
                dst[(int64_t)gy * lx + X0 + llx] = box[by * BW + llx + HW];
            }
        }
    }
    *amb_out = amb;
    *nexact_out = nexact;
    return e;
}

}  // namespace

}  // namespace fskmc
