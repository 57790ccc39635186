// Grouped window kernels for the spin-flip models with small cells: one warp
// runs 32/W cells of the same window at once, W lanes per cell (4, 8 or 16:
// the lanes that own the cell's 32-site words, rounded up to a power of two,
// and at least the lanes one flip's class refresh uses: 5 in 2D, 3 on a ring).
//
// Why: a cell's serial SSA (Eqs. totalrate and skeleton) is a chain of
// warp-uniform steps -- the class sums, the waiting time, the class choice --
// and on GB300 an FP64 warp instruction costs the FP64 pipe the same whether
// one lane or 32 execute it (the issue slot likewise). A 16x16 cell has 256
// sites, 8 lanes' worth of 32-site words, so a one-cell warp leaves 24 lanes
// idle in every step. Here the cells of a warp share every instruction.
//
// The groups of a warp run in lockstep: every loop iteration executes one
// event of each group whose window is still running; a group whose window
// has ended (waiting time past the edge, no rate left) stays in the loop
// with its side effects switched off until every group is done. Each group's
// draws, arithmetic and member order are exactly those of the one-cell
// kernel (fskmc_window.cu), so results are bit-identical to it and to the
// oracle: the same Philox counters (event index, window, cell, replica), the
// same ordered binary64 fused multiply-add chain or exact fixed-point sums,
// the same rank search in canonical (lane-major) order.
//
// Cells in a warp are independent: they are same-colour cells of one window
// (Eq. exact: their generators commute), each with its own shared-memory
// region; only warp-wide votes and width-W shuffles are shared.
#pragma once
#include <cuda/atomic>
#include <cuda_runtime.h>

#include "fskmc_device.cuh"
#include "fskmc_internal.h"

namespace fskmc {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// Per-cell shared memory: the cell and its halo (one byte per site), the
// class code of every own site, KS x W membership words (word l of class k
// holds sites 32l .. 32l+31, owned by lane l), 16 class counts, the counts
// as binary64, and per box row three bit words (the row's cell sites, its
// left and its right halo site; 16-wide cells of a byte lattice). Cells are
// spaced a multiple of 128 bytes plus W words apart, so the cells' words at
// the same offset fall in different banks.
struct GLayout {
    int BW, BH, nsite;
    int scls_off, mask_off, cnt_off, dcnt_off, rowb_off;
    int stride;
};

template <int MODEL>
__host__ __device__ inline GLayout make_glayout(int qx, int qy, int W)
{
    using TR = Traits<MODEL>;
    GLayout L;
    L.BW = qx + 2 * TR::HW;
    L.BH = qy + 2 * TR::HW;
    L.nsite = qx * qy;
    int o = (L.BW * L.BH + 15) & ~15;
    L.scls_off = o;
    o += (L.nsite + 15) & ~15;
    L.mask_off = o;
    o += 4 * TR::KS * W;
    L.cnt_off = o;
    o += 4 * MAX_CLASSES;
    L.dcnt_off = o;
    o += 8 * MAX_CLASSES;
    L.rowb_off = o;
    o += 12 * L.BH;
    L.stride = ((o + 127) & ~127) + 4 * W;
    return L;
}

// One group's fractional window (W lanes; every lane of the warp calls this
// together). valid = the group has a cell. Outputs (group-uniform): events,
// whether an edge decision was ambiguous, whether a consistency check failed,
// how many edge decisions the screened binary64 check left to the binary64
// clock.
// The class data are lane-parallel: lane l holds classes l, l + W, ... for
// the fixed-point prefix sums (width-W shuffle scans), converts their counts
// to binary64 for the ordered fused multiply-add chain (which every lane then
// runs), and owns membership word l for the rank search.
template <int MODEL, typename CLK, bool PERSIST, bool PACKED, int W>
__device__ void group_window(uint8_t *csm, const GLayout &Lo, const Replica &R, const CellGeom &G,
                             bool valid, const CellAt &at, uint32_t w, double hwin, bool screen, uint64_t seed,
                             const uint8_t *src, uint8_t *dst, int lane, uint32_t *ev_out,
                             bool *amb_out, bool *bad_out, uint32_t *nexact_out)
{
    using TR = Traits<MODEL>;
    static_assert(is_spin_flip<MODEL>(), "grouped cells are built for the spin-flip models");
    constexpr bool F64 = sizeof(CLK) == 8;
    constexpr int K = TR::K, HW = TR::HW;
    constexpr int CPL = (K + W - 1) / W;  // classes per lane: lane l holds classes l, l + W, ...
    constexpr bool ring = MODEL == ISING1D;
    constexpr int SK = ring ? 3 : 5;      // class stride of sigma; lanes refreshing one flip
    static_assert(W >= SK && W < 32, "a group needs a lane per refreshed site");
    const int gl = lane & (W - 1);
    const int gshift = lane & ~(W - 1);
    const uint32_t gbits = (1u << W) - 1u;
    const int qx = G.qx, qy = G.qy;
    const int BW = Lo.BW, BH = Lo.BH, nsite = Lo.nsite;
    const int NL = (nsite + 31) >> 5;  // lanes that own sites (<= W)
    uint8_t *box = csm;
    uint8_t *scls = csm + Lo.scls_off;
    uint32_t *mask = reinterpret_cast<uint32_t *>(csm + Lo.mask_off);
    int *cnt = reinterpret_cast<int *>(csm + Lo.cnt_off);
    double *dcnt = reinterpret_cast<double *>(csm + Lo.dcnt_off);
    uint32_t *rowb = reinterpret_cast<uint32_t *>(csm + Lo.rowb_off);  // [box row][cell, left, right]

    const int lx = at.lx, ly = at.ly;
    const uint32_t m = at.m;
    const int X0 = at.X0, Y0 = at.Y0;

    // Stage the cell and its halo (periodic wrap) from the window-start
    // state; on the ring only the cell's own row.
    const bool rows16 = !PACKED && (qx & 15) == 0 && (lx & 15) == 0 && (X0 & 15) == 0;
    // 16-wide cells of a byte lattice in 2D: the staging also records every
    // box row as bits, and the class build works on whole rows of bits
    const bool rowbits = rows16 && !ring && qx == 16;
    if (valid && rows16) {
        // byte lattice, cell width a multiple of 16: each box row is qx/16
        // aligned 16-byte chunks of the cell's row plus its two halo sites;
        // items (row, chunk or halo) in row-major steps of W, UB16 loads in
        // flight per lane before their stores
        constexpr int UB16 = F64 ? 8 : 2;  // the binary32 kernels keep their registers low (occupancy)
        const int nch = qx >> 4, per_row = nch + 2;
        const int total = (ring ? 1 : BH) * per_row;
        int by = ring ? HW : 0, c = gl;
        while (c >= per_row) { c -= per_row; ++by; }
        for (int i0 = gl; i0 < total; i0 += UB16 * W) {
            uint4 v[UB16];
            int bi[UB16], kind[UB16], rw[UB16];
#pragma unroll
            for (int u = 0; u < UB16; ++u) {
                kind[u] = -1;  // -1 none, 0 chunk, 1 halo site
                bi[u] = 0;
                rw[u] = 3 * by + (c < nch ? 0 : (c == nch ? 1 : 2));
                v[u] = make_uint4(0u, 0u, 0u, 0u);
                if (i0 + u * W < total) {
                    int gy = Y0 - HW + by;
                    gy += (gy < 0) ? ly : 0; gy -= (gy >= ly) ? ly : 0;
                    const uint8_t *row = src + (int64_t)gy * lx;
                    if (c < nch) {
                        const uint4 *p16 = reinterpret_cast<const uint4 *>(row + X0 + 16 * c);
                        v[u] = PERSIST ? __ldcg(p16) : *p16;
                        bi[u] = by * BW + HW + 16 * c;
                        kind[u] = 0;
                    } else {
                        int gx = c == nch ? X0 - 1 : X0 + qx;
                        gx += (gx < 0) ? lx : 0; gx -= (gx >= lx) ? lx : 0;
                        v[u].x = ld_site<PERSIST>(row + gx);
                        bi[u] = by * BW + (c == nch ? 0 : HW + qx);
                        kind[u] = 1;
                    }
                }
                c += W;
                while (c >= per_row) { c -= per_row; ++by; }
            }
#pragma unroll
            for (int u = 0; u < UB16; ++u) {
                if (kind[u] == 0) {
                    const uint32_t wv[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
                    for (int b = 0; b < 16; ++b) box[bi[u] + b] = (uint8_t)(wv[b >> 2] >> (8 * (b & 3)));
                    if (rowbits) {
                        // the chunk's 16 sites (states 0/1) as bits 1..16 of the
                        // box row: one multiply gathers a word's four bytes
                        uint32_t m16 = 0u;
#pragma unroll
                        for (int q4 = 0; q4 < 4; ++q4)
                            m16 |= ((((wv[q4] & 0x01010101u) * 0x00204081u) >> 21) & 0xFu) << (4 * q4);
                        rowb[rw[u]] = m16 << HW;
                    }
                } else if (kind[u] == 1) {
                    box[bi[u]] = (uint8_t)v[u].x;
                    if (rowbits) rowb[rw[u]] = (v[u].x & 1u) << (rw[u] % 3 == 1 ? 0 : HW + qx);
                }
            }
        }
    } else if (valid) {
        // walk the box in row-major steps of W without dividing by its width,
        // UB loads in flight per lane before their stores (fewer in the
        // binary32 kernels, which keep their registers low)
        constexpr int UB = F64 ? 8 : 4;
        const int total = ring ? BW : BW * BH;
        int by = ring ? HW : 0, bx = gl;
        while (bx >= BW) { bx -= BW; ++by; }
        for (int i0 = gl; i0 < total; i0 += UB * W) {
            uint32_t v[UB];
            int bi[UB], sh[UB];
#pragma unroll
            for (int u = 0; u < UB; ++u) {
                bi[u] = -1;
                v[u] = 0u;
                sh[u] = 0;
                if (i0 + u * W < total) {
                    int gy = Y0 - HW + by, gx = X0 - HW + bx;
                    gy += (gy < 0) ? ly : 0; gy -= (gy >= ly) ? ly : 0;
                    gx += (gx < 0) ? lx : 0; gx -= (gx >= lx) ? lx : 0;
                    bi[u] = by * BW + bx;
                    if (PACKED) {
                        const uint32_t *w32 = reinterpret_cast<const uint32_t *>(src) + (int64_t)gy * (lx >> 5) + (gx >> 5);
                        v[u] = PERSIST ? __ldcg(w32) : *w32;
                        sh[u] = gx & 31;
                    } else {
                        v[u] = ld_site<PERSIST>(src + (int64_t)gy * lx + gx);
                    }
                }
                bx += W;
                while (bx >= BW) { bx -= BW; ++by; }
            }
#pragma unroll
            for (int u = 0; u < UB; ++u)
                if (bi[u] >= 0) box[bi[u]] = (uint8_t)(PACKED ? (v[u] >> sh[u]) & 1u : v[u]);
        }
    }
    for (int i = gl; i < MAX_CLASSES; i += W) cnt[i] = 0;  // a cell-less group keeps zero rates
    __syncwarp();

    // Class build: lane gl classifies its run of 32 sites (word gl; words
    // past the cell's last site are zero). The class of a site is
    // SK sigma + n (n = occupied neighbours: 4 in 2D, 2 on the ring; the
    // states are 0/1, so n is the sum of the neighbours' bytes); the lane
    // gathers sigma and the three bits of n as bit planes over its sites and
    // forms each class's membership word from them.
    if (valid && rowbits) {
        // lane gl's word holds cell rows 2 gl and 2 gl + 1: their states and
        // the bit-sliced count of their occupied neighbours from box rows
        // 2 gl .. 2 gl + 3 (rows past the box are empty; their sites lie
        // past the cell and are masked off)
        uint32_t ps = 0u, p0 = 0u, p1 = 0u, p2 = 0u;
        const int i0 = gl * 32;
        const int nt = min(32, nsite - i0);
        if (nt > 0) {
            uint32_t rb[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int b = 2 * gl + r;
                rb[r] = b < BH ? (rowb[3 * b] | rowb[3 * b + 1] | rowb[3 * b + 2]) : 0u;
            }
            uint32_t sN = 0u, sS = 0u, sW = 0u, sE = 0u;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                ps |= ((rb[r + 1] >> 1) & 0xFFFFu) << (16 * r);
                sN |= ((rb[r] >> 1) & 0xFFFFu) << (16 * r);
                sS |= ((rb[r + 2] >> 1) & 0xFFFFu) << (16 * r);
                sW |= (rb[r + 1] & 0xFFFFu) << (16 * r);
                sE |= ((rb[r + 1] >> 2) & 0xFFFFu) << (16 * r);
            }
            // n = N + S + W + E, bit by bit: two half adders, then the carries
            const uint32_t a1 = sN ^ sS, c1 = sN & sS, a2 = sW ^ sE, c2 = sW & sE;
            const uint32_t c3 = a1 & a2;
            p0 = a1 ^ a2;
            p1 = c1 ^ c2 ^ c3;
            p2 = c1 & c2;
            // the class bytes, four sites per store: SK sigma + n
#pragma unroll
            for (int t4 = 0; t4 < 8; ++t4) {
                if (4 * t4 < nt) {
                    const auto e4 = [t4](uint32_t x) { return (((x >> (4 * t4)) & 0xFu) * 0x00204081u) & 0x01010101u; };
                    *reinterpret_cast<uint32_t *>(scls + i0 + 4 * t4) =
                        (uint32_t)SK * e4(ps) + e4(p0) + 2u * e4(p1) + 4u * e4(p2);
                }
            }
        }
        const uint32_t vm = nt >= 32 ? 0xffffffffu : (nt > 0 ? (1u << nt) - 1u : 0u);
#pragma unroll
        for (int kk = 0; kk < TR::KS; ++kk) {
            const int sg = kk / SK, v = kk % SK;
            uint32_t mk = vm & (sg ? ps : ~ps);
            mk &= (v & 1) ? p0 : ~p0;
            mk &= (v & 2) ? p1 : ~p1;
            mk &= (v & 4) ? p2 : ~p2;
            mask[kk * W + gl] = mk;
        }
    } else if (valid) {
        uint32_t ps = 0u, p0 = 0u, p1 = 0u, p2 = 0u;
        const int i0 = gl * 32;
        const int nt = min(32, nsite - i0);  // sites of this word (none past the cell's last)
        int lly = (int)fdiv((uint32_t)i0, G.fqx), llx = i0 - lly * qx;
#pragma unroll 4
        for (int t = 0; t < nt; ++t) {
            const int p = (lly + HW) * BW + llx + HW;
            const uint32_t s = box[p];
            const uint32_t n = ring ? (uint32_t)box[p - 1] + box[p + 1]
                                    : (uint32_t)box[p - BW] + box[p + BW] + box[p - 1] + box[p + 1];
            scls[i0 + t] = (uint8_t)(SK * s + n);
            ps |= s << t;
            p0 |= (n & 1u) << t;
            p1 |= ((n >> 1) & 1u) << t;
            p2 |= (n >> 2) << t;
            if (++llx == qx) { llx = 0; ++lly; }
        }
        const uint32_t vm = nt >= 32 ? 0xffffffffu : (nt > 0 ? (1u << nt) - 1u : 0u);
#pragma unroll
        for (int kk = 0; kk < TR::KS; ++kk) {
            const int sg = kk / SK, v = kk % SK;
            uint32_t mk = vm & (sg ? ps : ~ps);
            mk &= (v & 1) ? p0 : ~p0;
            mk &= (v & 2) ? p1 : ~p1;
            mk &= (v & 4) ? p2 : ~p2;
            mask[kk * W + gl] = mk;
        }
    }
    __syncwarp();
    if (valid) {
#pragma unroll
        for (int s = 0; s < CPL; ++s) {
            const int k = gl + W * s;
            if (k < K) {
                int c = 0;
                for (int l = 0; l < NL; ++l) c += __popc(mask[k * W + l]);
                cnt[k] = c;
            }
        }
    }
    __syncwarp();

    double rk[K];
#pragma unroll
    for (int k = 0; k < K; ++k) rk[k] = F64 ? R.r[k] : 0.0;
    uint64_t rq[CPL];
#pragma unroll
    for (int s = 0; s < CPL; ++s) {
        const int k = gl + W * s;
        rq[s] = (!F64 && k < K) ? R.rq[k] : 0ull;
    }
    const float qscale = R.qscale;
    const long long hbits = dbits(hwin);
    const float hf = (float)hwin;
    double tau = 0.0;
    float tauf = 0.0f;
    bool act = valid, amb = false, bad = false;
    uint32_t ev = 0;
    uint32_t rw2 = 0, rw3 = 0;
    double rl = 0.0, ruc = 0.0;
    float rlf = 0.0f;
    const uint32_t ctr3 = R.rep | (TAG_EVENT << 24);

    // Binary64 clock, screened edge check. Each event's window-edge
    // decision (end = tau + (-log u_t) / lambda against h) is taken from a
    // bounded estimate that needs no binary64 divide: the waiting time in
    // binary32 (l rounded toward zero over lambda truncated to binary32, a
    // reciprocal within one unit in the last place, three rounded products:
    // at most 4.5 2^-23 relative error) on an exact 64-bit integer clock in
    // units of h 2^-62, with a running bound E on its distance from the
    // binary64 clock (2^-20 of each estimate, plus 2^11 units per event for
    // the integer truncation and the binary64 roundings). An event is taken
    // if clock + estimate + E < 2^62 and refused if clock + estimate >=
    // 2^62 + E: the binary64 decision in both cases. The binary64 clock tau
    // itself runs W events behind, off the critical path: at the start of
    // each batch of W events, lane i divides event i's l by its lambda for
    // the batch just ended, and iteration i of the next batch adds that
    // waiting time to tau, in event order. An event the estimate cannot
    // decide (an end within about 2^-20 h of the edge, lambda outside the
    // binary32 range, or screening off; about one per thousand cell-windows
    // at 16x16 Ising cells and 369 events per window) catches up a
    // copy of tau and decides in binary64 on the spot; once such an event is
    // taken, so are the group's remaining decisions of the window (the
    // integer clock may then stand past 2^62).
    float sf;
    const bool screen_ok = edge_screen_scale(hwin, screen, sf);
    uint64_t clk = 0, err = 0;
    double lam_mine = 1.0, lq_prev = 0.0;  // lane i: event i of the batch
    int ntaken_cur = 0, ntaken_prev = 0;   // events taken in this batch, in the previous one
    uint32_t nexact = 0;
    bool near_edge = false;

    // Every running group executes event e in iteration e, so e is the same
    // for all of them and the draw batches stay aligned. The persistent
    // kernel, which keeps many warps per SM busy and is bound by issue, asks
    // whether any group is still running once per iteration, after the
    // window-edge checks, so that the last iteration of a window stops
    // before its class choice and rank search; the plain kernel, bound by
    // the latency of one warp's chain, asks at the top.
    for (uint32_t e = 0;; ++e) {
        if (!PERSIST && !__any_sync(FULL, act)) break;
        double Pd[K];
        double lamd = 0.0;
        uint64_t P[CPL];
        uint64_t lami = 0;
        if (F64) {
            if (PERSIST) {
#pragma unroll
                for (int s = 0; s < CPL; ++s) {
                    const int k = gl + W * s;
                    if (k < K) dcnt[k] = small_to_double(cnt[k]);  // one conversion per class, lane-parallel
                }
                __syncwarp();
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    lamd = __fma_rn(dcnt[k], rk[k], lamd);  // fma(0, r, x) == x
                    Pd[k] = lamd;
                }
            } else {
                // every lane converts all counts itself: fewer steps before the chain
                int cc[MAX_CLASSES];
#pragma unroll
                for (int q4 = 0; q4 < MAX_CLASSES; q4 += 4) {
                    const int4 v = *reinterpret_cast<const int4 *>(cnt + q4);
                    cc[q4] = v.x; cc[q4 + 1] = v.y; cc[q4 + 2] = v.z; cc[q4 + 3] = v.w;
                }
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    lamd = __fma_rn(small_to_double(cc[k]), rk[k], lamd);
                    Pd[k] = lamd;
                }
            }
            if (dbits(lamd) == 0) act = false;
        } else {
            // exact integer prefix sums in class order: a width-W scan per
            // class slot (over the slot's nc classes only: its last slot may
            // hold fewer than W), then the slots' running bases
#pragma unroll
            for (int s = 0; s < CPL; ++s) {
                const int k = gl + W * s;
                constexpr int nc_last = K - W * (CPL - 1);
                const int nc = s < CPL - 1 ? W : nc_last;
                P[s] = (uint64_t)(k < K ? (uint32_t)cnt[k] : 0u) * rq[s];
#pragma unroll
                for (int off = 1; off < W; off <<= 1) {
                    if (off < nc) {
                        const uint64_t v = __shfl_up_sync(FULL, P[s], off, W);
                        if (gl >= off) P[s] += v;
                    }
                }
            }
#pragma unroll
            for (int s = 0; s < CPL; ++s) {
                const int nc = s < CPL - 1 ? W : K - W * (CPL - 1);
                const uint64_t tot = __shfl_sync(FULL, P[s], nc - 1, W);
                P[s] += lami;
                lami += tot;
            }
            if (lami == 0ull) act = false;
        }
        if (e >= MAX_EVENTS_PER_WINDOW) {  // cannot happen with sane rates; never loop unboundedly
            bad = bad || act;
            act = false;
        }
        const int sl = (int)(e & (uint32_t)(W - 1));
        if (sl == 0) {
            if (F64) {
                // binary64 waiting times of the batch just ended, one event per lane
                const bool mine = gl < ntaken_cur;
                lq_prev = div_rn(mine ? rl : 1.0, mine ? lam_mine : 1.0);
                ntaken_prev = ntaken_cur;
                ntaken_cur = 0;
            }
            // W events' draws at once, one Philox block per lane
            const u32x4 o = draw(seed, e + (uint32_t)gl, w, (uint32_t)m, ctr3);
            if (F64) {
                const uint64_t b = ((uint64_t)o.x << 21) | (uint64_t)(o.y >> 11);
                rl = neg_log_u53(b + 1ull);
                ruc = u53_scaled(2ull * o.z + 1ull, 33);  // (o.z + 1/2) 2^-32
                rlf = __double2float_rz(rl);
            } else {
                rlf = -__logf(__fmul_rn(__uint2float_rn((o.x >> 8) + 1u), 0x1p-24f));
            }
            rw2 = o.z;
            rw3 = o.w;
        }
        const uint32_t w3 = __shfl_sync(FULL, rw3, sl, W);
        // The class, the member and the window-edge check of event e: the
        // edge estimate has no data dependence on the class choice and the
        // rank search, so the three interleave; the edge check is applied
        // before anything is written.
        int k;
        uint64_t Qs = 0, Es = 0;
        bool take = false, unsure = false;
        if (F64) {
            {  // the binary64 clock, W events behind
                const double v = __shfl_sync(FULL, lq_prev, sl, W);
                if (sl < ntaken_prev) tau = __dadd_rn(tau, v);
            }
            if (gl == sl) lam_mine = lamd;
            const double uc = __shfl_sync(FULL, ruc, sl, W);
            const float lf = __shfl_sync(FULL, rlf, sl, W);
            edge_screen(lf, lamd, sf, clk, err, screen_ok, near_edge, Qs, Es, take, unsure);
            if (PERSIST) {
                if (!take && !unsure) act = false;  // the event lies past the edge
                if (!__any_sync(FULL, act)) break;
            }
            const long long tb = dbits(__dmul_rn(uc, lamd));
            k = 0;
#pragma unroll
            for (int kk = 0; kk < K - 1; ++kk) k += dbits(Pd[kk]) <= tb ? 1 : 0;  // P is non-decreasing
        } else {
            const float lf = __shfl_sync(FULL, rlf, sl, W);
            const uint32_t w2 = __shfl_sync(FULL, rw2, sl, W);
            const float lamf = lami ? __fmul_rn(u64_to_float_rz(lami), qscale) : 0.0f;
            const float end = __fadd_rn(tauf, __fdividef(lf, lamf));
            if (end >= hf) act = false;
            if (act) tauf = end;
            if (PERSIST && !__any_sync(FULL, act)) break;
            const uint64_t t = (uint64_t)w2 * (lami >> 32) + (((uint64_t)w2 * (lami & 0xffffffffull)) >> 32);
            k = -1;
#pragma unroll
            for (int s = CPL - 1; s >= 0; --s) {
                const bool in = gl + W * s < K && t < P[s];
                const uint32_t b = (__ballot_sync(FULL, in) >> gshift) & gbits;
                if (b) k = W * s + __ffs(b) - 1;
            }
            if (k < 0) k = 0;  // only in a group whose window has ended
        }
        const int nk = cnt[k];
        const uint32_t j = (uint32_t)(((uint64_t)w3 * (uint64_t)(uint32_t)nk) >> 32);

        // Rank search: the j-th member of class k in canonical order (lanes
        // past the cell's words hold zero words, so the full-width scan
        // needs no branch).
        const uint32_t mw = gl < NL ? mask[k * W + gl] : 0u;
        const int c = __popc(mw);
        int incl = c;
#pragma unroll
        for (int off = 1; off < W; off <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, off, W);
            incl += gl >= off ? v : 0;
        }
        const uint32_t hit = (__ballot_sync(FULL, (uint32_t)incl > j) >> gshift) & gbits;
        const int owner = hit ? __ffs(hit) - 1 : 0;
        const int pick = __shfl_sync(FULL, select_bit(mw, (int)j - (incl - c)), owner, W);

        if (F64) {
            if (__any_sync(FULL, act && unsure)) {
                // binary64 decision: tau up to event e - 1 (the rest of the
                // previous batch, then this batch's events before e, all
                // taken), plus event e's waiting time
                double t = tau;
                for (int i = 1; i < W; ++i) {
                    const double v = __shfl_sync(FULL, lq_prev, i, W);
                    if (i > sl && i < ntaken_prev) t = __dadd_rn(t, v);
                }
                const bool mine = gl <= sl;
                const double lqc = div_rn(mine ? rl : 1.0, mine ? lam_mine : 1.0);
                for (int i = 0; i < W - 1; ++i) {
                    const double v = __shfl_sync(FULL, lqc, i, W);
                    if (i < sl) t = __dadd_rn(t, v);
                }
                const double end = __dadd_rn(t, __shfl_sync(FULL, lqc, sl, W));
                const long long eb = dbits(end);
                if (act && unsure) {
                    if (llabs(eb - hbits) < 9008ll) amb = true;  // |end - h| below ~1e-12 h
                    take = eb < hbits;
                    near_edge = true;
                    ++nexact;
                }
            }
            if (!take) act = false;
            if (act) {
                clk += Qs;
                err = Es;
                ++ntaken_cur;
            }
        }
        if (act && hit == 0u) {  // counts and masks disagree: stop rather than write out of bounds
            bad = true;
            act = false;
        }

        // Spin flip at the picked site: its class k = SK sigma + n becomes
        // k -+ SK, and each neighbour inside the cell changes n by +-1 (lanes
        // 1..4: N, E, S, W; on the ring lanes 1, 2: x + 1, x - 1).
        if (act) {
            const int site = owner * 32 + pick;
            const int sy = (int)fdiv((uint32_t)site, G.fqx), sx = site - sy * qx;
            const int sold = k >= SK;
            if (gl == 0) box[(sy + HW) * BW + sx + HW] = (uint8_t)(1 - sold);
            if (gl < SK) {
                int ux = sx, uy = sy;
                if (ring) { ux += gl == 1 ? 1 : (gl == 2 ? -1 : 0); }
                else if (gl > 0) { ux += dir_dx(gl - 1); uy += dir_dy(gl - 1); }
                if (ux >= 0 && ux < qx && uy >= 0 && uy < qy) {
                    const int i = uy * qx + ux;
                    int kold, knew;
                    if (gl == 0) { kold = k; knew = sold ? k - SK : k + SK; }
                    else { kold = (int8_t)scls[i]; knew = kold + (sold ? -1 : 1); }
                    scls[i] = (uint8_t)knew;
                    const int own = i >> 5;
                    const uint32_t bit = 1u << (i & 31);
                    atomicXor(&mask[kold * W + own], bit);
                    atomicXor(&mask[knew * W + own], bit);
                    atomicSub(&cnt[kold], 1);
                    atomicAdd(&cnt[knew], 1);
                }
            }
            ++ev;
        }
        __syncwarp();
    }

    // Write back the cell (a word shared with a neighbouring cell is updated
    // with atomics on this cell's bits only).
    if (valid) {
        if (PACKED) {
            uint32_t *dst32 = reinterpret_cast<uint32_t *>(dst);
            const int wa = X0 >> 5, nwr = ((X0 + qx - 1) >> 5) - wa + 1;
            for (int t = gl; t < qy * nwr; t += W) {
                const int row = t / nwr, wi = wa + (t - row * nwr);
                const uint8_t *brow = box + (row + HW) * BW + HW - X0;
                uint32_t *drow = dst32 + (int64_t)(Y0 + row) * (lx >> 5);
                const int xs = max(X0, wi << 5), xe = min(X0 + qx, (wi + 1) << 5);
                uint32_t msk = 0u, bits = 0u;
                for (int xx = xs; xx < xe; ++xx) {
                    const uint32_t b = 1u << (xx & 31);
                    msk |= b;
                    if (brow[xx]) bits |= b;
                }
                if (msk == 0xffffffffu) {
                    drow[wi] = bits;
                } else {
                    atomicAnd(drow + wi, ~msk);
                    atomicOr(drow + wi, bits);
                }
            }
        } else if (rows16) {
            // aligned 16-byte chunks of the cell's rows
            const int nch = qx >> 4;
            int row = 0, c = gl;
            while (c >= nch) { c -= nch; ++row; }
            for (int t = gl; t < qy * nch; t += W) {
                const uint8_t *b = box + (row + HW) * BW + HW + 16 * c;
                uint32_t wv[4];
#pragma unroll
                for (int q4 = 0; q4 < 4; ++q4)
                    wv[q4] = (uint32_t)b[4 * q4] | ((uint32_t)b[4 * q4 + 1] << 8) |
                             ((uint32_t)b[4 * q4 + 2] << 16) | ((uint32_t)b[4 * q4 + 3] << 24);
                *reinterpret_cast<uint4 *>(dst + (int64_t)(Y0 + row) * lx + X0 + 16 * c) =
                    make_uint4(wv[0], wv[1], wv[2], wv[3]);
                c += W;
                while (c >= nch) { c -= nch; ++row; }
            }
        } else {
            int lly = (int)fdiv((uint32_t)gl, G.fqx), llx = gl - lly * qx;
#pragma unroll 4
            for (int i = gl; i < nsite; i += W) {
                dst[(int64_t)(Y0 + lly) * lx + X0 + llx] = box[(lly + HW) * BW + llx + HW];
                llx += W;
                while (llx >= qx) { llx -= qx; ++lly; }
            }
        }
    }
    *ev_out = ev;
    *amb_out = amb;
    *bad_out = bad;
    *nexact_out = nexact;
}

// Totals of a warp's groups: events, ambiguous and failed cell-windows,
// edge decisions taken in binary64 (one atomic each per warp).
template <int W>
__device__ __forceinline__ void add_counters(unsigned long long *counters, int lane, bool valid,
                                             uint32_t ev, bool amb, bool bad, uint32_t nexact)
{
    const bool lead = valid && (lane & (W - 1)) == 0;
    const uint32_t tot = __reduce_add_sync(FULL, lead ? ev : 0u);
    const int na = __popc(__ballot_sync(FULL, lead && amb));
    const int nb = __popc(__ballot_sync(FULL, lead && bad));
    const uint32_t nr = __reduce_add_sync(FULL, lead ? nexact : 0u);
    if (lane == 0) {
        atomicAdd(&counters[0], (unsigned long long)tot);
        if (na) atomicAdd(&counters[1], (unsigned long long)na);
        if (nb) atomicAdd(&counters[3], (unsigned long long)nb);
        if (nr) atomicAdd(&counters[4], (unsigned long long)nr);
    }
}

// Plain engine: one launch per window; warp u runs active cells GC u ..
// GC u + GC - 1 of one replica (GC = 32/W cells per warp).
template <int MODEL, typename CLK, bool PACKED, int W>
__global__ void __launch_bounds__(256) fs_group_kernel(WindowArgs a, int nactive, int stride)
{
    constexpr int GC = 32 / W;
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int warp = blockIdx.x * (blockDim.x >> 5) + wib;
    if (warp * GC >= nactive) return;  // the whole warp
    const int cell = warp * GC + lane / W;
    const bool valid = cell < nactive;
    const Replica &R = a.reps[a.rep_index];
    int cx = 0, cy = 0;
    if (valid) {
        if (a.order) {  // heaviest-first issue list
            const int mo = a.order[cell];
            cy = mo / R.ncx;
            cx = mo - cy * R.ncx;
        } else {
            const int half = R.ncx >> 1;
            cy = cell / half;
            cx = 2 * (cell % half) + ((a.colour + cy) & 1);
        }
    }
    const GLayout Lo = make_glayout<MODEL>(a.geom.qx, a.geom.qy, W);
    uint8_t *csm = smem + (size_t)(wib * GC + lane / W) * stride;
    uint32_t ev;
    uint32_t nexact;
    bool amb, bad;
    group_window<MODEL, CLK, false, PACKED, W>(csm, Lo, R, a.geom, valid, cell_at(R, a.geom, cx, cy), a.w, a.h,
                                                a.screen != 0, a.seed,
                                                a.src + R.lat_off, a.dst + R.lat_off, lane, &ev,
                                                &amb, &bad, &nexact);
    if (valid && (lane & (W - 1)) == 0) a.workload[R.cell_off + cy * R.ncx + cx] = (int32_t)ev;
    add_counters<W>(a.counters, lane, valid, ev, amb, bad, nexact);
}

// Persistent engine (in-place spin-flip models): a task is a chunk of GC
// consecutive active cells of one window (they never depend on each other);
// chunks are dequeued window-major, so a chunk waits only on chunks of
// earlier windows, which running warps hold or have finished. Each group
// waits for its own cell's dependencies -- its previous active window and
// its edge neighbours' last active window before this one (epoch = 1 + last
// active window) -- with the bounded, backed-off polls of wait_epochs.
template <int MODEL, typename CLK, bool PACKED, int W>
__global__ void __launch_bounds__(256) fs_group_persistent_kernel(const __grid_constant__ PParams P, int stride)
{
    constexpr int GC = 32 / W;
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int gl = lane & (W - 1);
    uint8_t *csm = smem + (size_t)(wib * GC + lane / W) * stride;
    const GLayout Lo = make_glayout<MODEL>(P.geom.qx, P.geom.qy, W);
    const int per_window = P.total_active;
    const int chunks = (per_window + GC - 1) / GC;
    const unsigned long long total = (unsigned long long)P.nwin * (unsigned long long)chunks;

    for (;;) {
        // the dequeue and the abort flag in one round trip
        unsigned long long t = 0;
        int ab = 0;
        if (lane == 0) {
            t = atomicAdd(P.queue, 1ull);
            ab = *(volatile int32_t *)P.abort_flag;
        }
        t = __shfl_sync(FULL, t, 0);
        if (t >= total) break;
        if (__shfl_sync(FULL, ab, 0)) break;
        const int i = (int)(t / (unsigned long long)chunks);
        const int ch = (int)(t % (unsigned long long)chunks);
        const int u = ch * GC + lane / W;
        const bool valid = u < per_window;
        const int a = valid ? u : ch * GC;  // a cell-less group borrows the chunk's first cell's replica
        // one schedule for all replicas: the window's colour and dependencies
        // load beside the cell's replica
        int ccol = 0;
        int2 pv = make_int2(0, 0);
        if (!P.colour_per_replica) {
            ccol = P.colour[i];
            pv = P.prev[i];
        }
        const int2 rk = P.cell_rk[a];
        const int r = rk.x;
        const int k = rk.y;
        const Replica &R = P.reps[r];
        const int64_t widx = P.colour_per_replica ? (int64_t)r * P.nwin + i : i;
        if (P.colour_per_replica) {
            ccol = P.colour[widx];
            pv = P.prev[widx];
        }
        int cx, cy;
        if (P.order) {
            const int mo = P.order[R.cell_off + ccol * ((R.ncx >> 1) * R.ncy) + k];
            cy = mo / R.ncx;
            cx = mo - cy * R.ncx;
        } else {
            const int half = R.ncx >> 1;
            cy = k / half;
            cx = 2 * (k % half) + ((ccol + cy) & 1);
        }
        const int m = cy * R.ncx + cx;
        int32_t *ep = P.epoch + R.cell_off;
        uint8_t *cur = P.lat + R.lat_off;

        // Dependency 0: the cell's previous active window; 1..4: the edge
        // neighbours' (E, S, W, N) last active window before this one. A ring
        // (one row of cells) has no vertical neighbours. Lane gl of a group
        // waits on dependencies gl, gl + W.
        bool ok = true;
#pragma unroll
        for (int d0 = 0; d0 < 5; d0 += W) {
            const int d = d0 + gl;
            const int ex = d == 1 ? 1 : (d == 3 ? -1 : 0);
            const int ey = d == 2 ? 1 : (d == 4 ? -1 : 0);
            const int dcx = (cx + ex + R.ncx) % R.ncx, dcy = (cy + ey + R.ncy) % R.ncy;
            const int target = (d == 0 ? pv.x : pv.y) + 1;
            const bool dep = valid && d < 5 && target > 0 && !(ey != 0 && R.ncy == 1);
            if (ok) ok = wait_epochs(ep, dcy * R.ncx + dcx, dep, target, P, lane);  // warp-uniform
        }
        if (!ok) break;

        uint32_t ev;
        uint32_t nexact;
        bool amb, bad;
        group_window<MODEL, CLK, true, PACKED, W>(csm, Lo, R, P.geom, valid, cell_at(R, P.geom, cx, cy), P.w0 + (uint32_t)i,
                                                   P.h[i], P.screen != 0, P.seed, cur, cur, lane, &ev, &amb, &bad,
                                                   &nexact);
        if (valid && gl == 0) P.workload[R.cell_off + m] = (int32_t)ev;
        add_counters<W>(P.counters, lane, valid, ev, amb, bad, nexact);
        // the warp barrier orders the group's writes before its lead lane's
        // release store (release is cumulative), which publishes them
        __syncwarp();
        if (valid && gl == 0) {
            cuda::atomic_ref<int32_t, cuda::thread_scope_device> ea(ep[m]);
            ea.store(i + 1, cuda::memory_order_release);
        }
    }
}

}  // namespace

}  // namespace fskmc
