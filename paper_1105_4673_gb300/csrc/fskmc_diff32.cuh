// The binary32-clock window of a 32-wide adsorption/desorption + diffusion
// cell held in registers, one cell per warp, lane y owning row y.
//
// The generic one-cell window (fskmc_cell.cuh) keeps every class as
// shared-memory membership bits (eight slot bits per site for the hops) and
// after each event re-classes every member within two sites of the changed
// ones. Here lane y holds its row as one occupancy mask o plus its halo
// sites, and every class is recounted after each event from the masks by
// bit slicing: the occupied-neighbour count n of each site as three bit
// planes, the site classes 5 sigma + n, and the hop classes 10 + n (Section
// 2's directed slots: the origin occupied with n occupied neighbours, the
// target empty), counted per direction with the window colour's ownership
// masks. Same classes and rates as the binary64 form, the same draws,
// fixed-point class sums and binary32 clock as the other binary32 paths; the
// members of a class are numbered in another order, so the result is
// statistically, not bitwise, that of the binary64 form.
//
// Members of a class in lane y, in order: site classes, the row's sites of
// that class by x; hop classes 10 + n, the hops from the row's sites up,
// down, left and right (each by x; a hop across the cell's edge into the
// halo is a member if the window owns that cross slot: horizontal ones in E
// windows, vertical ones in O windows), then the hops into the row from the
// halo (O windows: from the top halo row into row 0 in lane 0, from the
// bottom halo row into the last row in the last lane; E windows: from the
// left and the right halo site of the row).
#pragma once
#include <cuda_runtime.h>

#include "fskmc_device.cuh"
#include "fskmc_internal.h"
#include "fskmc_zgb32.cuh"
#include "philox.cuh"

namespace fskmc {

namespace {

// Per-window constants of diff32_window, in shared memory behind the staged
// rows.
struct alignas(16) Diff32Const {
    uint64_t rq[16];  // the class rates in fixed point (15 classes)
    uint64_t seed;
    uint8_t *dst;
    float qscale, hf;
    uint32_t ctr3, w, m;
    int32_t X0, Y0, lx, ly;
};

// Shared memory diff32_window needs per warp: the staged box rows (the cell
// and two halo rows above and below, 64 bytes each), the constants, and per
// lane 16 bytes of class counts and 48 bytes of member masks.
__host__ __device__ constexpr int diff32_smem(int qy)
{
    return 64 * (qy + 4) + (int)sizeof(Diff32Const) + 32 * 16 + 32 * 48;
}

// Bit-sliced sum of four masks (each bit position 0..4): planes p0, p1, p2.
__device__ __forceinline__ void add4(uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t &p0, uint32_t &p1,
                                     uint32_t &p2)
{
    const uint32_t s1 = a ^ b, c1 = a & b, s2 = c ^ d, c2 = c & d;
    const uint32_t c3 = s1 & s2;
    p0 = s1 ^ s2;
    p1 = c1 ^ c2 ^ c3;  // c1 + c2 + c3 <= 2, and 2 only as c1 = c2 = 1
    p2 = c1 & c2;
}

// Positions whose bit-sliced count (p0, p1, p2) equals n (0..4).
__device__ __forceinline__ uint32_t eqn(uint32_t p0, uint32_t p1, uint32_t p2, int n)
{
    return (n & 1 ? p0 : ~p0) & (n & 2 ? p1 : ~p1) & (n & 4 ? p2 : ~p2);
}


// One cell's binary32-clock window (qx == 32, 2 <= qy <= 32), the cell at
// `at` in the byte lattice src (== dst: the model updates in place). wsm:
// diff32_smem(qy) bytes of 16-byte aligned shared memory. Returns the
// events; *bad_out is set if a rank search found no member (never, unless
// the counts and masks disagree) or a window ran away.
template <bool PERSIST>
__device__ uint32_t diff32_window(uint8_t *wsm, const Replica &R, const CellGeom &G, const CellAt &at,
                                  int colour, uint32_t w, double hwin, uint64_t seed, const uint8_t *src,
                                  uint8_t *dst, int lane, bool *bad_out)
{
    constexpr unsigned FULLW = 0xffffffffu;
    const int qy = G.qy, BH = qy + 4;
    const bool ew = colour == 0;
    const bool row = lane < qy, first = lane == 0, last = lane == qy - 1;
    const uint32_t rowm = row ? ~0u : 0u;

    // Stage the box rows y = -2 .. qy + 1, each as four aligned 16-byte
    // chunks (the 16 sites left of the cell, its 32, the 16 right of it).
    uint8_t *raw = wsm;
    {
        const int lx = at.lx, ly = at.ly, X0 = at.X0, Y0 = at.Y0;
        const int xl = X0 >= 16 ? X0 - 16 : X0 - 16 + lx;
        const int xr = X0 + 32 < lx ? X0 + 32 : X0 + 32 - lx;
        for (int i = lane; i < 4 * BH; i += 32) {
            const int by = i >> 2, part = i & 3;
            int gy = Y0 - 2 + by;
            gy += (gy < 0) ? ly : 0; gy -= (gy >= ly) ? ly : 0;
            const int gx = part == 0 ? xl : (part == 3 ? xr : X0 + 16 * (part - 1));
            cp_async16(raw + by * 64 + 16 * part, src + (int64_t)gy * lx + gx);
        }
    }
    Diff32Const *Cw = reinterpret_cast<Diff32Const *>(wsm + 64 * BH);
    uint32_t *clw = reinterpret_cast<uint32_t *>(wsm + 64 * BH + sizeof(Diff32Const)) + 4 * lane;
    uint4 *mw = reinterpret_cast<uint4 *>(wsm + 64 * BH + sizeof(Diff32Const) + 32 * 16) + 3 * lane;
    if (lane < 16) Cw->rq[lane] = lane < 15 ? R.rq[lane] : 0ull;
    if (lane == 0) {
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
    const volatile Diff32Const &C = *Cw;
    // lane y: row y (box row y + 2) as the occupancy mask o, and hb: its halo
    // sites x = -1 (bit 0), -2 (bit 1), 32 (bit 2), 33 (bit 3); lane 0 also
    // the halo rows y = -1 (H1) and y = -2 (H2) with row -1's sites x = -1
    // (hb bit 4) and 32 (bit 5); the last lane likewise the rows y = qy (H1)
    // and qy + 1 (H2) with row qy's corner sites (qy >= 2: two lanes).
    uint32_t o = 0u, H1 = 0u, H2 = 0u, hb = 0u, tmp;
    if (row) {
        const uint8_t *r = raw + (lane + 2) * 64 + 16;
        zgb_row_masks(r, tmp, o);
        hb = (r[-1] & 1u) | ((r[-2] & 1u) << 1) | ((r[32] & 1u) << 2) | ((r[33] & 1u) << 3);
    }
    if (first || last) {
        const uint8_t *h1 = raw + (first ? 1 : qy + 2) * 64 + 16, *h2 = raw + (first ? 0 : qy + 3) * 64 + 16;
        zgb_row_masks(h1, tmp, H1);
        zgb_row_masks(h2, tmp, H2);
        hb |= ((h1[-1] & 1u) << 4) | ((h1[32] & 1u) << 5);
    }

    float tauf = 0.0f, rlf = 0.0f;
    uint32_t rw2 = 0u, rw3 = 0u, ev = 0u;
    for (;;) {
        // The classes of the current state. Neighbours of the row's sites:
        // up, down (the rows of lanes y -+ 1, or a halo row), left, right.
        uint32_t oN = __shfl_up_sync(FULLW, o, 1), oS = __shfl_down_sync(FULLW, o, 1);
        if (first) oN = H1;
        if (last) oS = H1;
        const uint32_t hl1 = hb & 1u, hr1 = (hb >> 2) & 1u;
        const uint32_t oW = (o << 1) | hl1, oE = __funnelshift_r(o, hr1, 1);
        uint32_t p0, p1, p2;
        add4(oN, oS, oW, oE, p0, p1, p2);  // occupied neighbours of each site
        // hops out of the row: origin occupied, target empty, the slot owned
        const uint32_t dN = o & ~oN & ((first && ew) ? 0u : ~0u);
        const uint32_t dS = o & ~oS & ((last && ew) ? 0u : ~0u);
        const uint32_t dW = o & ~oW & (ew ? ~0u : ~1u);
        const uint32_t dE = o & ~oE & (ew ? ~0u : 0x7FFFFFFFu);
        // hops into the row from the halo (O windows: the halo row H1 in lane
        // 0 / the last lane; E windows: the left and right halo sites), with
        // the occupied-neighbour counts of their origins (the target is empty)
        const uint32_t H1L = (H1 << 1) | ((hb >> 4) & 1u), H1R = __funnelshift_r(H1, (hb >> 5) & 1u, 1);
        uint32_t v0, v1, v2;
        add4(H2, H1L, H1R, 0u, v0, v1, v2);
        const uint32_t iv = ((first || last) && !ew) ? (H1 & ~o) : 0u;
        uint32_t hlu = __shfl_up_sync(FULLW, hl1, 1), hld = __shfl_down_sync(FULLW, hl1, 1);
        uint32_t hru = __shfl_up_sync(FULLW, hr1, 1), hrd = __shfl_down_sync(FULLW, hr1, 1);
        if (first) { hlu = (hb >> 4) & 1u; hru = (hb >> 5) & 1u; }
        if (last) { hld = (hb >> 4) & 1u; hrd = (hb >> 5) & 1u; }
        const uint32_t il = ew ? (hl1 & ~o & 1u) : 0u, ir = ew ? (hr1 & (~o >> 31)) : 0u;
        const uint32_t nl = ((hb >> 1) & 1u) + hlu + hld, nr = ((hb >> 3) & 1u) + hru + hrd;
        // per-lane counts, class k in byte k % 4 of word k / 4
        uint32_t cw0 = 0u, cw1 = 0u, cw2 = 0u, cw3 = 0u;
        const auto put = [&](int k, uint32_t v) {
            const uint32_t sv = v << (8 * (k & 3));
            if (k < 4) cw0 |= sv;
            else if (k < 8) cw1 |= sv;
            else if (k < 12) cw2 |= sv;
            else cw3 |= sv;
        };
#pragma unroll
        for (int n = 0; n < 5; ++n) {
            const uint32_t e = eqn(p0, p1, p2, n);
            put(n, (uint32_t)__popc(rowm & ~o & e));
            put(5 + n, (uint32_t)__popc(o & e));
            if (n < 4) {
                const uint32_t ev_n = eqn(v0, v1, 0u, n);
                put(10 + n, (uint32_t)(__popc(dN & e) + __popc(dS & e) + __popc(dW & e) + __popc(dE & e) +
                                       __popc(iv & ev_n) + (il && nl == (uint32_t)n) + (ir && nr == (uint32_t)n)));
            }
        }
        *reinterpret_cast<uint4 *>(clw) = make_uint4(cw0, cw1, cw2, cw3);
        mw[0] = make_uint4(p0, p1, p2, dN);
        mw[1] = make_uint4(dS, dW, dE, iv);
        mw[2] = make_uint4(v0, v1, il | (ir << 1) | (nl << 2) | (nr << 4), 0u);
        // class totals (pairs of 16-bit sums), then lane k < 14 holds class
        // k's total and its fixed-point prefix sum
        const int kl = lane < 14 ? lane : 13;
        uint32_t rs = 0u;
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            const uint32_t wq = q < 2 ? cw0 : (q < 4 ? cw1 : (q < 6 ? cw2 : cw3));
            const uint32_t x = (wq >> (16 * (q & 1))) & 0xFFFFu;
            const uint32_t tq = __reduce_add_sync(FULLW, (x & 0xFFu) | ((x & 0xFF00u) << 8));
            rs = (kl >> 1) == q ? tq : rs;
        }
        const uint32_t nmine = lane < 14 ? (rs >> (16 * (kl & 1))) & 0xFFFFu : 0u;
        uint64_t P = (uint64_t)nmine * C.rq[kl];
#pragma unroll
        for (int off = 1; off < 16; off <<= 1) {
            const uint64_t v = __shfl_up_sync(FULLW, P, off, 16);
            if ((lane & 15) >= off) P += v;
        }
        const uint64_t lami = __shfl_sync(FULLW, P, 13);
        if (lami == 0ull) break;
        if (ev >= MAX_EVENTS_PER_WINDOW) {
            *bad_out = true;
            break;
        }
        if ((ev & 31u) == 0u) {  // 32 events' draws at once, one Philox block per lane
            const u32x4 d = draw(C.seed, ev + (uint32_t)lane, C.w, C.m, C.ctr3);
            rlf = -__logf(__fmul_rn(__uint2float_rn((d.x >> 8) + 1u), 0x1p-24f));
            rw2 = d.z;
            rw3 = d.w;
        }
        const int sl = (int)(ev & 31u);
        const float lg = __shfl_sync(FULLW, rlf, sl);
        const float lamf = __fmul_rn(u64_to_float_rz(lami), C.qscale);
        const float end = __fadd_rn(tauf, __fdividef(lg, lamf));
        if (end >= C.hf) break;
        tauf = end;
        // class: the first k with (w2 lambda) >> 32 < P_k (exact integers)
        const uint32_t w2 = __shfl_sync(FULLW, rw2, sl), w3 = __shfl_sync(FULLW, rw3, sl);
        const uint64_t t = (uint64_t)w2 * (lami >> 32) + (((uint64_t)w2 * (lami & 0xffffffffull)) >> 32);
        const uint32_t hk = __ballot_sync(FULLW, lane < 14 && t < P);
        const int k = __ffs(hk) - 1;
        const uint32_t nk = __shfl_sync(FULLW, nmine, k);
        const uint32_t j = (uint32_t)(((uint64_t)w3 * (uint64_t)nk) >> 32);
        // member j of class k: the owner lane by a prefix scan of the lanes'
        // counts, then the member in the owner's masks
        const int c = (int)((clw[k >> 2] >> (8 * (k & 3))) & 0xFFu);
        int incl = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(FULLW, incl, off);
            if (lane >= off) incl += v;
        }
        const uint32_t hit = __ballot_sync(FULLW, (uint32_t)incl > j);
        if (hit == 0u) {
            *bad_out = true;
            break;
        }
        const int owner = __ffs(hit) - 1;
        // kind: 0 site, 1-4 hop out up / down / left / right, 5 hop in from
        // the halo row, 6 from the left halo site, 7 from the right one
        int code = 0;
        if (lane == owner) {
            int r = (int)j - (incl - c);
            const uint4 m0 = mw[0], m1 = mw[1], m2 = mw[2];
            int kind = 0;
            uint32_t msk;
            if (k < 10) {
                msk = (k >= 5 ? o : ~o) & eqn(m0.x, m0.y, m0.z, k % 5);
            } else {
                const int n = k - 10;
                const uint32_t e = eqn(m0.x, m0.y, m0.z, n);
                const uint32_t a1 = m0.w & e, a2 = m1.x & e, a3 = m1.y & e, a4 = m1.z & e;
                const uint32_t a5 = m1.w & eqn(m2.x, m2.y, 0u, n);
                const uint32_t hx = m2.z;
                const uint32_t a6 = ((hx & 1u) && ((hx >> 2) & 3u) == (uint32_t)n) ? 1u : 0u;
                const uint32_t a7 = (((hx >> 1) & 1u) && ((hx >> 4) & 3u) == (uint32_t)n) ? 1u : 0u;
                const int c1 = __popc(a1), c2 = __popc(a2), c3 = __popc(a3), c4 = __popc(a4), c5 = __popc(a5);
                msk = a1; kind = 1;
                if (r >= c1) {
                    r -= c1; msk = a2; kind = 2;
                    if (r >= c2) {
                        r -= c2; msk = a3; kind = 3;
                        if (r >= c3) {
                            r -= c3; msk = a4; kind = 4;
                            if (r >= c4) {
                                r -= c4; msk = a5; kind = 5;
                                if (r >= c5) {
                                    r -= c5; msk = a6 ? 1u : 0x80000000u; kind = a6 ? 6 : 7;
                                    if (a6 && r >= 1) { r -= 1; msk = 0x80000000u; kind = 7; }
                                }
                            }
                        }
                    }
                }
            }
            code = (kind << 5) | select_bit(msk, r);
        }
        code = __shfl_sync(FULLW, code, owner);
        const int kind = code >> 5, x = code & 31, y = owner;
        const uint32_t bit = 1u << x;
        if (kind == 0) {
            if (lane == y) o ^= bit;  // adsorption or desorption
        } else if (kind <= 4) {
            // the particle leaves (x, y) for the neighbour up, down, left or right
            if (lane == y) o &= ~bit;
            if (kind == 1) {
                if (y == 0) { if (lane == 0) H1 |= bit; }
                else if (lane == y - 1) o |= bit;
            } else if (kind == 2) {
                if (y == qy - 1) { if (lane == y) H1 |= bit; }
                else if (lane == y + 1) o |= bit;
            } else if (lane == y) {
                if (kind == 3) { if (x == 0) hb |= 1u; else o |= bit >> 1; }
                else { if (x == 31) hb |= 4u; else o |= bit << 1; }
            }
        } else if (lane == y) {
            // a particle of the halo enters (x, y)
            o |= bit;
            if (kind == 5) H1 &= ~bit;
            else if (kind == 6) hb &= ~1u;
            else hb &= ~4u;
        }
        ++ev;
    }

    // Write back: the cell's rows, and the owned halo ends (the halo columns
    // in E windows, the halo rows in O windows)
    uint8_t *const out = C.dst;
    const int lx = C.lx, ly = C.ly, X0 = C.X0, Y0 = C.Y0;
    if (row) zgb_store_row(out + (int64_t)(Y0 + lane) * lx + X0, ~o, o);
    if (ew) {
        if (row) {
            const int gy = Y0 + lane;
            const int gxl = X0 > 0 ? X0 - 1 : lx - 1, gxr = X0 + 32 < lx ? X0 + 32 : 0;
            out[(int64_t)gy * lx + gxl] = (uint8_t)(hb & 1u);
            out[(int64_t)gy * lx + gxr] = (uint8_t)((hb >> 2) & 1u);
        }
    } else {
        if (first) zgb_store_row(out + (int64_t)(Y0 > 0 ? Y0 - 1 : ly - 1) * lx + X0, ~H1, H1);
        if (last) zgb_store_row(out + (int64_t)(Y0 + qy < ly ? Y0 + qy : 0) * lx + X0, ~H1, H1);
    }
    return ev;
}

}  // namespace

}  // namespace fskmc
