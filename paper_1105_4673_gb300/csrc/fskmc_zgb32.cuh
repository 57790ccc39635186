// The binary32-clock window of a 32-wide ZGB cell held in registers, one
// cell per warp, lane y owning row y.
//
// The generic one-cell window (fskmc_cell.cuh) keeps every class as
// membership bit masks in shared memory -- for the pair classes one bit per
// directed slot, eight per site -- and after each event re-classes the
// slots around the changed sites one lane per slot, with shared atomics.
// Here the whole cell state is two 32-bit masks per lane (e: empty sites
// of the row, a: sites holding A; B is neither) plus the row's two halo
// sites, and every class is recomputed from them after each event by a few
// bitwise operations per lane, branch-free: no shared memory, no atomics.
//
// The pair events (B2 adsorbs on two empty neighbours; A and B react) are
// taken on undirected bonds at twice the directed rate. This is the same
// process: every owned bond is owned in both directions (Section 2's
// directed slots (u, v) and (v, u) are both members of the class or
// neither), both directions have the same rate, and the event's outcome
// does not depend on the direction. Only the order in which the members of
// a class are numbered differs from the directed-slot form; as everywhere
// with the binary32 clock, the result is statistically, not bitwise, that
// of the binary64 form. The draws, the fixed-point class sums and the
// binary32 clock are the generic binary32 path's.
//
// Members of a pair class in lane y, in order: the horizontal bonds of row
// y ((x, y)-(x+1, y), x = 0..31; x = 31 is the cross bond to the right halo,
// owned in E windows), the vertical bonds below row y ((x, y)-(x, y+1); for
// the last row the cross bond to the bottom halo, owned in O windows), the
// left cross bond ((-1, y)-(0, y), E windows) and, in lane 0 only, the
// vertical cross bonds to the top halo ((x, -1)-(x, 0), O windows).
#pragma once
#include <cuda_runtime.h>

#include "fskmc_device.cuh"
#include "fskmc_internal.h"
#include "philox.cuh"

namespace fskmc {

namespace {

// Masks of the 32 sites at p (16-byte aligned) in states 0 (empty) and 1 (A),
// from bytes holding 0, 1 or 2: a byte's bit 0 marks A, neither of its low
// two bits empty; one multiply gathers the four flags of a word (bit 8k to
// bit 21 + k, no carries between them) into a nibble.
__device__ __forceinline__ void zgb_row_masks(const uint8_t *p, uint32_t &e, uint32_t &a)
{
    const uint4 u0 = *reinterpret_cast<const uint4 *>(p), u1 = *reinterpret_cast<const uint4 *>(p + 16);
    const uint32_t v[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
    e = 0u;
    a = 0u;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t ta = v[k] & 0x01010101u;                       // bit 0 of each byte: A
        const uint32_t te = ~(v[k] | (v[k] >> 1)) & 0x01010101u;      // neither bit: empty
        e |= ((te * 0x00204081u) >> 21 & 0xFu) << (4 * k);
        a |= ((ta * 0x00204081u) >> 21 & 0xFu) << (4 * k);
    }
}

// 4 mask bits -> 4 bytes of 0/1 (bit k to bit 8k by one multiply).
__device__ __forceinline__ uint32_t zgb_expand4(uint32_t m4)
{
    return ((m4 & 0xFu) * 0x00204081u) & 0x01010101u;
}

// The 32 bytes of a row (states 0 empty, 1 A, 2 B) from its masks, as two
// 16-byte stores to p (16-byte aligned).
__device__ __forceinline__ void zgb_store_row(uint8_t *p, uint32_t e, uint32_t a)
{
    const uint32_t b = ~(e | a);
    uint32_t wv[8];
#pragma unroll
    for (int g = 0; g < 8; ++g) wv[g] = zgb_expand4(a >> (4 * g)) + 2u * zgb_expand4(b >> (4 * g));
    uint4 *d = reinterpret_cast<uint4 *>(p);
    d[0] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
    d[1] = make_uint4(wv[4], wv[5], wv[6], wv[7]);
}

// Lane y's bonds of pair class k (1: both ends empty; 2: one end A, the
// other B), by kind: H horizontal bonds of row y (bit x: (x, y)-(x+1, y)),
// V vertical bonds below it (bit x: (x, y)-(x, y+1)), N (lane 0) vertical
// bonds to the top halo, L (bit 0) the left cross bond. e, a: row y; eB,
// aB: the row below (the bottom halo row for the last row); eN, aN: the top
// halo row (read in lane 0 only); hl*, hr*: the row's left and right halo
// sites (0/1); ew: an E
// window (horizontal cross bonds owned), otherwise an O window (vertical
// cross bonds owned). Rows without sites (lanes >= qy) have e = a = 0 and
// row = false.
struct ZgbBonds {
    uint32_t H, V, N, L;
};

__device__ __forceinline__ ZgbBonds zgb_bonds(int k, bool row, bool last, bool first, bool ew, uint32_t e,
                                              uint32_t a, uint32_t eB, uint32_t aB, uint32_t eN, uint32_t aN,
                                              uint32_t hle, uint32_t hla, uint32_t hre, uint32_t hra)
{
    const uint32_t b = row ? ~(e | a) : 0u;
    const uint32_t bB = ~(eB | aB), bN = ~(eN | aN);
    const uint32_t hlb = 1u - hle - hla, hrb = 1u - hre - hra;
    // the right neighbour of every site of the row (site 31's is the right halo site)
    const uint32_t eR = (e >> 1) | (hre << 31), aR = (a >> 1) | (hra << 31), bR = (b >> 1) | (hrb << 31);
    const uint32_t ownH = ew ? ~0u : 0x7FFFFFFFu;          // bond 31 crosses to the right halo
    const uint32_t ownV = !last ? ~0u : (ew ? 0u : ~0u);   // the last row's bonds cross to the bottom halo
    const uint32_t ownN = (first && !ew) ? ~0u : 0u;        // lane 0: bonds to the top halo
    const uint32_t ownL = ew ? 1u : 0u;
    ZgbBonds B;
    if (k == 1) {
        B.H = e & eR & ownH;
        B.V = e & eB & ownV;
        B.N = eN & e & ownN;
        B.L = hle & e & ownL;
    } else {
        B.H = ((a & bR) | (b & aR)) & ownH;
        B.V = ((a & bB) | (b & aB)) & ownV;
        B.N = ((aN & b) | (bN & a)) & ownN;
        B.L = ((hla & b) | (hlb & a)) & ownL & 1u;
    }
    return B;
}

__device__ __forceinline__ int zgb_bond_count(const ZgbBonds &B)
{
    return __popc(B.H) + __popc(B.V) + __popc(B.N) + (int)B.L;
}

// The per-window constants of zgb32_window, in shared memory behind the
// staging rows and read (volatile) where they are used, so that across the
// event loop the registers hold only the cell's state.
struct alignas(16) Zgb32Const {
    uint64_t rq[4];  // the class rates in fixed point, the pair classes' doubled (undirected bonds)
    uint64_t seed;
    uint8_t *dst;
    float qscale, hf;
    uint32_t ctr3, w, m;
    int32_t X0, Y0, lx, ly;
};

// Shared memory zgb32_window needs per warp.
__host__ __device__ constexpr int zgb32_smem(int qy)
{
    return 64 * (qy + 2) + (int)sizeof(Zgb32Const);
}

// One cell's binary32-clock window (qx == 32, 2 <= qy <= 32), the cell at `at`
// in the byte lattice src (== dst: ZGB updates in place). wsm: zgb32_smem(qy)
// bytes of 16-byte aligned shared memory. Returns the events; *bad_out is
// set if a rank search found no member (never, unless the counts and masks
// disagree) or a window ran away.
template <bool PERSIST>
__device__ uint32_t zgb32_window(uint8_t *wsm, const Replica &R, const CellGeom &G, const CellAt &at,
                                 int colour, uint32_t w, double hwin, uint64_t seed, const uint8_t *src,
                                 uint8_t *dst, int lane, bool *bad_out)
{
    constexpr unsigned FULLW = 0xffffffffu;
    const int qy = G.qy, BH = qy + 2;
    const bool ew = colour == 0;
    const bool row = lane < qy, first = lane == 0, last = lane == qy - 1;

    // Stage: every box row (the rows above and below the cell too) as four
    // aligned 16-byte chunks -- the 16 sites left of the cell, its 32, the 16
    // right of it -- all in flight at once.
    uint8_t *raw = wsm;
    {
        const int lx = at.lx, ly = at.ly, X0 = at.X0, Y0 = at.Y0;
        const int xl = X0 >= 16 ? X0 - 16 : X0 - 16 + lx;
        const int xr = X0 + 32 < lx ? X0 + 32 : X0 + 32 - lx;
        for (int i = lane; i < 4 * BH; i += 32) {
            const int by = i >> 2, part = i & 3;
            int gy = Y0 - 1 + by;
            gy += (gy < 0) ? ly : 0; gy -= (gy >= ly) ? ly : 0;
            const int gx = part == 0 ? xl : (part == 3 ? xr : X0 + 16 * (part - 1));
            cp_async16(raw + by * 64 + 16 * part, src + (int64_t)gy * lx + gx);
        }
    }
    Zgb32Const *Cw = reinterpret_cast<Zgb32Const *>(wsm + 64 * BH);
    if (lane == 0) {
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
    // lane y: row y (box row y + 1) and its halo sites; (eH, aH): in lane 0
    // the top halo row, in the last lane the bottom halo row (qy >= 2: two
    // different lanes)
    uint32_t e = 0u, a = 0u, eH = 0u, aH = 0u;
    uint32_t hle = 0u, hla = 0u, hre = 0u, hra = 0u;
    if (row) {
        const uint8_t *rr = raw + (lane + 1) * 64 + 16;
        zgb_row_masks(rr, e, a);
        hle = rr[-1] == 0; hla = rr[-1] == 1;
        hre = rr[32] == 0; hra = rr[32] == 1;
    }
    if (first) zgb_row_masks(raw + 16, eH, aH);
    if (last) zgb_row_masks(raw + (qy + 1) * 64 + 16, eH, aH);

    float tauf = 0.0f, rlf = 0.0f;
    uint32_t rw2 = 0u, rw3 = 0u, ev = 0u;
    for (;;) {
        // the classes of the current state: each lane's member counts, the
        // totals (every lane) and the fixed-point rate sums
        uint32_t eB = __shfl_down_sync(FULLW, e, 1), aB = __shfl_down_sync(FULLW, a, 1);
        if (last) { eB = eH; aB = aH; }
        int cl[4];
        cl[0] = __popc(e);
        cl[3] = __popc(a);
        cl[1] = zgb_bond_count(zgb_bonds(1, row, last, first, ew, e, a, eB, aB, eH, aH, hle, hla, hre, hra));
        cl[2] = zgb_bond_count(zgb_bonds(2, row, last, first, ew, e, a, eB, aB, eH, aH, hle, hla, hre, hra));
        uint32_t n[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) n[k] = __reduce_add_sync(FULLW, (uint32_t)cl[k]);
        const uint64_t P0 = (uint64_t)n[0] * C.rq[0], P1 = P0 + (uint64_t)n[1] * C.rq[1];
        const uint64_t P2 = P1 + (uint64_t)n[2] * C.rq[2], lami = P2 + (uint64_t)n[3] * C.rq[3];
        if (lami == 0ull) break;
        if (ev >= MAX_EVENTS_PER_WINDOW) {
            *bad_out = true;
            break;
        }
        if ((ev & 31u) == 0u) {  // 32 events' draws at once, one Philox block per lane
            const u32x4 o = draw(C.seed, ev + (uint32_t)lane, C.w, C.m, C.ctr3);
            rlf = -__logf(__fmul_rn(__uint2float_rn((o.x >> 8) + 1u), 0x1p-24f));
            rw2 = o.z;
            rw3 = o.w;
        }
        const int sl = (int)(ev & 31u);
        const float l = __shfl_sync(FULLW, rlf, sl);
        const uint32_t w2 = __shfl_sync(FULLW, rw2, sl), w3 = __shfl_sync(FULLW, rw3, sl);
        const float lamf = __fmul_rn(u64_to_float_rz(lami), C.qscale);
        const float end = __fadd_rn(tauf, __fdividef(l, lamf));
        if (end >= C.hf) break;
        tauf = end;
        // class: the first k with (w2 lambda) >> 32 < P_k (exact integers)
        const uint64_t t = (uint64_t)w2 * (lami >> 32) + (((uint64_t)w2 * (lami & 0xffffffffull)) >> 32);
        const int k = t < P0 ? 0 : (t < P1 ? 1 : (t < P2 ? 2 : 3));
        const uint32_t nk = k == 0 ? n[0] : (k == 1 ? n[1] : (k == 2 ? n[2] : n[3]));
        const uint32_t j = (uint32_t)(((uint64_t)w3 * (uint64_t)nk) >> 32);
        // member j of class k: the owner lane by a prefix scan of the lanes'
        // counts, then the bit in the owner's masks
        const int c = k == 0 ? cl[0] : (k == 1 ? cl[1] : (k == 2 ? cl[2] : cl[3]));
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
        // kind: 0 site, 1 horizontal bond, 2 vertical bond, 3 left cross bond, 4 top-halo bond
        int code = 0;
        if (lane == owner) {
            int r = (int)j - (incl - c);
            int kind, x;
            uint32_t msk;
            if (k == 0 || k == 3) {
                kind = 0;
                msk = k == 0 ? e : a;
            } else {
                // the lane's members in order: horizontal bonds, vertical
                // bonds, the left cross bond, the top-halo bonds; one select
                // in the mask that holds member r
                const ZgbBonds B = zgb_bonds(k, row, last, first, ew, e, a, eB, aB, eH, aH, hle, hla, hre, hra);
                const int ph = __popc(B.H), pv = __popc(B.V);
                msk = B.H; kind = 1;
                if (r >= ph) {
                    r -= ph; msk = B.V; kind = 2;
                    if (r >= pv) {
                        r -= pv; msk = B.L; kind = 3;
                        if (r >= (int)B.L) { r -= (int)B.L; msk = B.N; kind = 4; }
                    }
                }
            }
            x = select_bit(msk, r);
            code = kind * 32 + x;
        }
        code = __shfl_sync(FULLW, code, owner);
        const int kind = code >> 5, x = code & 31, y = owner;
        // apply: the changed sites' masks (site events change one site;
        // B2 adsorption makes both ends B, the reaction both ends empty)
        const uint32_t bit = 1u << x;
        if (kind == 0) {
            if (lane == y) {
                if (k == 0) { e &= ~bit; a |= bit; }
                else { a &= ~bit; e |= bit; }
            }
        } else {
            const bool toB = k == 1;
            // the ends: (x, y) always except for the top-halo bond's halo end;
            // the other end by kind
            uint32_t m0 = 0u, m1 = 0u;  // bits of row y and of the row below to change
            bool hr1 = false, hl1 = false, top1 = false, bot1 = false;
            if (kind == 1) { m0 = bit | (x < 31 ? bit << 1 : 0u); hr1 = x == 31; }
            else if (kind == 2) { m0 = bit; m1 = bit; bot1 = y == qy - 1; }
            else if (kind == 3) { m0 = 1u; hl1 = true; }
            else { m0 = bit; top1 = true; }
            if (lane == y) {
                e = toB ? (e & ~m0) : (e | m0);
                a &= ~m0;
                if (hr1) { hre = toB ? 0u : 1u; hra = 0u; }
                if (hl1) { hle = toB ? 0u : 1u; hla = 0u; }
                if (top1 || bot1) { eH = toB ? (eH & ~bit) : (eH | bit); aH &= ~bit; }
            }
            if (kind == 2 && !bot1 && lane == y + 1) {
                e = toB ? (e & ~m1) : (e | m1);
                a &= ~m1;
            }
        }
        ++ev;
    }

    // Write back: the cell's rows, and the owned halo ends (the halo columns
    // in E windows, the halo rows in O windows)
    uint8_t *const out = C.dst;
    const int lx = C.lx, ly = C.ly, X0 = C.X0, Y0 = C.Y0;
    if (row) zgb_store_row(out + (int64_t)(Y0 + lane) * lx + X0, e, a);
    if (ew) {
        if (row) {
            const int gy = Y0 + lane;
            const int gxl = X0 > 0 ? X0 - 1 : lx - 1, gxr = X0 + 32 < lx ? X0 + 32 : 0;
            out[(int64_t)gy * lx + gxl] = (uint8_t)(hle ? 0 : (hla ? 1 : 2));
            out[(int64_t)gy * lx + gxr] = (uint8_t)(hre ? 0 : (hra ? 1 : 2));
        }
    } else {
        if (first) zgb_store_row(out + (int64_t)(Y0 > 0 ? Y0 - 1 : ly - 1) * lx + X0, eH, aH);
        if (last) zgb_store_row(out + (int64_t)(Y0 + qy < ly ? Y0 + qy : 0) * lx + X0, eH, aH);
    }
    return ev;
}

}  // namespace

}  // namespace fskmc
