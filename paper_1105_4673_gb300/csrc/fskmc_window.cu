// Fractional-step window kernel: one warp per coarse cell.
//
// In a window of colour c and length h every cell of colour c runs its own
// serial SSA (Eqs. totalrate and skeleton) on its sites, reading neighbours
// outside its write set as they were when the window began (Section 2.2,
// Step 1 / Step 3). The cell's write set lives in shared memory for the whole
// window; the rate-class counts are exact integers kept incrementally; the
// chosen member is found by an integer rank search over per-lane membership
// bit masks (popcount, warp prefix scan, ballot).
//
// Per event, in the binary64 clock mode, the arithmetic is exactly the
// oracle's: lambda is the ordered fused multiply-add chain over the class
// counts, the waiting time is -log(u_t)/lambda, the class is the first k with
// u_c*lambda < P_k (P_k the same chain's partial sums), the member is the
// j-th of its class in canonical order with j = (w3 * n_k) >> 32. Only log()
// may differ from the host's by an ulp; a window whose edge decision lands
// within 1e-12 (relative) of the edge is counted as ambiguous.
//
// Lanes own contiguous runs of s = ceil(qx*qy/32) sites in local row-major
// order, so the canonical member order (site-major, then slot) is lane-major.
#include <cuda/atomic>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "fskmc_internal.h"
#include "fskmc_persistent.h"
#include "philox.cuh"

namespace fskmc {

namespace {

constexpr double EDGE_TOL = 1e-12;
constexpr uint32_t MAX_EVENTS_PER_WINDOW = 1u << 26;

template <int MODEL>
struct Traits;
// K classes; KS site classes and KB slot classes with their own masks;
// HW halo width; R radius (in sites) within which an event can change a
// member's class.
template <> struct Traits<ADSDES> { static constexpr int K = 10, KS = 10, KB = 0, HW = 1, R = 1; };
template <> struct Traits<ISING> { static constexpr int K = 10, KS = 10, KB = 0, HW = 1, R = 1; };
template <> struct Traits<DIFFUSION> { static constexpr int K = 15, KS = 10, KB = 5, HW = 2, R = 2; };
template <> struct Traits<ZGB> { static constexpr int K = 4, KS = 2, KB = 2, HW = 1, R = 1; };

__device__ __forceinline__ int dir_dx(int d) { return d == 1 ? 1 : (d == 3 ? -1 : 0); }
__device__ __forceinline__ int dir_dy(int d) { return d == 0 ? -1 : (d == 2 ? 1 : 0); }

// Is class k a slot (two-site) class, and which mask holds it.
template <int MODEL>
__device__ __forceinline__ bool is_slot(int k)
{
    if (MODEL == DIFFUSION) return k >= 10;
    if (MODEL == ZGB) return k == 1 || k == 2;
    return false;
}
template <int MODEL>
__device__ __forceinline__ int mask_of(int k)
{
    if (MODEL == DIFFUSION) return k >= 10 ? k - 10 : k;
    if (MODEL == ZGB) return k == 0 ? 0 : (k == 3 ? 1 : k - 1);
    return k;
}
template <int MODEL>
__device__ __forceinline__ int slot_class_of_mask(int mb)
{
    return MODEL == DIFFUSION ? 10 + mb : 1 + mb;
}

// Box = the cell plus a halo of HW sites, row stride BW.
template <int MODEL>
__device__ __forceinline__ int occ4(const uint8_t *box, int BW, int p)
{
    return (box[p - BW] == 1) + (box[p + 1] == 1) + (box[p + BW] == 1) + (box[p - 1] == 1);
}

template <int MODEL>
__device__ __forceinline__ int site_class(const uint8_t *box, int BW, int p)
{
    int s = box[p];
    if (MODEL == ZGB) return s == 0 ? 0 : (s == 1 ? 3 : -1);
    return 5 * s + occ4<MODEL>(box, BW, p);
}

template <int MODEL>
__device__ __forceinline__ int slot_class(const uint8_t *box, int BW, int po, int pt)
{
    int so = box[po], st = box[pt];
    if (MODEL == DIFFUSION) return (so == 1 && st == 0) ? 10 + occ4<MODEL>(box, BW, po) : -1;
    if (MODEL == ZGB) {
        if (so == 0 && st == 0) return 1;
        if ((so == 1 && st == 2) || (so == 2 && st == 1)) return 2;
        return -1;
    }
    return -1;
}

// Does a cell of colour col own slot d (0..3 outward, 4..7 inward) of local
// site (lx, ly)? Bonds inside the cell belong to it; a horizontal bond across
// a cell edge belongs to the E cell, a vertical one to the O cell.
__device__ __forceinline__ bool slot_owned(int lx, int ly, int d, int qx, int qy, int col)
{
    int dir = d & 3;
    int nlx = lx + dir_dx(dir), nly = ly + dir_dy(dir);
    bool inside = nlx >= 0 && nlx < qx && nly >= 0 && nly < qy;
    bool cross = (dir & 1) ? (col == 0) : (col == 1);
    return (d >= 4) ? (!inside && cross) : (inside || cross);
}

// binary64 / binary32 clock arithmetic.
template <typename T>
struct Clock;
template <>
struct Clock<double> {
    static __device__ __forceinline__ double neglog_ut(uint32_t w0, uint32_t w1)
    {
        uint64_t b = ((uint64_t)w0 << 21) | (uint64_t)(w1 >> 11);
        double u = __dmul_rn(__ull2double_rn(b + 1ull), 0x1p-53);
        return -log(u);
    }
    static __device__ __forceinline__ double uc(uint32_t w2)
    {
        return __dmul_rn(__dadd_rn(__uint2double_rn(w2), 0.5), 0x1p-32);
    }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ double rate(const Replica &R, int k) { return R.r[k]; }
};
template <>
struct Clock<float> {
    static __device__ __forceinline__ float neglog_ut(uint32_t w0, uint32_t)
    {
        float u = __fmul_rn(__uint2float_rn((w0 >> 8) + 1u), 0x1p-24f);
        return -logf(u);
    }
    static __device__ __forceinline__ float uc(uint32_t w2)
    {
        return __fmul_rn(__fadd_rn(__uint2float_rn(w2 >> 8), 0.5f), 0x1p-24f);
    }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
    static __device__ __forceinline__ float rate(const Replica &R, int k) { return R.rf[k]; }
};

// Position of the r-th (0-based) set bit of m (r < popc(m)).
__device__ __forceinline__ int select_bit(uint32_t m, int r)
{
    int pos = 0, c;
    c = __popc(m & 0xFFFFu); if (r >= c) { r -= c; m >>= 16; pos += 16; }
    c = __popc(m & 0xFFu);   if (r >= c) { r -= c; m >>= 8;  pos += 8; }
    c = __popc(m & 0xFu);    if (r >= c) { r -= c; m >>= 4;  pos += 4; }
    c = __popc(m & 0x3u);    if (r >= c) { r -= c; m >>= 2;  pos += 2; }
    c = (int)(m & 1u);       if (r >= c) { pos += 1; }
    return pos;
}

struct Layout {
    int BW, BH, nsite, s, SW;
    int box_bytes, scls_bytes, sitemask_words, slotmask_words;
    int bytes;
};

template <int MODEL>
__host__ __device__ inline Layout make_layout(int qx, int qy)
{
    using TR = Traits<MODEL>;
    Layout L;
    L.BW = qx + 2 * TR::HW;
    L.BH = qy + 2 * TR::HW;
    L.nsite = qx * qy;
    L.s = (L.nsite + 31) / 32;
    L.SW = TR::KB ? (8 * L.s + 31) / 32 : 0;
    L.box_bytes = (L.BW * L.BH + 15) & ~15;
    L.scls_bytes = (L.nsite + 15) & ~15;
    L.sitemask_words = TR::KS * 32;
    L.slotmask_words = TR::KB * L.SW * 32;
    L.bytes = L.box_bytes + L.scls_bytes + 4 * (L.sitemask_words + L.slotmask_words) +
              4 * MAX_CLASSES;
    return L;
}

// Global-memory access for staging: through L2 only in the persistent
// kernel, whose cells read sites that other SMs wrote within the same launch.
template <bool PERSIST>
__device__ __forceinline__ uint8_t ld_site(const uint8_t *p)
{
    if (PERSIST) return __ldcg(p);
    return *p;
}

// Copy the sites of inactive cell (cx, cy) that no active cell writes in a
// window of colour col (ping-pong mode): columns 1..qx-2 of an O cell in E
// windows, rows 1..qy-2 of an E cell in O windows.
template <bool PERSIST>
__device__ void copy_unwritten(const uint8_t *src, uint8_t *dst, int lx, int ly, int qx, int qy,
                               int cx, int cy, int col, int lane)
{
    const int X0 = cx * qx, Y0 = cy * qy;
    if (col == 0) {
        for (int i = lane; i < qy * (qx - 2); i += 32) {
            int yy = Y0 + i / (qx - 2), xx = X0 + 1 + i % (qx - 2);
            int64_t o = (int64_t)yy * lx + xx;
            dst[o] = ld_site<PERSIST>(src + o);
        }
    } else {
        for (int i = lane; i < qx * (qy - 2); i += 32) {
            int yy = Y0 + 1 + i / qx, xx = X0 + i % qx;
            int64_t o = (int64_t)yy * lx + xx;
            dst[o] = ld_site<PERSIST>(src + o);
        }
    }
}

// One cell's fractional window. Returns the number of events; *amb is set
// if an edge decision landed within EDGE_TOL of the window end.
template <int MODEL, typename CLK, bool PERSIST>
__device__ uint32_t cell_window(uint8_t *wsm, const Replica &R, int qx, int qy, int cx, int cy,
                                int colour, uint32_t w, double hwin, uint64_t seed,
                                const uint8_t *src, uint8_t *dst, int lane, bool *amb_out,
                                bool *bad_out)
{
    using TR = Traits<MODEL>;
    using C = Clock<CLK>;
    constexpr int K = TR::K, HW = TR::HW, RR = TR::R;

    const Layout Lo = make_layout<MODEL>(qx, qy);
    uint8_t *box = wsm;
    uint8_t *scls = wsm + Lo.box_bytes;
    uint32_t *sitemask = reinterpret_cast<uint32_t *>(scls + Lo.scls_bytes);
    uint32_t *slotmask = sitemask + Lo.sitemask_words;
    int *cnt = reinterpret_cast<int *>(slotmask + Lo.slotmask_words);

    const int lx = R.lx, ly = R.ly;
    const int m = cy * R.ncx + cx;
    const int X0 = cx * qx, Y0 = cy * qy;
    const int BW = Lo.BW, BH = Lo.BH, s = Lo.s, SW = Lo.SW, nsite = Lo.nsite;

    // Stage the cell and its halo (periodic wrap) from the window-start state.
    for (int i = lane; i < BW * BH; i += 32) {
        int by = i / BW, bx = i - by * BW;
        int gy = Y0 - HW + by, gx = X0 - HW + bx;
        gy += (gy < 0) ? ly : 0; gy -= (gy >= ly) ? ly : 0;
        gx += (gx < 0) ? lx : 0; gx -= (gx >= lx) ? lx : 0;
        box[i] = ld_site<PERSIST>(src + (int64_t)gy * lx + gx);
    }
    for (int i = lane; i < Lo.sitemask_words + Lo.slotmask_words; i += 32) sitemask[i] = 0u;
    if (lane < MAX_CLASSES) cnt[lane] = 0;
    __syncwarp();

    // Class build: each lane classifies its own run of sites and slots.
    const int i0 = lane * s;
    for (int t = 0; t < s; ++t) {
        int i = i0 + t;
        if (i >= nsite) break;
        int llx = i % qx, lly = i / qx;
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

    // SSA loop (Eqs. totalrate and skeleton on the cell).
    CLK rk[K];
#pragma unroll
    for (int k = 0; k < K; ++k) rk[k] = C::rate(R, k);
    const CLK h = (CLK)hwin;
    CLK tau = (CLK)0;
    bool amb = false;
    uint32_t e = 0;
    uint32_t rw2 = 0, rw3 = 0;
    CLK rl = (CLK)0;
    const uint32_t ctr3 = R.rep | (TAG_EVENT << 24);

    for (;;) {
        CLK P[K];
        CLK lam = (CLK)0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            lam = C::fma((CLK)cnt[k], rk[k], lam);
            P[k] = lam;
        }
        if (lam == (CLK)0) break;
        if (e >= MAX_EVENTS_PER_WINDOW) {  // cannot happen with sane rates; never loop unboundedly
            *bad_out = true;
            break;
        }
        if ((e & 31u) == 0u) {
            // 32 events' draws at once, one Philox block per lane
            u32x4 o = draw(seed, e + (uint32_t)lane, w, (uint32_t)m, ctr3);
            rl = C::neglog_ut(o.x, o.y);
            rw2 = o.z;
            rw3 = o.w;
        }
        const int src_lane = (int)(e & 31u);
        const CLK l = __shfl_sync(0xffffffffu, rl, src_lane);
        const uint32_t w2 = __shfl_sync(0xffffffffu, rw2, src_lane);
        const uint32_t w3 = __shfl_sync(0xffffffffu, rw3, src_lane);
        const CLK E = C::div(l, lam);
        const CLK end = C::add(tau, E);
        if (fabs((double)end - (double)h) < EDGE_TOL * (double)h) amb = true;
        if (end >= h) break;
        tau = end;

        const CLK t = C::mul(C::uc(w2), lam);
        int k = -1;
#pragma unroll
        for (int kk = K - 1; kk >= 0; --kk)
            if (t < P[kk]) k = kk;
        if (k < 0) {  // binary32 only: t rounded up to lambda; take the last non-empty class
#pragma unroll
            for (int kk = 0; kk < K; ++kk)
                if (cnt[kk] > 0 && rk[kk] > (CLK)0) k = kk;
            if (k < 0) break;
        }
        const int nk = cnt[k];
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
        if (slot) { site = owner * s + (pick >> 3); d = pick & 7; }
        else { site = owner * s + pick; }
        const int slx = site % qx, sly = site / qx;
        const int p = (sly + HW) * BW + slx + HW;
        int po = p, pt = p;
        if (slot) {
            int dir = d & 3;
            int pn = p + dir_dy(dir) * BW + dir_dx(dir);
            if (d < 4) pt = pn; else po = pn;
        }
        // Apply the event (the update sigma -> sigma^{x,omega}).
        if (lane == 0) {
            if (MODEL == ADSDES || MODEL == ISING) {
                box[p] ^= 1;
            } else if (MODEL == DIFFUSION) {
                if (k < 10) box[p] ^= 1;
                else { box[po] = 0; box[pt] = 1; }
            } else {
                if (k == 0) box[p] = 1;
                else if (k == 3) box[p] = 0;
                else if (k == 1) { box[po] = 2; box[pt] = 2; }
                else { box[po] = 0; box[pt] = 0; }
            }
        }
        __syncwarp();

        // Refresh the classes of every site within RR of the changed sites,
        // one site per lane.
        {
            int ox = (po % BW) - HW, oy = (po / BW) - HW;
            int tx = (pt % BW) - HW, ty = (pt / BW) - HW;
            int x0 = min(ox, tx) - RR, x1 = max(ox, tx) + RR;
            int y0 = min(oy, ty) - RR, y1 = max(oy, ty) + RR;
            int rw = x1 - x0 + 1;
            int ux = x0 + lane % rw, uy = y0 + lane / rw;
            if (lane < rw * (y1 - y0 + 1) && ux >= 0 && ux < qx && uy >= 0 && uy < qy) {
                int i = uy * qx + ux;
                int own = i / s, tt = i - own * s;
                int pu = (uy + HW) * BW + ux + HW;
                int knew = site_class<MODEL>(box, BW, pu);
                int kold = (int8_t)scls[i];
                if (knew != kold) {
                    scls[i] = (uint8_t)knew;
                    uint32_t bit = 1u << tt;
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
                        int dir = dd & 3;
                        int pn = pu + dir_dy(dir) * BW + dir_dx(dir);
                        int kn = (dd < 4) ? slot_class<MODEL>(box, BW, pu, pn)
                                          : slot_class<MODEL>(box, BW, pn, pu);
                        int bitpos = tt * 8 + dd;
                        int wofs = (bitpos >> 5) * 32 + own;
                        uint32_t bit = 1u << (bitpos & 31);
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
        __syncwarp();
        ++e;
    }

    // Write back the write set: own sites, plus the halo ends of owned cross
    // bonds for the two-site models (columns in E windows, rows in O windows).
    for (int i = lane; i < nsite; i += 32) {
        int llx = i % qx, lly = i / qx;
        dst[(int64_t)(Y0 + lly) * lx + X0 + llx] = box[(lly + HW) * BW + llx + HW];
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
    return e;
}

// Plain engine: one launch per window, one warp per active cell of one replica.
template <int MODEL, typename CLK>
__global__ void __launch_bounds__(512) fs_window_kernel(WindowArgs a, int nactive, int smem_per_warp)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int g = blockIdx.x * (blockDim.x >> 5) + wib;
    if (g >= nactive) return;
    const Replica &R = a.reps[a.rep_index];
    const int half = R.ncx >> 1;
    const int cy = g / half;
    const int cx = 2 * (g % half) + ((a.colour + cy) & 1);
    const uint8_t *src = a.src + R.lat_off;
    uint8_t *dst = a.dst + R.lat_off;
    if (a.src != a.dst) {
        // the inactive neighbour whose unwritten sites this warp copies:
        // right of an E cell, below an O cell
        int ncx2 = a.colour == 0 ? (cx + 1) % R.ncx : cx;
        int ncy2 = a.colour == 0 ? cy : (cy + 1) % R.ncy;
        copy_unwritten<false>(src, dst, R.lx, R.ly, a.qx, a.qy, ncx2, ncy2, a.colour, lane);
    }
    bool amb = false, bad = false;
    uint32_t e = cell_window<MODEL, CLK, false>(smem + (size_t)wib * smem_per_warp, R, a.qx, a.qy,
                                                cx, cy, a.colour, a.w, a.h, a.seed, src, dst,
                                                lane, &amb, &bad);
    if (lane == 0) {
        a.workload[R.cell_off + cy * R.ncx + cx] = (int32_t)e;
        atomicAdd(&a.counters[0], (unsigned long long)e);
        if (amb) atomicAdd(&a.counters[1], 1ull);
        if (bad) atomicAdd(&a.counters[3], 1ull);
    }
}

// ---------------------------------------------------------------------------
// Persistent engine. Tasks are (window i, replica r, cell m) for every cell,
// active or not, dequeued from one global counter in the order: window-major;
// within a window all active cells (every replica) before all inactive ones.
// A task waits only on tasks that precede it in that order, so a dequeued
// task's prerequisites are always held by running warps.
//   epoch[m] = i + 1 once every write to, and read of, cell m's sites for
//   windows <= i is complete.
//   Active (m, i): needs epoch >= i on m and its 4 edge neighbours (in place)
//   or its 3x3 neighbourhood (ping-pong), then runs the window.
//   Inactive (m, i): in ping-pong mode waits on its 3x3 neighbourhood and
//   copies its unwritten sites; then waits until its 4 active edge
//   neighbours (the only cells that write into it) reach epoch i + 1.
// Every wait polls at most spin_limit times; on expiry the warp raises the
// abort flag, counts a timeout and the whole launch drains.
// ---------------------------------------------------------------------------
struct PParams {
    const Replica *reps;
    int32_t nrep, qx, qy;
    uint8_t *lat, *lat2;
    int32_t *workload;
    unsigned long long *counters;
    const int32_t *act_prefix;  // [nrep + 1] prefix sums of active cells per window
    int32_t total_cells, total_active;
    const int8_t *colour;
    int32_t colour_per_replica;
    const double *h;
    int64_t nwin;
    uint32_t w0;
    uint64_t seed;
    uint32_t spin_limit;
    int32_t *epoch;
    unsigned long long *queue;
    int32_t *abort_flag;
};

__device__ __forceinline__ int ld_acquire(const int32_t *p)
{
    cuda::atomic_ref<const int32_t, cuda::thread_scope_device> a(*p);
    return a.load(cuda::memory_order_acquire);
}

// Lanes 0..nd-1 poll deps[lane] until epoch >= target. Returns false on
// timeout or abort.
__device__ bool wait_epochs(const int32_t *ep, int dep, bool has_dep, int target,
                            const PParams &P, int lane)
{
    uint32_t spins = 0;
    for (;;) {
        bool ok = !has_dep || ld_acquire(ep + dep) >= target;
        if (__all_sync(0xffffffffu, ok)) break;
        if (spins >= P.spin_limit) {
            if (lane == 0) {
                atomicExch(P.abort_flag, 1);
                atomicAdd(&P.counters[2], 1ull);
            }
            return false;
        }
        ++spins;
        if ((spins & 63u) == 0u) {
            int ab = *(volatile int32_t *)P.abort_flag;
            if (__any_sync(0xffffffffu, ab != 0)) return false;
        }
        __nanosleep(spins < 64 ? 20 : 200);
    }
    __threadfence();
    __syncwarp();
    return true;
}

template <int MODEL, typename CLK>
__global__ void __launch_bounds__(256) fs_persistent_kernel(const PParams *pp, int smem_per_warp)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const PParams P = *pp;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    uint8_t *wsm = smem + (size_t)wib * smem_per_warp;
    const bool pingpong = P.lat2 != nullptr;
    const unsigned long long total = (unsigned long long)P.nwin * (unsigned long long)P.total_cells;

    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(P.queue, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= total) break;
        int ab = 0;
        if (lane == 0) ab = *(volatile int32_t *)P.abort_flag;
        if (__shfl_sync(0xffffffffu, ab, 0)) break;
        const int i = (int)(t / (unsigned long long)P.total_cells);
        const int u = (int)(t % (unsigned long long)P.total_cells);
        const bool active = u < P.total_active;
        const int a = active ? u : u - P.total_active;
        int lo = 0, hi = P.nrep;  // last r with act_prefix[r] <= a
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (P.act_prefix[mid] <= a) lo = mid; else hi = mid;
        }
        const int r = lo;
        const int k = a - P.act_prefix[r];
        const Replica &R = P.reps[r];
        const int wcol = P.colour[P.colour_per_replica ? (int64_t)r * P.nwin + i : i];
        const int ccol = active ? wcol : 1 - wcol;
        const int half = R.ncx >> 1;
        const int cy = k / half;
        const int cx = 2 * (k % half) + ((ccol + cy) & 1);
        const int m = cy * R.ncx + cx;
        int32_t *ep = P.epoch + R.cell_off;
        uint8_t *cur = (pingpong && (i & 1)) ? P.lat2 : P.lat;
        uint8_t *nxt = pingpong ? ((i & 1) ? P.lat : P.lat2) : cur;
        cur += R.lat_off;
        nxt += R.lat_off;

        // dependency of this lane: 3x3 neighbourhood (lanes 0..8) or
        // self + 4 edge neighbours (lanes 0..4)
        int ddx = 0, ddy = 0;
        bool has = false;
        if (pingpong) {
            has = lane < 9;
            ddx = lane % 3 - 1;
            ddy = lane / 3 - 1;
        } else {
            has = lane < 5;
            ddx = lane == 1 ? 1 : (lane == 3 ? -1 : 0);
            ddy = lane == 2 ? 1 : (lane == 4 ? -1 : 0);
        }
        const int dcx = (cx + ddx + R.ncx) % R.ncx, dcy = (cy + ddy + R.ncy) % R.ncy;
        const int dep = dcy * R.ncx + dcx;
        bool ok = true;
        if (active || pingpong) ok = wait_epochs(ep, dep, has, i, P, lane);
        if (!ok) break;
        if (active) {
            bool amb = false, bad = false;
            uint32_t e = cell_window<MODEL, CLK, true>(wsm, R, P.qx, P.qy, cx, cy, ccol,
                                                      P.w0 + (uint32_t)i, P.h[i], P.seed, cur,
                                                      nxt, lane, &amb, &bad);
            if (lane == 0) {
                P.workload[R.cell_off + m] = (int32_t)e;
                atomicAdd(&P.counters[0], (unsigned long long)e);
                if (amb) atomicAdd(&P.counters[1], 1ull);
                if (bad) atomicAdd(&P.counters[3], 1ull);
            }
        } else {
            if (pingpong) copy_unwritten<true>(cur, nxt, R.lx, R.ly, P.qx, P.qy, cx, cy, wcol, lane);
            // the active edge neighbours write into this cell: wait for them
            int ex = lane == 0 ? 1 : (lane == 1 ? -1 : 0);
            int ey = lane == 2 ? 1 : (lane == 3 ? -1 : 0);
            int ncx2 = (cx + ex + R.ncx) % R.ncx, ncy2 = (cy + ey + R.ncy) % R.ncy;
            ok = wait_epochs(ep, ncy2 * R.ncx + ncx2, lane < 4, i + 1, P, lane);
            if (!ok) break;
        }
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            cuda::atomic_ref<int32_t, cuda::thread_scope_device> ea(ep[m]);
            ea.store(i + 1, cuda::memory_order_release);
        }
    }
}
template <int MODEL>
cudaError_t launch_model(int fp32, const WindowArgs &a, int nactive, int wpb, cudaStream_t st)
{
    const int spw = make_layout<MODEL>(a.qx, a.qy).bytes;
    size_t smem = (size_t)spw * wpb;
    int blocks = (nactive + wpb - 1) / wpb;
    if (blocks == 0) return cudaSuccess;
    if (fp32) {
        auto kern = fs_window_kernel<MODEL, float>;
        if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<blocks, 32 * wpb, smem, st>>>(a, nactive, spw);
    } else {
        auto kern = fs_window_kernel<MODEL, double>;
        if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<blocks, 32 * wpb, smem, st>>>(a, nactive, spw);
    }
    return cudaGetLastError();
}

template <int MODEL>
void *persistent_kernel_ptr(int fp32)
{
    return fp32 ? (void *)fs_persistent_kernel<MODEL, float> : (void *)fs_persistent_kernel<MODEL, double>;
}

void *persistent_kernel_for(int model, int fp32)
{
    switch (model) {
    case ADSDES: return persistent_kernel_ptr<ADSDES>(fp32);
    case ISING: return persistent_kernel_ptr<ISING>(fp32);
    case DIFFUSION: return persistent_kernel_ptr<DIFFUSION>(fp32);
    case ZGB: return persistent_kernel_ptr<ZGB>(fp32);
    }
    return nullptr;
}

}  // namespace

size_t window_smem_per_warp(int model, int qx, int qy)
{
    switch (model) {
    case ADSDES: return make_layout<ADSDES>(qx, qy).bytes;
    case ISING: return make_layout<ISING>(qx, qy).bytes;
    case DIFFUSION: return make_layout<DIFFUSION>(qx, qy).bytes;
    case ZGB: return make_layout<ZGB>(qx, qy).bytes;
    }
    return 0;
}

cudaError_t launch_window(int model, int fp32, const WindowArgs &a, int nactive, int wpb,
                          cudaStream_t st)
{
    switch (model) {
    case ADSDES: return launch_model<ADSDES>(fp32, a, nactive, wpb, st);
    case ISING: return launch_model<ISING>(fp32, a, nactive, wpb, st);
    case DIFFUSION: return launch_model<DIFFUSION>(fp32, a, nactive, wpb, st);
    case ZGB: return launch_model<ZGB>(fp32, a, nactive, wpb, st);
    }
    return cudaErrorInvalidValue;
}

// Device buffers of the persistent engine and the graph that launches it:
// reset the per-cell epochs and the queue, then run the persistent kernel.
struct PersistentState {
    int model = -1, fp32 = -1, wpb = -1, grid = 0;
    PParams *d_params = nullptr;
    int32_t *d_epoch = nullptr;
    unsigned long long *d_queue = nullptr;  // [0] queue, [1] abort flag (low word)
    int32_t *d_prefix = nullptr;
    int8_t *d_colour = nullptr;
    size_t colour_cap = 0;
    double *d_h = nullptr;
    size_t h_cap = 0;
    int32_t total_cells = 0;
    int32_t *h_abort = nullptr;  // pinned
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
};

void persistent_free(PersistentState *st)
{
    if (!st) return;
    if (st->exec) cudaGraphExecDestroy(st->exec);
    if (st->graph) cudaGraphDestroy(st->graph);
    cudaFree(st->d_params);
    cudaFree(st->d_epoch);
    cudaFree(st->d_queue);
    cudaFree(st->d_prefix);
    cudaFree(st->d_colour);
    cudaFree(st->d_h);
    cudaFreeHost(st->h_abort);
    delete st;
}

#define PCK(call)                                                     \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) { *msg = #call; return e_; }           \
    } while (0)

cudaError_t persistent_run(PersistentState **pst, const PersistentRun &run, cudaStream_t s,
                           std::string *msg)
{
    if (run.nwin == 0) return cudaSuccess;
    PersistentState *st = *pst;
    if (!st) {
        st = new PersistentState();
        *pst = st;
        PCK(cudaMalloc(&st->d_params, sizeof(PParams)));
        PCK(cudaMalloc(&st->d_epoch, sizeof(int32_t) * (size_t)run.total_cells));
        PCK(cudaMalloc(&st->d_queue, 2 * sizeof(unsigned long long)));
        PCK(cudaMalloc(&st->d_prefix, sizeof(int32_t) * (size_t)(run.nrep + 1)));
        PCK(cudaMallocHost(&st->h_abort, sizeof(int32_t)));
        std::vector<int32_t> pre(run.nrep + 1, 0);
        for (int r = 0; r < run.nrep; ++r)
            pre[r + 1] = pre[r] + run.reps_host[r].ncx * run.reps_host[r].ncy / 2;
        PCK(cudaMemcpyAsync(st->d_prefix, pre.data(), sizeof(int32_t) * pre.size(),
                            cudaMemcpyHostToDevice, s));
        st->total_cells = run.total_cells;
    }
    // (Re)build the graph when the kernel variant or launch shape changes.
    if (st->model != run.model || st->fp32 != run.fp32 || st->wpb != run.wpb) {
        if (st->exec) { cudaGraphExecDestroy(st->exec); st->exec = nullptr; }
        if (st->graph) { cudaGraphDestroy(st->graph); st->graph = nullptr; }
        void *kern = persistent_kernel_for(run.model, run.fp32);
        const int spw = (int)window_smem_per_warp(run.model, run.qx, run.qy);
        const size_t smem = (size_t)spw * run.wpb;
        PCK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0, dev = 0, nsm = 0;
        PCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * run.wpb, smem));
        PCK(cudaGetDevice(&dev));
        PCK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        if (per_sm < 1) { *msg = "persistent kernel does not fit on an SM"; return cudaErrorInvalidConfiguration; }
        st->grid = per_sm * nsm;
        cudaStream_t cs;
        PCK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        PCK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        cudaMemsetAsync(st->d_epoch, 0, sizeof(int32_t) * (size_t)st->total_cells, cs);
        cudaMemsetAsync(st->d_queue, 0, 2 * sizeof(unsigned long long), cs);
        const PParams *pp = st->d_params;
        void *args[] = {(void *)&pp, (void *)&spw};
        cudaLaunchKernel(kern, dim3(st->grid), dim3(32 * run.wpb), args, smem, cs);
        cudaError_t ce = cudaStreamEndCapture(cs, &st->graph);
        cudaStreamDestroy(cs);
        if (ce != cudaSuccess) { *msg = "graph capture"; return ce; }
        PCK(cudaGraphInstantiate(&st->exec, st->graph, 0));
        st->model = run.model;
        st->fp32 = run.fp32;
        st->wpb = run.wpb;
    }
    const size_t ncol = (size_t)run.nwin * (run.colour_per_replica ? run.nrep : 1);
    if (ncol > st->colour_cap) {
        cudaFree(st->d_colour);
        st->d_colour = nullptr;
        PCK(cudaMalloc(&st->d_colour, ncol));
        st->colour_cap = ncol;
    }
    if ((size_t)run.nwin > st->h_cap) {
        cudaFree(st->d_h);
        st->d_h = nullptr;
        PCK(cudaMalloc(&st->d_h, sizeof(double) * (size_t)run.nwin));
        st->h_cap = (size_t)run.nwin;
    }
    PCK(cudaMemcpyAsync(st->d_colour, run.colour, ncol, cudaMemcpyHostToDevice, s));
    PCK(cudaMemcpyAsync(st->d_h, run.h, sizeof(double) * (size_t)run.nwin, cudaMemcpyHostToDevice, s));
    PParams P;
    P.reps = run.reps_dev;
    P.nrep = run.nrep;
    P.qx = run.qx;
    P.qy = run.qy;
    P.lat = run.lat;
    P.lat2 = run.lat2;
    P.workload = run.workload;
    P.counters = run.counters;
    P.act_prefix = st->d_prefix;
    P.total_cells = run.total_cells;
    P.total_active = run.total_cells / 2;
    P.colour = st->d_colour;
    P.colour_per_replica = run.colour_per_replica ? 1 : 0;
    P.h = st->d_h;
    P.nwin = run.nwin;
    P.w0 = (uint32_t)run.w0;
    P.seed = run.seed;
    P.spin_limit = run.spin_limit;
    P.epoch = st->d_epoch;
    P.queue = st->d_queue;
    P.abort_flag = reinterpret_cast<int32_t *>(st->d_queue + 1);
    PCK(cudaMemcpyAsync(st->d_params, &P, sizeof P, cudaMemcpyHostToDevice, s));
    PCK(cudaGraphLaunch(st->exec, s));
    PCK(cudaMemcpyAsync(st->h_abort, P.abort_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PCK(cudaStreamSynchronize(s));
    if (*st->h_abort) { *msg = "a bounded wait gave up"; return cudaErrorTimeout; }
    return cudaSuccess;
}

}  // namespace fskmc
