// Device helpers shared by the window kernels (fskmc_window.cu: one cell
// per warp, all models; fskmc_group.cu: several small cells per warp,
// spin-flip models) and the persistent engine's task parameters.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "fskmc_internal.h"
#include "fskmc_logtab.h"
#include "philox.cuh"

namespace fskmc {

namespace {

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
template <> struct Traits<ISING1D> { static constexpr int K = 6, KS = 6, KB = 0, HW = 1, R = 1; };

// Spin-flip models: class = SPIN_STRIDE * sigma + n, n = occupied neighbours.
template <int MODEL>
constexpr bool is_spin_flip() { return MODEL == ADSDES || MODEL == ISING || MODEL == ISING1D; }

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
    if (MODEL == ISING1D) return 3 * s + (box[p - 1] == 1) + (box[p + 1] == 1);  // ring: x -+ 1
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

// Positions within a 4-bit nibble: entry 4n + r (2 bits) is the position of
// the r-th set bit of nibble n (0 where n has fewer than r + 1 set bits),
// packed 16 entries per 32-bit word.
struct NibbleSelect {
    uint32_t w[4];
};
__host__ __device__ constexpr NibbleSelect make_nibble_select()
{
    NibbleSelect t{{0u, 0u, 0u, 0u}};
    for (int n = 0; n < 16; ++n) {
        int r = 0;
        for (int b = 0; b < 4; ++b) {
            if ((n >> b) & 1) {
                const int idx = 4 * n + r;
                t.w[idx >> 4] |= (uint32_t)b << (2 * (idx & 15));
                ++r;
            }
        }
    }
    return t;
}

// Position of the r-th (0-based) set bit of m (r < popc(m); any other r
// gives some position in 0..31). Branch-free: byte popcounts by the SWAR
// bit-count steps, their running sums by one multiply, the byte holding the
// bit by a bytewise compare of those sums with r, then the nibble within
// the byte and a 2-bit table of positions within a nibble.
__device__ __forceinline__ int select_bit(uint32_t m, int r)
{
    constexpr NibbleSelect NS = make_nibble_select();
    uint32_t c = m - ((m >> 1) & 0x55555555u);
    c = (c & 0x33333333u) + ((c >> 2) & 0x33333333u);
    c = (c + (c >> 4)) & 0x0F0F0F0Fu;
    const uint32_t p = c * 0x01010101u;  // byte i: set bits in bytes 0..i (at most 32)
    // bytes whose running sum exceeds r have their top bit left set
    const uint32_t gt = ((p | 0x80808080u) - (uint32_t)(r + 1) * 0x01010101u) & 0x80808080u;
    const int b = min(4 - __popc(gt), 3);  // whole bytes before the bit
    const int sh = 8 * b;
    const int before = (int)(((p << 8) >> sh) & 0xFFu);
    const uint32_t v = (m >> sh) & 0xFFu;
    int rr = r - before;
    const int c4 = __popc(v & 15u);
    const bool hi = rr >= c4;
    const uint32_t nib = hi ? (v >> 4) : (v & 15u);
    rr -= hi ? c4 : 0;
    const int idx = ((int)nib * 4 + rr) & 63;
    const int q = idx >> 4;
    const uint32_t word = q < 2 ? (q == 0 ? NS.w[0] : NS.w[1]) : (q == 2 ? NS.w[2] : NS.w[3]);
    return sh + (hi ? 4 : 0) + (int)((word >> (2 * (idx & 15))) & 3u);
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv &f)
{
    return (uint32_t)(((uint64_t)n * f.M) >> 32);
}

// Bit pattern of a non-negative double: orders like the value.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }

// x (0 < x < 2^63) as a binary32 with its significand truncated to 24 bits,
// built on the integer pipes (the 64-bit conversion instruction runs on the
// FP64 pipe).
__device__ __forceinline__ float u64_to_float_rz(uint64_t x)
{
    const int lz = __clzll((long long)x);
    const uint32_t m = (uint32_t)((x << lz) >> 40);
    return __uint_as_float(((uint32_t)(190 - lz) << 23) | (m & 0x7FFFFFu));
}

// a / b rounded to nearest (ties to even) for a >= 0 and b > 0, on the
// integer pipes and branch-free. With 53-bit significands ma, mb the quotient
// significand is Q = floor(N / mb), N = ma 2^52 (ma >= mb) or ma 2^53, in
// [2^52, 2^53). A 64-bit fixed-point reciprocal X ~ 2^116 / mb is seeded by
// the binary32 reciprocal of mb's leading 24 bits (rcp.approx: relative error
// about 2^-22) and refined by two Newton-Raphson steps
// X <- X + X (2^116 - mb X) / 2^116 (each squares the relative error; the
// residual is formed exactly from the 128-bit product mb X). The estimate
// Q0 = (ma X) >> (116 - s) is then at most one below Q (checked on the CPU
// in exact integer arithmetic for 2^-21 seed errors); the exact remainder
// R = N - Q mb (its low 64 bits suffice, |R| < 2^63) corrects Q and decides
// the rounding (2R against mb), as in long division. GB300's FP64 pipe is the
// window kernels' scarcest unit; this keeps the divide off it. slow is set
// for operands or quotients outside the normal range (zero, subnormal, huge),
// where the caller uses the hardware divide.
__device__ __forceinline__ double div_int(double a, double b, bool &slow)
{
    const unsigned long long A = (unsigned long long)__double_as_longlong(a);
    const unsigned long long B = (unsigned long long)__double_as_longlong(b);
    const int ea = (int)(A >> 52), eb = (int)(B >> 52);
    const unsigned long long FRAC = (1ull << 52) - 1ull;
    const unsigned long long ma = (A & FRAC) | (1ull << 52), mb = (B & FRAC) | (1ull << 52);
    const float mf = __uint_as_float(0x3F800000u | (uint32_t)((B >> 29) & 0x7FFFFFu));
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(mf));
    const uint32_t rb = __float_as_uint(rf);  // rf in (0.5, 1]: X0 = rf 2^64
    unsigned long long X = (rb >> 23) >= 127u ? ~0ull
                                               : (unsigned long long)((rb & 0x7FFFFFu) | 0x800000u) << 40;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const unsigned long long hi = __umul64hi(mb, X), lo = mb * X;
        const unsigned long long T = (hi << 12) | (lo >> 52);  // (mb X) >> 52, mod 2^64
        const long long E = (long long)(0ull - T);                // (2^116 - mb X) >> 52, signed
        const unsigned long long corr = __umul64hi(X, E < 0 ? (unsigned long long)(-E) : (unsigned long long)E);
        X = E < 0 ? X - corr - 1ull : X + corr;
    }
    const bool ge = ma >= mb;
    int e = ea - eb + (ge ? 1023 : 1022);
    const unsigned long long qh = __umul64hi(ma, X), ql = ma * X;
    unsigned long long Q = ge ? qh : ((qh << 1) | (ql >> 63));
    long long R = (long long)((ma << (ge ? 52 : 53)) - Q * mb);
    {
        const bool neg = R < 0;
        Q -= neg ? 1ull : 0ull;
        R += neg ? (long long)mb : 0ll;
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool big = R >= (long long)mb;
        Q += big ? 1ull : 0ull;
        R -= big ? (long long)mb : 0ll;
    }
    const unsigned long long R2 = (unsigned long long)R << 1;
    Q += (R2 > mb || (R2 == mb && (Q & 1ull))) ? 1ull : 0ull;
    const bool carry = Q == (1ull << 53);
    Q = carry ? (1ull << 52) : Q;
    e += carry ? 1 : 0;
    slow = ea == 0 || ea >= 2047 || eb == 0 || eb >= 2047 || e < 1 || e > 2046 || R < 0 ||
           R >= (long long)mb;
    return __longlong_as_double((long long)(((unsigned long long)e << 52) | (Q & FRAC)));
}

// a / b rounded to nearest (ties to even) for a >= 0 and b > 0: div_int, with
// the hardware divide for operands or quotients outside its range.
__device__ __forceinline__ double div_rn(double a, double b)
{
    bool slow;
    const double q = div_int(a, b, slow);
    return slow ? __ddiv_rn(a, b) : q;
}

// a / b rounded to nearest (ties to even) for a >= 0 and b > 0 without a
// divide instruction, branch-free, so that it can overlap other work of the
// event loop. The binary32 reciprocal of b's significand (rcp.approx, within
// one unit of its last place; with the truncation of the operand the seed
// is within 2^-22 of 1/b) is refined by two Newton-Raphson steps
// x <- x + x (1 - b x), each of which squares the relative error, so the
// rounded product q0 = a x lies within about two units in the last place of
// a / b. The exact remainder R = N - Q mb of the significand division
// (N = ma 2^52 or ma 2^53, Q the candidate significand) then corrects Q to
// floor(N / mb) and decides the rounding (2R against mb), as in long
// division. R fits in 64 bits because |Q - N/mb| is a few units, so only the
// low 64 bits of N and Q mb are needed. slow is set for operands or
// quotients outside the normal range (zero, subnormal, huge); the caller
// then uses the hardware divide.
__device__ __forceinline__ double div_newton(double a, double b, bool &slow)
{
    const unsigned long long A = (unsigned long long)__double_as_longlong(a);
    const unsigned long long B = (unsigned long long)__double_as_longlong(b);
    const int ea = (int)(A >> 52), eb = (int)(B >> 52);
    const unsigned long long FRAC = (1ull << 52) - 1ull;
    const unsigned long long ma = (A & FRAC) | (1ull << 52), mb = (B & FRAC) | (1ull << 52);
    // seed: 1 / (b's significand truncated to 24 bits) in binary32, rescaled
    const float mf = __uint_as_float(0x3F800000u | (uint32_t)((B >> 29) & 0x7FFFFFu));
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(mf));
    const uint32_t rb = __float_as_uint(rf);
    const uint32_t xe = (rb >> 23) + 1919u - (uint32_t)eb;  // binary64 exponent field of rf / 2^(eb-1023)
    const double x0 = __hiloint2double((int)((xe << 20) | ((rb >> 3) & 0xFFFFFu)), (int)(rb << 29));
    double t = __fma_rn(-b, x0, 1.0);
    double x = __fma_rn(x0, t, x0);
    t = __fma_rn(-b, x, 1.0);
    x = __fma_rn(x, t, x);
    const double q0 = __dmul_rn(a, x);
    // the result's binade: Q = floor(N / mb) in [2^52, 2^53)
    const bool ge = ma >= mb;
    int e = ea - eb + (ge ? 1023 : 1022);
    const unsigned long long Nlo = ma << (ge ? 52 : 53);
    const unsigned long long QB = (unsigned long long)__double_as_longlong(q0);
    const int eq = (int)(QB >> 52);
    const unsigned long long mq = (QB & FRAC) | (1ull << 52);
    unsigned long long Q = eq > e ? (mq << 1) : (eq < e ? (mq >> 1) : mq);
    long long R = (long long)(Nlo - Q * mb);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const bool neg = R < 0;
        Q -= neg ? 1ull : 0ull;
        R += neg ? (long long)mb : 0ll;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const bool big = R >= (long long)mb;
        Q += big ? 1ull : 0ull;
        R -= big ? (long long)mb : 0ll;
    }
    const unsigned long long R2 = (unsigned long long)R << 1;
    Q += (R2 > mb || (R2 == mb && (Q & 1ull))) ? 1ull : 0ull;
    const bool carry = Q == (1ull << 53);
    Q = carry ? (1ull << 52) : Q;
    e += carry ? 1 : 0;
    slow = ea == 0 || ea >= 2047 || eb == 0 || eb > 2044 || e < 1 || e > 2046 || eq < e - 1 || eq > e + 1 ||
           R < 0 || R >= (long long)mb;
    return __longlong_as_double((long long)(((unsigned long long)e << 52) | (Q & FRAC)));
}

// Exact binary64 value of an integer 0 <= n < 2^20, built on the integer
// pipes (exponent from the leading-zero count, significand by a shift).
__device__ __forceinline__ double small_to_double(int n)
{
    const int lz = __clz(n);
    const uint32_t hi = ((uint32_t)(1054 - lz) << 20) | (((uint32_t)n << ((lz - 11) & 31)) & 0xFFFFFu);
    return __hiloint2double(n ? (int)hi : 0, 0);
}

// v * 2^-s exactly, for 1 <= v < 2^53 and a result in the normal range,
// built on the integer pipes (exponent from the leading-zero count).
__device__ __forceinline__ double u53_scaled(uint64_t v, int s)
{
    const int lz = __clzll((long long)v);
    const uint64_t frac = ((v << lz) << 1) >> 12;
    return __longlong_as_double((long long)(((uint64_t)(1086 - lz - s) << 52) | frac));
}

// -log(u) for u = n 2^-53, 1 <= n <= 2^53: the waiting-time numerator of the
// binary64 clock. Table-driven (Tang's reduction in its reciprocal form; the
// tables and their derivation are in fskmc_logtab.h and gen_logtab.py):
// u = 2^E m with m in [0.75, 1.5); r = m invc - 1 is exact (one fused
// multiply-add, invc has 8 significant bits), log1p(r) for |r| <= 2^-7 is
// its Taylor polynomial to r^8, and E ln2_hi - log(invc)_hi is exact, so the
// only sizeable rounding is the last addition: within 0.66 units in the last
// place (correctly rounded for 99.6% of random n). Branch-free, so several
// calls in flight overlap; u = 1 gives +0.
__device__ __forceinline__ double neg_log_u53(uint64_t n)
{
    const int lz = __clzll((long long)n);
    const uint64_t frac = ((n << lz) << 1) >> 12;  // the 52 bits after n's leading one
    const int i = (int)(frac >> 45);               // the reduction interval
    const bool half = i >= 64;                     // m >= 1.5: use m / 2
    const double m = __longlong_as_double((long long)(((uint64_t)(half ? 1022 : 1023) << 52) | frac));
    const int ne = lz - 10 - (half ? 1 : 0);       // -E, 0 <= -E <= 53
    const double invc = __ldg(&LOG_TAB[i][0]), lch = __ldg(&LOG_TAB[i][1]), lcl = __ldg(&LOG_TAB[i][2]);
    const double r = __fma_rn(m, invc, -1.0);
    double q = __fma_rn(r, -0.125, 1.0 / 7.0);
    q = __fma_rn(r, q, -1.0 / 6.0);
    q = __fma_rn(r, q, 0.2);
    q = __fma_rn(r, q, -0.25);
    q = __fma_rn(r, q, 1.0 / 3.0);
    q = __fma_rn(r, q, -0.5);
    const double r2 = __dmul_rn(r, r);
    const double me = small_to_double(ne);          // -E
    const double hi = __fma_rn(-me, LOG_LN2_HI, lch);  // exact
    const double lo = __fma_rn(-me, LOG_LN2_LO, lcl);
    const double tail = __dadd_rn(r, __fma_rn(r2, q, lo));
    return __dsub_rn(0.0, __dadd_rn(hi, tail));
}

// Global-memory access for staging: through L2 only in the persistent
// kernel, whose cells read sites that other SMs wrote within the same launch.
// Where a cell sits: its origin (X0, Y0) in the periodic lx x ly lattice it
// is staged from and written back to, and its id m in the random counters
// (the cell's index in its lattice's cell grid).
struct CellAt {
    int X0, Y0, lx, ly;
    uint32_t m;
};

__device__ __forceinline__ CellAt cell_at(const Replica &R, const CellGeom &G, int cx, int cy)
{
    return CellAt{cx * G.qx, cy * G.qy, R.lx, R.ly, (uint32_t)(cy * R.ncx + cx)};
}

// Asynchronous 16-byte copy global -> shared (cp.async, cached in L2 only,
// so data other SMs wrote before an acquire are seen), and the wait for all
// of this thread's copies in flight. Both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

template <bool PERSIST>
__device__ __forceinline__ uint8_t ld_site(const uint8_t *p)
{
    if (PERSIST) return __ldcg(p);
    return *p;
}

// Screened window-edge check of the binary64 clock (Eq. skeleton: is
// end = tau + (-log u_t) / lambda past the window length h?). The waiting
// time is estimated in binary32 -- lf = -log u_t rounded toward zero, over
// lambda truncated to binary32, a reciprocal within one unit in the last
// place, three rounded products: at most 4.5 2^-23 relative error -- in
// units of h 2^-62 (sf = 2^62 / h in binary32) and added to an exact 64-bit
// integer clock clk. err bounds the distance of clk from the binary64 clock:
// 2^-20 of each estimate, plus 2^11 units per event for the truncation to an
// integer and the binary64 roundings of tau (at most 2^-52 h, i.e. 2^10
// units, each). Q and E are the event's estimate and the bound with it.
// take: clk + Q + E < 2^62, so the binary64 end lies before h; unsure:
// neither that nor clk + Q >= 2^62 + E (the binary64 end at or past h), or
// lambda outside the binary32 range, or screening off (ok false), or
// `near`: the caller then decides in binary64.
__device__ __forceinline__ void edge_screen(float lf, double lam, float sf, uint64_t clk, uint64_t err,
                                            bool ok, bool near, uint64_t &Q, uint64_t &E, bool &take,
                                            bool &unsure)
{
    const uint64_t lb = (uint64_t)dbits(lam);
    const int fe = (int)(lb >> 52) - 896;  // binary32 exponent field of lambda
    const bool inrange = ok && fe >= 1 && fe <= 250;
    const float lamf = __uint_as_float(((uint32_t)fe << 23) | (uint32_t)((lb >> 29) & 0x7FFFFFu));
    float rr;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rr) : "f"(lamf));
    const uint32_t qb = __float_as_uint(__fmul_rn(__fmul_rn(lf, rr), sf));
    const int qe = (int)(qb >> 23) - 150;  // estimate = (24-bit significand) 2^qe
    const uint64_t qm = (uint64_t)((qb & 0x7FFFFFu) | 0x800000u);
    Q = qe >= 40 ? (1ull << 63) : (qe >= 0 ? qm << qe : (qe > -24 ? qm >> -qe : 0ull));
    E = err + (Q >> 20) + 2048ull;
    const uint64_t rem = (1ull << 62) - clk;
    take = inrange && Q + E < rem;
    unsure = near || !inrange || (!take && Q < rem + E);
}

// binary32 2^62 / h for the screened edge check, and whether h is in its range
__device__ __forceinline__ bool edge_screen_scale(double h, bool on, float &sf)
{
    const bool ok = on && h > 1e-15 && h < 1e15;
    sf = ok ? (float)(0x1p62 / h) : 0.0f;
    return ok;
}

struct PParams {
    const Replica *reps;
    int32_t nrep;
    CellGeom geom;
    uint8_t *lat, *lat2;
    int32_t *workload;
    unsigned long long *counters;
    const int32_t *act_prefix;  // [nrep + 1] prefix sums of active cells per window
    const int2 *cell_rk;        // [total_active]: replica and index within it of a window's a-th active cell
    int32_t total_cells, total_active;
    const int8_t *colour;
    int32_t colour_per_replica;
    const int2 *prev;          // per (replica,) window: last earlier window of the same / other colour
    const int32_t *order;      // per replica and colour: active cells heaviest first, or null
    int32_t inplace;           // in-place models: only active cells have tasks
    int32_t screen;            // binary64 clock: screened window-edge decisions
    const double *h;
    int64_t nwin;
    uint32_t w0;
    uint64_t seed;
    uint32_t spin_limit;
    int32_t *epoch;
    unsigned long long *queue;
    int32_t *abort_flag;
};

// Lanes with has_dep poll ep[dep] until it reaches their target. Polls are
// relaxed loads with exponential back-off (128 ns doubling to 4 us), so
// waiting warps leave the issue slots to working ones; one acquire fence
// after success orders the cell's later reads. Returns false on timeout
// (after P.spin_limit polls) or when another warp raised the abort flag.
__device__ bool wait_epochs(const int32_t *ep, int dep, bool has_dep, int target,
                            const PParams &P, int lane)
{
    uint32_t spins = 0;
    unsigned ns = 128;
    for (;;) {
        bool ok = !has_dep || *(volatile const int32_t *)(ep + dep) >= target;
        if (__all_sync(0xffffffffu, ok)) break;
        if (spins >= P.spin_limit) {
            if (lane == 0) {
                atomicExch(P.abort_flag, 1);
                atomicAdd(&P.counters[2], 1ull);
            }
            return false;
        }
        ++spins;
        if ((spins & 15u) == 0u) {
            int ab = *(volatile int32_t *)P.abort_flag;
            if (__any_sync(0xffffffffu, ab != 0)) return false;
        }
        __nanosleep(ns);
        if ((spins & 3u) == 0u && ns < 4096u) ns <<= 1;
    }
    // the relaxed polls that saw the flags and this fence form an acquire;
    // the warp barrier orders the other lanes' later reads after it
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    __syncwarp();
    return true;
}

}  // namespace

}  // namespace fskmc
