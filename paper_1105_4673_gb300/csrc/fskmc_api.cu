// Host side of the C ABI declared in include/fskmc.h: contexts, argument
// validation, class-rate tables, processor communication schedules and the
// plain (one launch per window) engine.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "fskmc.h"
#include "fskmc_internal.h"
#include "fskmc_persistent.h"
#include "philox.cuh"

using fskmc::Replica;

struct fskmc_ctx {
    int model = 0, nclass = 0, nstates = 2;
    int nrep = 0;
    int qx = 0, qy = 0;
    bool batch = false;
    std::vector<Replica> reps;
    Replica *d_reps = nullptr;
    uint8_t *d_lat[2] = {nullptr, nullptr};  // [1] only for the ping-pong model
    int cur = 0;                             // which buffer holds the state
    bool packed = false;                     // 1 bit per site in device memory
    uint8_t *d_stage = nullptr;              // byte-per-site staging (packed contexts)
    int64_t total_sites = 0;
    int32_t total_cells = 0;
    int32_t *d_workload = nullptr;
    unsigned long long *d_counters = nullptr;  // events, ambiguous, timeouts, check failures, binary64 edge checks
    unsigned int *d_scratch_u32 = nullptr;
    unsigned long long *d_obs = nullptr;
    int obs_cap = 0;
    uint64_t w = 0;        // global window index
    uint64_t windows = 0;  // windows run
    fskmc_clock clock = FSKMC_CLOCK_FP64;
    fskmc_engine engine = FSKMC_ENGINE_PLAIN;
    int wpb = 2;
    int grouping = 2;      // several small cells per warp: 0 off, 1 on, 2 auto (spin-flip models)
    int edge_screen = 1;   // binary64 clock: screened window-edge decisions
    uint32_t spin_limit = 1u << 20;
    fskmc_task_order order = FSKMC_ORDER_AUTO;
    int nsm = 152;                       // SMs of the context's device
    int32_t *d_order = nullptr;          // issue lists, total_cells entries
    int32_t *d_order_scratch = nullptr;  // bucket histograms and cursors
    cudaStream_t stream = nullptr;
    fskmc::PersistentState *pers = nullptr;
    int nest_qx = 0, nest_qy = 0;        // super-cell shape of the nested scheme (0: off)
    int nest_inner = 0, nest_n = 1;      // inner schedule (LIE / STRANG) and inner steps
    std::string err;
};

namespace {

thread_local std::string g_create_error;

fskmc_status fail(fskmc_ctx *c, fskmc_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf; else g_create_error = buf;
    return st;
}

#define CK(ctx, call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail((ctx), FSKMC_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

bool finite_nonneg(double v) { return std::isfinite(v) && v >= 0.0; }

// Class rates in class order; the same formulas and the same order of
// floating-point operations as the model definitions in include/fskmc.h.
int class_rates(int model, const fskmc_rates &q, double *r)
{
    switch (model) {
    case fskmc::ADSDES:
        for (int n = 0; n < 5; ++n) {
            r[n] = q.ka;
            r[5 + n] = q.kd * std::exp(-(q.betaJ * (double)n));
        }
        return 10;
    case fskmc::ISING:
        for (int n = 0; n < 5; ++n) {
            r[n] = q.ka;
            r[5 + n] = q.kd * std::exp(-(4.0 * q.betaJ) * (double)(n - 2));
        }
        return 10;
    case fskmc::DIFFUSION:
        for (int n = 0; n < 5; ++n) {
            r[n] = q.ka;
            r[5 + n] = q.kd * std::exp(-(q.betaJ * (double)n));
            r[10 + n] = q.nu * std::exp(-(q.betaJ * (double)n));
        }
        return 15;
    case fskmc::ZGB:
        r[0] = q.yA;
        r[1] = (1.0 - q.yA) * 0.25;
        r[2] = q.kr * 0.25;
        r[3] = q.kd;
        return 4;
    case fskmc::ISING1D:
        for (int n = 0; n < 3; ++n) {
            r[n] = q.ka;
            r[3 + n] = q.kd * std::exp(-(q.betaJ * (double)n - q.betah));
        }
        return 6;
    }
    return -1;
}

fskmc_status check_rates(int model, const fskmc_rates &q)
{
    switch (model) {
    case fskmc::ADSDES:
    case fskmc::ISING:
        if (!finite_nonneg(q.ka) || !finite_nonneg(q.kd) || !std::isfinite(q.betaJ))
            return fail(nullptr, FSKMC_EINVAL, "rates: ka, kd must be finite and >= 0, betaJ finite");
        break;
    case fskmc::DIFFUSION:
        if (!finite_nonneg(q.ka) || !finite_nonneg(q.kd) || !finite_nonneg(q.nu) ||
            !std::isfinite(q.betaJ))
            return fail(nullptr, FSKMC_EINVAL, "rates: ka, kd, nu must be finite and >= 0, betaJ finite");
        break;
    case fskmc::ZGB:
        if (!(q.yA >= 0.0 && q.yA <= 1.0) || !finite_nonneg(q.kr) || !finite_nonneg(q.kd))
            return fail(nullptr, FSKMC_EINVAL, "rates: yA must be in [0,1], kr and kd finite and >= 0");
        break;
    case fskmc::ISING1D:
        if (!finite_nonneg(q.ka) || !finite_nonneg(q.kd) || !std::isfinite(q.betaJ) ||
            !std::isfinite(q.betah))
            return fail(nullptr, FSKMC_EINVAL,
                        "rates: ka, kd must be finite and >= 0, betaJ and betah finite");
        break;
    default:
        return fail(nullptr, FSKMC_EINVAL, "unknown model %d", model);
    }
    double r[16];
    int nc = class_rates(model, q, r);
    for (int k = 0; k < nc; ++k)
        if (!std::isfinite(r[k]) || r[k] < 0.0 || (float)r[k] == INFINITY)
            return fail(nullptr, FSKMC_EINVAL, "rate of class %d is not finite (%g)", k, r[k]);
    return FSKMC_OK;
}

fskmc_status check_geometry(int model, const fskmc_lattice &L, int qx, int qy)
{
    if (L.bitpacked != 0 && L.bitpacked != 1) return fail(nullptr, FSKMC_EINVAL, "bitpacked must be 0 or 1");
    if (L.bitpacked && model != fskmc::ADSDES && model != fskmc::ISING && model != fskmc::ISING1D)
        return fail(nullptr, FSKMC_EINVAL, "bit-packed lattices are for the spin-flip models");
    if (L.bitpacked && L.lx % 32)
        return fail(nullptr, FSKMC_EINVAL, "bit-packed lattices need lx to be a multiple of 32");
    if (L.lx > FSKMC_MAX_SIDE || L.ly > FSKMC_MAX_SIDE)
        return fail(nullptr, FSKMC_EINVAL, "lattice side above %d (%d x %d)", FSKMC_MAX_SIDE, L.lx, L.ly);
    if (model == fskmc::ISING1D) {
        // a ring of lx sites: one row of cells qx x 1
        if (L.ly != 1 || qy != 1)
            return fail(nullptr, FSKMC_EINVAL, "ISING1D is a ring: ly and qy must be 1");
        if (qx < 1 || qx > fskmc::MAX_Q_RING)
            return fail(nullptr, FSKMC_EINVAL, "ring cell length %d out of range 1..%d", qx,
                        fskmc::MAX_Q_RING);
        if (L.lx < 2 * qx || L.lx % (2 * qx))
            return fail(nullptr, FSKMC_EINVAL, "ring of %d sites is not a positive multiple of 2*%d",
                        L.lx, qx);
        return FSKMC_OK;
    }
    if (qx < 1 || qy < 1 || qx > fskmc::MAX_Q || qy > fskmc::MAX_Q)
        return fail(nullptr, FSKMC_EINVAL, "cell shape %dx%d out of range 1..32", qx, qy);
    if (L.lx < 2 * qx || L.ly < 2 * qy || L.lx % (2 * qx) || L.ly % (2 * qy))
        return fail(nullptr, FSKMC_EINVAL,
                    "lattice %dx%d is not a positive multiple of twice the cell %dx%d", L.lx,
                    L.ly, qx, qy);
    if ((int64_t)L.lx * L.ly > (int64_t)1 << 31)
        return fail(nullptr, FSKMC_EINVAL, "lattice too large (%d x %d)", L.lx, L.ly);
    if ((model == fskmc::DIFFUSION || model == fskmc::ZGB) && (qx < 2 || qy < 2))
        return fail(nullptr, FSKMC_EINVAL, "two-site models need cells of at least 2x2");
    if (model == fskmc::DIFFUSION && (L.lx < qx + 4 || L.ly < qy + 4))
        return fail(nullptr, FSKMC_EINVAL,
                    "diffusion needs lx >= qx+4 and ly >= qy+4 (two-site frozen halo)");
    return FSKMC_OK;
}

int64_t nsteps(double dt, double T)
{
    if (!(dt > 0.0) || !(T >= 0.0) || !std::isfinite(dt) || !std::isfinite(T)) return -1;
    double n = std::floor(T / dt + 0.5);
    if (std::fabs(n * dt - T) > 1e-9 * T) return -1;
    if (n > 1e9) return -1;
    return (int64_t)n;
}

struct Win {
    int colour;
    double h;
};

// Windows of a run starting at global window index w0 (Section 3): LIE
// E(dt) O(dt); STRANG E(dt/2) O(dt) E(dt/2); RANDOM 2 windows of dt per step,
// colour = bit 0 of word 0 of Philox(seed, (0, w, 0, rep | 3<<24)), 0 = E;
// RANDOM_ORDER per step (c, 1-c) with c drawn the same way at the step's
// first window index.
void build_schedule(int scheme, int64_t n, double dt, uint64_t seed, uint32_t rep, uint64_t w0,
                    std::vector<Win> &out)
{
    out.clear();
    const uint32_t c3 = rep | (fskmc::TAG_SCHED << 24);
    for (int64_t i = 0; i < n; ++i) {
        uint32_t w = (uint32_t)(w0 + out.size());
        switch (scheme) {
        case FSKMC_LIE:
            out.push_back({0, dt});
            out.push_back({1, dt});
            break;
        case FSKMC_STRANG:
            out.push_back({0, dt * 0.5});
            out.push_back({1, dt});
            out.push_back({0, dt * 0.5});
            break;
        case FSKMC_RANDOM:
            out.push_back({(int)(fskmc::draw(seed, 0, w, 0, c3).x & 1u), dt});
            out.push_back({(int)(fskmc::draw(seed, 0, w + 1, 0, c3).x & 1u), dt});
            break;
        case FSKMC_RANDOM_ORDER: {
            int c = (int)(fskmc::draw(seed, 0, w, 0, c3).x & 1u);
            out.push_back({c, dt});
            out.push_back({1 - c, dt});
            break;
        }
        }
    }
}

// Fixed-point rates of the binary32-clock path: R_k = round(r_k 2^qshift)
// with the largest qshift that keeps every cell's total rate below 2^62
// (members per cell times the largest rate), so all rate-class sums are
// exact 64-bit integers.
void set_fixed_point(Replica &R, int nclass, int members)
{
    double rmax = 0.0;
    for (int k = 0; k < nclass; ++k) rmax = std::max(rmax, R.r[k]);
    int shift = 40;
    if (rmax > 0.0) {
        int ex = 0;
        std::frexp((double)members * rmax, &ex);  // members * rmax < 2^ex
        shift = 62 - ex;
    }
    shift = std::min(100, std::max(-100, shift));
    R.qshift = shift;
    R.qscale = std::ldexp(1.0f, -shift);
    for (int k = 0; k < fskmc::MAX_CLASSES; ++k)
        R.rq[k] = k < nclass ? (uint64_t)std::nearbyint(std::ldexp(R.r[k], shift)) : 0ull;
}

fskmc_status make_ctx(int n, const fskmc_lattice *lats, fskmc_model model,
                      const fskmc_rates *rates, fskmc_cell_shape cell, void *stream, bool batch,
                      fskmc_ctx **out)
{
    if (!out || !lats || !rates) return fail(nullptr, FSKMC_EINVAL, "NULL argument");
    *out = nullptr;
    if ((int)model < 0 || (int)model > 4) return fail(nullptr, FSKMC_EINVAL, "unknown model %d", (int)model);
    if (n < 1 || n > 65536) return fail(nullptr, FSKMC_EINVAL, "replica count %d out of range", n);
    int qx = cell.qx, qy = cell.qy;
    if (qx == 0 && qy == 0 && (int)model == fskmc::ISING1D) {
        // Ring: the longest cell in {1024, ..., 32} that every ring admits
        // and that leaves at least 152 active cells in total, else the
        // longest admissible one.
        int best = 0;
        for (int q = fskmc::MAX_Q_RING; q >= 32; q >>= 1) {
            bool ok = true;
            int64_t cells = 0;
            for (int r = 0; r < n && ok; ++r) {
                ok = lats[r].ly == 1 && lats[r].lx >= 2 * q && lats[r].lx % (2 * q) == 0;
                cells += ok ? lats[r].lx / q / 2 : 0;
            }
            if (!ok) continue;
            if (!best) best = q;
            if (cells >= 152) { best = q; break; }
        }
        if (!best) return fail(nullptr, FSKMC_EINVAL, "no ring cell length in {32..1024} fits every ring");
        qx = best;
        qy = 1;
    } else if (qx == 0 && qy == 0) {
        // Autotuner: the largest square cell in {32, 16, 8} that every
        // replica admits and that leaves at least 152 active cells in total
        // (one per SM); falling back to the largest admissible one.
        int best = 0;
        for (int q : {32, 16, 8}) {
            bool ok = true;
            int64_t cells = 0;
            for (int r = 0; r < n && ok; ++r) {
                ok = check_geometry(model, lats[r], q, q) == FSKMC_OK;
                cells += ok ? (int64_t)(lats[r].lx / q) * (lats[r].ly / q) / 2 : 0;
            }
            if (!ok) continue;
            if (!best) best = q;
            if (cells >= 152) { best = q; break; }
        }
        if (!best) return fail(nullptr, FSKMC_EINVAL, "no cell size in {8,16,32} fits every lattice");
        qx = qy = best;
    }
    for (int r = 0; r < n; ++r) {
        if (lats[r].bitpacked != lats[0].bitpacked)
            return fail(nullptr, FSKMC_EINVAL, "all replicas must share the bit-packed setting");
        fskmc_status st = check_geometry(model, lats[r], qx, qy);
        if (st) return st;
        st = check_rates(model, rates[r]);
        if (st) return st;
    }
    fskmc_ctx *c = new fskmc_ctx();
    c->model = model;
    c->nstates = (int)model == fskmc::ZGB ? 3 : 2;
    c->nrep = n;
    c->qx = qx;
    c->qy = qy;
    c->batch = batch;
    c->packed = lats[0].bitpacked != 0;
    c->stream = (cudaStream_t)stream;
    {
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0)
            c->nsm = nsm;
    }
    c->reps.resize(n);
    int64_t off = 0;
    int32_t coff = 0;
    for (int r = 0; r < n; ++r) {
        Replica &R = c->reps[r];
        std::memset(&R, 0, sizeof R);
        R.lx = lats[r].lx;
        R.ly = lats[r].ly;
        R.ncx = R.lx / qx;
        R.ncy = R.ly / qy;
        R.lat_off = off;
        R.cell_off = coff;
        R.rep = (uint32_t)r;
        c->nclass = class_rates(model, rates[r], R.r);
        const bool two_site = (int)model == fskmc::DIFFUSION || (int)model == fskmc::ZGB;
        set_fixed_point(R, c->nclass, qx * qy * (two_site ? 9 : 1));
        const int64_t bytes = c->packed ? (int64_t)(R.lx / 32) * R.ly * 4 : (int64_t)R.lx * R.ly;
        off += (bytes + 255) & ~(int64_t)255;
        coff += R.ncx * R.ncy;
    }
    int64_t max_sites = 0;
    for (const Replica &R : c->reps) max_sites = std::max(max_sites, (int64_t)R.lx * R.ly);
    c->total_sites = off;
    c->total_cells = coff;
    cudaError_t e;
    e = cudaMalloc(&c->d_lat[0], (size_t)off);
    if (e == cudaSuccess && (int)model == fskmc::DIFFUSION) e = cudaMalloc(&c->d_lat[1], (size_t)off);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_reps, sizeof(Replica) * n);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_workload, sizeof(int32_t) * (size_t)coff);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_counters, sizeof(unsigned long long) * 5);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_scratch_u32, sizeof(unsigned int) * 4);
    if (e == cudaSuccess && c->packed) e = cudaMalloc(&c->d_stage, (size_t)max_sites);
    if (e != cudaSuccess) {
        fskmc_destroy(c);
        return fail(nullptr, e == cudaErrorMemoryAllocation ? FSKMC_ENOMEM : FSKMC_ECUDA,
                    "device allocation failed: %s", cudaGetErrorString(e));
    }
    e = cudaMemsetAsync(c->d_lat[0], 0, (size_t)off, c->stream);
    if (e == cudaSuccess && c->d_lat[1]) e = cudaMemsetAsync(c->d_lat[1], 0, (size_t)off, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_workload, 0, sizeof(int32_t) * (size_t)coff, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_counters, 0, sizeof(unsigned long long) * 5, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_reps, c->reps.data(), sizeof(Replica) * n, cudaMemcpyHostToDevice,
                            c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        fskmc_destroy(c);
        return fail(nullptr, FSKMC_ECUDA, "context setup failed: %s", cudaGetErrorString(e));
    }
    *out = c;
    g_create_error.clear();
    return FSKMC_OK;
}

fskmc_status upload_reps(fskmc_ctx *c)
{
    CK(c, cudaMemcpyAsync(c->d_reps, c->reps.data(), sizeof(Replica) * c->nrep,
                          cudaMemcpyHostToDevice, c->stream));
    return FSKMC_OK;
}

// One window of every replica on the plain engine.
// Replicas per call of the ordering kernels (bounds their scratch).
constexpr int ORDER_GROUP = 1024;

// Heaviest-first issue lists for windows with `active` active cells: always
// (WORKLOAD), never (NATURAL), or (AUTO) in the plain engine when a window's
// cells fill the GPU in one wave (8 to 16 per SM): then the block
// scheduler's round-robin over SMs spreads the heavy cells evenly. With
// several waves of cells the scheduler balances by itself and row-major
// order keeps neighbouring halos in cache; with few cells the windows are
// too short to pay for the ordering launch; the persistent engine's queue
// overlaps windows.
// Lanes per cell of the window kernels for this context: grouped cells
// wherever the model and cell size allow, unless grouping is switched off
// (AUTO and ON agree: the grouped kernels were faster in every engine and
// clock on the spin-flip workloads).
int lanes_per_cell(const fskmc_ctx *c)
{
    if (c->grouping == 0) return 32;
    // ZGB, 32-wide cells, binary32 clock: eight cells per warp (4 lanes
    // each, rows a multiple of 8 from 16; persistent engine) or four (8
    // lanes, a multiple of 4 from 8; fskmc_zgbquad.cu), else two (16 lanes,
    // an even number of rows; fskmc_zgbpair.cu)
    if (c->model == FSKMC_ZGB) {
        if (c->clock != FSKMC_CLOCK_FP32) return 32;
        // eight cells per warp, 4 lanes each (rows a multiple of 8 from 16),
        // else four, 8 lanes each (a multiple of 4 from 8), else two
        if (fskmc::zgb_multi_shape(8, c->qx, c->qy)) return 4;
        if (fskmc::zgb_multi_shape(4, c->qx, c->qy)) return 8;
        return fskmc::zgb_pair_shape(c->qx, c->qy) ? 16 : 32;
    }
    const int W = fskmc::group_width(c->model, c->qx, c->qy);
    return W >= 32 ? 32 : W;
}

bool use_order(const fskmc_ctx *c, int64_t active, bool persistent)
{
    if (c->order == FSKMC_ORDER_WORKLOAD) return true;
    if (c->order == FSKMC_ORDER_NATURAL) return false;
    return !persistent && active >= (int64_t)c->nsm * 8 && active <= (int64_t)c->nsm * 16;
}

fskmc_status ensure_order_buffers(fskmc_ctx *c)
{
    if (c->d_order) return FSKMC_OK;
    const size_t scratch = (size_t)std::min(c->nrep, ORDER_GROUP) * 2 * fskmc::ORDER_BUCKETS * 2;
    CK(c, cudaMalloc(&c->d_order, sizeof(int32_t) * (size_t)c->total_cells));
    CK(c, cudaMalloc(&c->d_order_scratch, sizeof(int32_t) * scratch));
    return FSKMC_OK;
}

// Issue lists of replicas [r0, r0 + n) for colours c0..c1.
fskmc_status build_order(fskmc_ctx *c, int r0, int n, int c0, int c1)
{
    fskmc_status st = ensure_order_buffers(c);
    if (st) return st;
    const size_t half = (size_t)std::min(c->nrep, ORDER_GROUP) * 2 * fskmc::ORDER_BUCKETS;
    for (int g = r0; g < r0 + n; g += ORDER_GROUP) {
        const int ng = std::min(ORDER_GROUP, r0 + n - g);
        CK(c, fskmc::launch_order(c->reps.data(), c->d_reps, g, ng, c0, c1, c->qx, c->qy,
                                  c->d_workload, c->d_order, c->d_order_scratch,
                                  c->d_order_scratch + half, c->stream));
    }
    return FSKMC_OK;
}

fskmc_status plain_window(fskmc_ctx *c, const std::vector<std::vector<Win>> &sched, size_t i,
                          uint64_t w, uint64_t seed, bool ordered, int lanes)
{
    const int fp32 = c->clock == FSKMC_CLOCK_FP32;
    const bool pingpong = c->d_lat[1] != nullptr;
    for (int r = 0; r < c->nrep; ++r) {
        const Win &win = sched[sched.size() == 1 ? 0 : r][i];
        fskmc::WindowArgs a;
        a.reps = c->d_reps;
        a.rep_index = r;
        a.geom = fskmc::make_geom(c->qx, c->qy);
        a.colour = win.colour;
        a.w = (uint32_t)w;
        a.h = win.h;
        a.seed = seed;
        a.src = c->d_lat[c->cur];
        a.dst = pingpong ? c->d_lat[1 - c->cur] : c->d_lat[c->cur];
        a.workload = c->d_workload;
        a.counters = c->d_counters;
        a.packed = c->packed ? 1 : 0;
        a.order = nullptr;
        a.lanes_per_cell = lanes;
        a.screen = c->edge_screen;
        const Replica &R = c->reps[r];
        int nactive = R.ncx * R.ncy / 2;
        if (ordered) a.order = c->d_order + R.cell_off + (size_t)win.colour * nactive;
        CK(c, fskmc::launch_window(c->model, fp32, a, nactive, c->wpb, c->stream));
    }
    if (pingpong) c->cur ^= 1;
    return FSKMC_OK;
}

// Run a schedule (one window list, or one per replica) on the context's
// engine, starting at window index c->w.
fskmc_status exec_windows(fskmc_ctx *c, const std::vector<std::vector<Win>> &sched, uint64_t seed)
{
    const size_t nw = sched[0].size();
    if (c->engine == FSKMC_ENGINE_PERSISTENT) {
        std::vector<int8_t> col(sched.size() * nw);
        std::vector<double> hh(nw);
        for (size_t r = 0; r < sched.size(); ++r)
            for (size_t i = 0; i < nw; ++i) col[r * nw + i] = (int8_t)sched[r][i].colour;
        for (size_t i = 0; i < nw; ++i) hh[i] = sched[0][i].h;
        fskmc::PersistentRun pr;
        pr.model = c->model;
        pr.fp32 = c->clock == FSKMC_CLOCK_FP32;
        pr.qx = c->qx;
        pr.qy = c->qy;
        pr.nrep = c->nrep;
        pr.reps_host = c->reps.data();
        pr.reps_dev = c->d_reps;
        pr.lat = c->d_lat[c->cur];
        pr.lat2 = c->d_lat[1] ? c->d_lat[1 - c->cur] : nullptr;
        pr.workload = c->d_workload;
        pr.counters = c->d_counters;
        pr.total_cells = c->total_cells;
        pr.colour = col.data();
        pr.colour_per_replica = sched.size() > 1;
        pr.h = hh.data();
        pr.nwin = (int64_t)nw;
        pr.w0 = c->w;
        pr.seed = seed;
        pr.wpb = std::min(c->wpb, 8);  // the persistent kernel is built for <= 256 threads
        pr.spin_limit = c->spin_limit;
        pr.packed = c->packed;
        pr.lanes_per_cell = lanes_per_cell(c);
        pr.screen = c->edge_screen != 0;
        pr.order = nullptr;
        if (use_order(c, c->total_cells / 2, true)) {
            fskmc_status st = build_order(c, 0, c->nrep, 0, 1);
            if (st) return st;
            pr.order = c->d_order;
        }
        std::string msg;
        cudaError_t e = fskmc::persistent_run(&c->pers, pr, c->stream, &msg);
        if (e == cudaErrorTimeout) {
            c->w += nw;
            c->windows += nw;
            return fail(c, FSKMC_ETIMEOUT, "persistent run: %s; the lattice is undefined", msg.c_str());
        }
        if (e != cudaSuccess) return fail(c, FSKMC_ECUDA, "persistent run: %s (%s)", cudaGetErrorString(e), msg.c_str());
        if (c->d_lat[1] && (nw & 1)) c->cur ^= 1;
    } else {
        // issue lists from the workloads at the start of the run
        int64_t most = 0;
        for (const Replica &R : c->reps) most = std::max<int64_t>(most, R.ncx * R.ncy / 2);
        const bool ordered = use_order(c, most, false);
        if (ordered) {
            fskmc_status st = build_order(c, 0, c->nrep, 0, 1);
            if (st) return st;
        }
        const int lanes = lanes_per_cell(c);
        for (size_t i = 0; i < nw; ++i) {
            fskmc_status st = plain_window(c, sched, i, c->w + i, seed, ordered, lanes);
            if (st) return st;
        }
    }
    return FSKMC_OK;
}

// Warps per block of the nested kernel: one per active sub-cell of a
// super-cell's inner window, at most 16, fewer if shared memory runs out.
int nested_wpb(const fskmc_ctx *c, int lanes)
{
    const int nact = (c->nest_qx / c->qx) * (c->nest_qy / c->qy) / 2;
    const int per_warp = lanes < 32 ? 32 / lanes : 1;
    int wpb = std::min((nact + per_warp - 1) / per_warp, 16);
    while (wpb > 1 && fskmc::nested_smem(c->model, c->nest_qx, c->nest_qy, c->qx, c->qy, wpb, lanes) > 227 * 1024)
        --wpb;
    return wpb;
}

// The nested scheme (fskmc_set_nesting): every outer window of the
// schedule runs the inner schedule inside each super-cell of its colour,
// one launch per outer window and replica.
fskmc_status nested_windows(fskmc_ctx *c, const std::vector<std::vector<Win>> &sched, uint64_t seed)
{
    const size_t nw = sched[0].size();
    const uint64_t ninner = (uint64_t)(c->nest_inner == FSKMC_LIE ? 2 : 3) * (uint64_t)c->nest_n;
    if ((c->w + nw) * ninner > 0xFFFFFFFFull)
        return fail(c, FSKMC_EINVAL, "nested run: inner window index beyond 2^32");
    const int lanes = lanes_per_cell(c);
    const int wpb = nested_wpb(c, lanes);
    const int super_bytes = ((c->nest_qx + 2) * (c->nest_qy + 2) + 15) & ~15;
    for (size_t i = 0; i < nw; ++i) {
        for (int r = 0; r < c->nrep; ++r) {
            const Win &win = sched[sched.size() == 1 ? 0 : r][i];
            const Replica &R = c->reps[r];
            fskmc::NestedArgs a;
            a.reps = c->d_reps;
            a.rep_index = r;
            a.geom = fskmc::make_geom(c->qx, c->qy);
            a.Qx = c->nest_qx;
            a.Qy = c->nest_qy;
            a.colour = win.colour;
            a.w0 = (uint32_t)((c->w + i) * ninner);
            a.inner = c->nest_inner == FSKMC_LIE ? 0 : 1;
            a.ninner = (int32_t)ninner;
            a.d = win.h / (double)c->nest_n;
            a.dhalf = a.d * 0.5;
            a.seed = seed;
            a.lat = c->d_lat[c->cur];
            a.workload = c->d_workload;
            a.counters = c->d_counters;
            a.packed = c->packed ? 1 : 0;
            a.screen = c->edge_screen;
            a.super_bytes = super_bytes;
            a.lanes = lanes;
            const int nsuper = (R.lx / c->nest_qx) * (R.ly / c->nest_qy) / 2;
            CK(c, fskmc::launch_nested(c->model, c->clock == FSKMC_CLOCK_FP32, a, nsuper, wpb, c->stream));
        }
    }
    return FSKMC_OK;
}

// Byte-per-site view of a replica's lattice for the init/copy kernels: the
// replica's own storage, or the staging buffer of a packed context.
uint8_t *byte_view(fskmc_ctx *c, int r)
{
    return c->packed ? c->d_stage : c->d_lat[c->cur] + c->reps[r].lat_off;
}

// Packed contexts: pack the staging buffer into replica r's words.
cudaError_t commit_view(fskmc_ctx *c, int r)
{
    if (!c->packed) return cudaSuccess;
    const Replica &R = c->reps[r];
    return fskmc::launch_pack(c->d_stage, reinterpret_cast<uint32_t *>(c->d_lat[c->cur] + R.lat_off),
                              R.lx, R.ly, c->stream);
}

}  // namespace

extern "C" {

fskmc_status fskmc_create(const fskmc_lattice *lattice, fskmc_model model,
                          const fskmc_rates *rates, fskmc_cell_shape cell, void *stream,
                          fskmc_ctx **out)
{
    return make_ctx(1, lattice, model, rates, cell, stream, false, out);
}

fskmc_status fskmc_batch_create(int32_t n, const fskmc_lattice *lattices, fskmc_model model,
                                const fskmc_rates *rates, fskmc_cell_shape cell, void *stream,
                                fskmc_ctx **out)
{
    return make_ctx(n, lattices, model, rates, cell, stream, true, out);
}

void fskmc_destroy(fskmc_ctx *c)
{
    if (!c) return;
    if (c->stream || c->d_lat[0]) cudaStreamSynchronize(c->stream);
    fskmc::persistent_free(c->pers);
    cudaFree(c->d_lat[0]);
    cudaFree(c->d_lat[1]);
    cudaFree(c->d_reps);
    cudaFree(c->d_workload);
    cudaFree(c->d_counters);
    cudaFree(c->d_scratch_u32);
    cudaFree(c->d_stage);
    cudaFree(c->d_obs);
    cudaFree(c->d_order);
    cudaFree(c->d_order_scratch);
    delete c;
}

const char *fskmc_last_error(const fskmc_ctx *c)
{
    return c ? c->err.c_str() : g_create_error.c_str();
}

fskmc_status fskmc_set_replica_id(fskmc_ctx *c, uint32_t id)
{
    if (!c) return FSKMC_EINVAL;
    if (c->batch) return fail(c, FSKMC_EINVAL, "replica ids of a batch are fixed");
    if (id >= (1u << 24)) return fail(c, FSKMC_EINVAL, "replica id must be < 2^24");
    c->reps[0].rep = id;
    return upload_reps(c);
}

fskmc_status fskmc_set_clock(fskmc_ctx *c, fskmc_clock clock)
{
    if (!c) return FSKMC_EINVAL;
    if (clock != FSKMC_CLOCK_FP64 && clock != FSKMC_CLOCK_FP32)
        return fail(c, FSKMC_EINVAL, "unknown clock %d", (int)clock);
    c->clock = clock;
    return FSKMC_OK;
}

fskmc_status fskmc_set_engine(fskmc_ctx *c, fskmc_engine engine)
{
    if (!c) return FSKMC_EINVAL;
    if (engine != FSKMC_ENGINE_PLAIN && engine != FSKMC_ENGINE_PERSISTENT)
        return fail(c, FSKMC_EINVAL, "unknown engine %d", (int)engine);
    c->engine = engine;
    return FSKMC_OK;
}

fskmc_status fskmc_set_warps_per_block(fskmc_ctx *c, int32_t warps)
{
    if (!c) return FSKMC_EINVAL;
    if (warps < 1 || warps > 16) return fail(c, FSKMC_EINVAL, "warps per block must be 1..16");
    size_t need = std::max({fskmc::window_smem_per_warp(c->model, c->qx, c->qy),
                            fskmc::group_smem_per_warp(c->model, c->qx, c->qy),
                            c->model == FSKMC_ZGB ? std::max(fskmc::zgb_pair_smem_per_warp(c->qy),
                                                             fskmc::zgb_multi_smem_per_warp(8))
                                                  : (size_t)0}) *
                  (size_t)warps;
    if (need > 200 * 1024) return fail(c, FSKMC_EINVAL, "%d warps need %zu B of shared memory", warps, need);
    c->wpb = warps;
    return FSKMC_OK;
}

fskmc_status fskmc_set_cell_grouping(fskmc_ctx *c, int32_t on)
{
    if (!c) return FSKMC_EINVAL;
    if (on < 0 || on > 2) return fail(c, FSKMC_EINVAL, "cell grouping must be 0 (off), 1 (on) or 2 (auto)");
    c->grouping = on;
    return FSKMC_OK;
}

fskmc_status fskmc_set_edge_screen(fskmc_ctx *c, int32_t on)
{
    if (!c) return FSKMC_EINVAL;
    if (on != 0 && on != 1) return fail(c, FSKMC_EINVAL, "edge screen must be 0 (off) or 1 (on)");
    c->edge_screen = on;
    return FSKMC_OK;
}

fskmc_status fskmc_set_nesting(fskmc_ctx *c, fskmc_cell_shape sup, fskmc_scheme inner, int32_t n_inner)
{
    if (!c) return FSKMC_EINVAL;
    if (sup.qx == 0 && sup.qy == 0) {
        c->nest_qx = c->nest_qy = 0;
        return FSKMC_OK;
    }
    if (c->model != fskmc::ADSDES && c->model != fskmc::ISING)
        return fail(c, FSKMC_EINVAL, "nesting is built for the 2D spin-flip models (ADSDES, ISING_ARRHENIUS)");
    if (inner != FSKMC_LIE && inner != FSKMC_STRANG)
        return fail(c, FSKMC_EINVAL, "inner schedule must be LIE or STRANG");
    if (n_inner < 1) return fail(c, FSKMC_EINVAL, "n_inner must be >= 1");
    if (sup.qx < 2 * c->qx || sup.qy < 2 * c->qy || sup.qx % (2 * c->qx) || sup.qy % (2 * c->qy))
        return fail(c, FSKMC_EINVAL, "super-cell %dx%d is not a multiple of twice the cell %dx%d", sup.qx,
                    sup.qy, c->qx, c->qy);
    for (const Replica &R : c->reps)
        if (R.lx % (2 * sup.qx) || R.ly % (2 * sup.qy))
            return fail(c, FSKMC_EINVAL, "lattice %dx%d is not a multiple of twice the super-cell %dx%d",
                        R.lx, R.ly, sup.qx, sup.qy);
    if (c->packed && sup.qx % 32)
        return fail(c, FSKMC_EINVAL, "bit-packed lattices need super-cells a multiple of 32 wide");
    if (fskmc::nested_smem(c->model, sup.qx, sup.qy, c->qx, c->qy, 1, 32) > 227 * 1024 ||
        fskmc::nested_smem(c->model, sup.qx, sup.qy, c->qx, c->qy, 1, fskmc::group_width(c->model, c->qx, c->qy)) > 227 * 1024)
        return fail(c, FSKMC_EINVAL, "super-cell %dx%d does not fit one block's shared memory", sup.qx, sup.qy);
    c->nest_qx = sup.qx;
    c->nest_qy = sup.qy;
    c->nest_inner = (int)inner;
    c->nest_n = n_inner;
    return FSKMC_OK;
}

fskmc_status fskmc_set_task_order(fskmc_ctx *c, fskmc_task_order order)
{
    if (!c) return FSKMC_EINVAL;
    if ((int)order < 0 || (int)order > 2) return fail(c, FSKMC_EINVAL, "unknown task order %d", (int)order);
    c->order = order;
    return FSKMC_OK;
}

fskmc_status fskmc_set_spin_limit(fskmc_ctx *c, uint32_t polls)
{
    if (!c) return FSKMC_EINVAL;
    c->spin_limit = polls;
    return FSKMC_OK;
}

fskmc_status fskmc_info(const fskmc_ctx *c, int32_t out[6])
{
    if (!c || !out) return FSKMC_EINVAL;
    out[0] = c->qx;
    out[1] = c->qy;
    out[2] = c->nrep;
    out[3] = c->total_cells;
    out[4] = c->wpb;
    out[5] = lanes_per_cell(c);
    return FSKMC_OK;
}

fskmc_status fskmc_init_random(fskmc_ctx *c, uint64_t seed, double coverage)
{
    if (!c) return FSKMC_EINVAL;
    if (!(coverage >= 0.0 && coverage <= 1.0)) return fail(c, FSKMC_EINVAL, "coverage must be in [0,1]");
    for (int r = 0; r < c->nrep; ++r) {
        const Replica &R = c->reps[r];
        CK(c, fskmc::launch_init_bernoulli(byte_view(c, r), R.lx, R.ly, seed, coverage, R.rep,
                                           c->stream));
        CK(c, commit_view(c, r));
    }
    return FSKMC_OK;
}

fskmc_status fskmc_init_bump(fskmc_ctx *c, uint64_t seed, double amp, double width, int32_t species)
{
    if (!c) return FSKMC_EINVAL;
    if (!(amp >= 0.0 && amp <= 1.0) || !(width > 0.0) || !std::isfinite(width))
        return fail(c, FSKMC_EINVAL, "amp must be in [0,1] and width > 0");
    if (species < 0 || species >= c->nstates) return fail(c, FSKMC_EINVAL, "species %d not a state", species);
    for (int r = 0; r < c->nrep; ++r) {
        const Replica &R = c->reps[r];
        fskmc::u32x4 cc = fskmc::draw(seed, 0, 0xFFFFFFFFu, 0, R.rep | (fskmc::TAG_SCHED << 24));
        int x0 = (int)(cc.x % (uint32_t)R.lx), y0 = (int)(cc.y % (uint32_t)R.ly);
        std::vector<double> g(R.lx + R.ly);
        double two_s2 = 2.0 * width * width;
        for (int x = 0; x < R.lx; ++x) {
            int d = std::abs(x - x0);
            if (R.lx - d < d) d = R.lx - d;
            g[x] = std::exp(-((double)d * (double)d) / two_s2);
        }
        for (int y = 0; y < R.ly; ++y) {
            int d = std::abs(y - y0);
            if (R.ly - d < d) d = R.ly - d;
            g[R.lx + y] = std::exp(-((double)d * (double)d) / two_s2);
        }
        double *dg = nullptr;
        CK(c, cudaMallocAsync(&dg, sizeof(double) * g.size(), c->stream));
        CK(c, cudaMemcpyAsync(dg, g.data(), sizeof(double) * g.size(), cudaMemcpyHostToDevice, c->stream));
        CK(c, fskmc::launch_init_bump(byte_view(c, r), R.lx, R.ly, seed, dg, dg + R.lx, amp, species,
                                      R.rep, c->stream));
        CK(c, commit_view(c, r));
        CK(c, cudaFreeAsync(dg, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    return FSKMC_OK;
}

fskmc_status fskmc_set_state(fskmc_ctx *c, int32_t replica, const uint8_t *src, int32_t is_device)
{
    if (!c) return FSKMC_EINVAL;
    if (replica < 0 || replica >= c->nrep || !src) return fail(c, FSKMC_EINVAL, "bad replica or NULL src");
    const Replica &R = c->reps[replica];
    size_t n = (size_t)R.lx * R.ly;
    uint8_t *dst = byte_view(c, replica);
    CK(c, cudaMemcpyAsync(dst, src, n, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          c->stream));
    CK(c, cudaMemsetAsync(c->d_scratch_u32, 0, sizeof(unsigned int), c->stream));
    CK(c, fskmc::launch_validate(dst, (int64_t)n, c->nstates, c->d_scratch_u32, c->stream));
    unsigned int bad = 0;
    CK(c, cudaMemcpyAsync(&bad, c->d_scratch_u32, sizeof bad, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (bad) {
        CK(c, cudaMemsetAsync(dst, 0, n, c->stream));
        CK(c, commit_view(c, replica));
        return fail(c, FSKMC_EINVAL, "%u sites hold a value that is not a state of the model", bad);
    }
    CK(c, commit_view(c, replica));
    return FSKMC_OK;
}

fskmc_status fskmc_get_state(fskmc_ctx *c, int32_t replica, uint8_t *dst, int32_t is_device)
{
    if (!c) return FSKMC_EINVAL;
    if (replica < 0 || replica >= c->nrep || !dst) return fail(c, FSKMC_EINVAL, "bad replica or NULL dst");
    const Replica &R = c->reps[replica];
    size_t n = (size_t)R.lx * R.ly;
    if (c->packed)
        CK(c, fskmc::launch_unpack(reinterpret_cast<const uint32_t *>(c->d_lat[c->cur] + R.lat_off),
                                   c->d_stage, R.lx, R.ly, c->stream));
    CK(c, cudaMemcpyAsync(dst, c->packed ? c->d_stage : c->d_lat[c->cur] + R.lat_off, n,
                          is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (!is_device) CK(c, cudaStreamSynchronize(c->stream));
    return FSKMC_OK;
}

fskmc_status fskmc_state_layout(const fskmc_ctx *c, int64_t *out)
{
    if (!c || !out) return FSKMC_EINVAL;
    for (int r = 0; r < c->nrep; ++r) out[r] = c->reps[r].lat_off;
    out[c->nrep] = c->total_sites;
    return FSKMC_OK;
}

fskmc_status fskmc_set_state_all(fskmc_ctx *c, const uint8_t *src, int32_t is_device)
{
    if (!c) return FSKMC_EINVAL;
    if (!src) return fail(c, FSKMC_EINVAL, "NULL src");
    if (c->packed) return fail(c, FSKMC_EINVAL, "a bit-packed context takes its states one replica at a time");
    // the byte lattices are laid out as the state buffer: one copy, one check
    uint8_t *dst = c->d_lat[c->cur];
    const int64_t n = c->total_sites;
    CK(c, cudaMemcpyAsync(dst, src, (size_t)n, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          c->stream));
    CK(c, cudaMemsetAsync(c->d_scratch_u32, 0, sizeof(unsigned int), c->stream));
    CK(c, fskmc::launch_validate(dst, n, c->nstates, c->d_scratch_u32, c->stream));
    unsigned int bad = 0;
    CK(c, cudaMemcpyAsync(&bad, c->d_scratch_u32, sizeof bad, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (bad) {
        CK(c, cudaMemsetAsync(dst, 0, (size_t)n, c->stream));
        return fail(c, FSKMC_EINVAL, "%u bytes hold a value that is not a state of the model", bad);
    }
    return FSKMC_OK;
}

fskmc_status fskmc_get_state_all(fskmc_ctx *c, uint8_t *dst, int32_t is_device)
{
    if (!c) return FSKMC_EINVAL;
    if (!dst) return fail(c, FSKMC_EINVAL, "NULL dst");
    if (c->packed) return fail(c, FSKMC_EINVAL, "a bit-packed context gives its states one replica at a time");
    CK(c, cudaMemcpyAsync(dst, c->d_lat[c->cur], (size_t)c->total_sites,
                          is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (!is_device) CK(c, cudaStreamSynchronize(c->stream));
    return FSKMC_OK;
}

fskmc_status fskmc_run(fskmc_ctx *c, fskmc_scheme scheme, double dt, double T, uint64_t seed)
{
    if (!c) return FSKMC_EINVAL;
    if ((int)scheme < 0 || (int)scheme > 3) return fail(c, FSKMC_EINVAL, "unknown scheme %d", (int)scheme);
    int64_t n = nsteps(dt, T);
    if (n < 0) return fail(c, FSKMC_EINVAL, "dt must be > 0, T >= 0 and T/dt an integer (dt=%g T=%g)", dt, T);
    const bool per_replica = (scheme == FSKMC_RANDOM || scheme == FSKMC_RANDOM_ORDER) && c->nrep > 1;
    std::vector<std::vector<Win>> sched(per_replica ? c->nrep : 1);
    for (size_t r = 0; r < sched.size(); ++r)
        build_schedule(scheme, n, dt, seed, c->reps[r].rep, c->w, sched[r]);
    fskmc_status st = c->nest_qx ? nested_windows(c, sched, seed) : exec_windows(c, sched, seed);
    if (st) return st;
    c->w += sched[0].size();
    c->windows += sched[0].size() * (c->nest_qx ? (uint64_t)(c->nest_inner == FSKMC_LIE ? 2 : 3) * c->nest_n : 1);
    return FSKMC_OK;
}

fskmc_status fskmc_window(fskmc_ctx *c, int32_t colour, double h, uint64_t seed)
{
    if (!c) return FSKMC_EINVAL;
    if (colour != 0 && colour != 1) return fail(c, FSKMC_EINVAL, "colour must be 0 or 1");
    if (!(h > 0.0) || !std::isfinite(h)) return fail(c, FSKMC_EINVAL, "window length must be > 0");
    std::vector<std::vector<Win>> sched(1, std::vector<Win>{{colour, h}});
    fskmc_status st = c->nest_qx ? nested_windows(c, sched, seed) : exec_windows(c, sched, seed);
    if (st) return st;
    c->w += 1;
    c->windows += c->nest_qx ? (uint64_t)(c->nest_inner == FSKMC_LIE ? 2 : 3) * c->nest_n : 1;
    return FSKMC_OK;
}

fskmc_status fskmc_get_window_index(const fskmc_ctx *c, uint64_t *w)
{
    if (!c || !w) return FSKMC_EINVAL;
    *w = c->w;
    return FSKMC_OK;
}

fskmc_status fskmc_set_window_index(fskmc_ctx *c, uint64_t w)
{
    if (!c) return FSKMC_EINVAL;
    if (w >= (1ull << 32)) return fail(c, FSKMC_EINVAL, "window index must be < 2^32");
    c->w = w;
    return FSKMC_OK;
}

fskmc_status fskmc_observables(fskmc_ctx *c, int32_t replica, double *coverage, double *energy,
                               double *paircorr, int32_t rmax)
{
    if (!c) return FSKMC_EINVAL;
    if (replica < 0 || replica >= c->nrep) return fail(c, FSKMC_EINVAL, "bad replica %d", replica);
    const Replica &R = c->reps[replica];
    if (!coverage || !energy || rmax < 0 || rmax > R.lx || (R.ly > 1 && rmax > R.ly) ||
        (rmax > 0 && !paircorr))
        return fail(c, FSKMC_EINVAL, "bad observables arguments");
    int need = 4 + 2 * rmax;
    if (need > c->obs_cap) {
        cudaFree(c->d_obs);
        c->d_obs = nullptr;
        CK(c, cudaMalloc(&c->d_obs, sizeof(unsigned long long) * need));
        c->obs_cap = need;
    }
    CK(c, cudaMemsetAsync(c->d_obs, 0, sizeof(unsigned long long) * need, c->stream));
    CK(c, fskmc::launch_observables(c->d_lat[c->cur] + R.lat_off, R.lx, R.ly, rmax, c->d_obs,
                                    c->stream, c->packed));
    std::vector<unsigned long long> h(need);
    CK(c, cudaMemcpyAsync(h.data(), c->d_obs, sizeof(unsigned long long) * need, cudaMemcpyDeviceToHost,
                          c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    const double N = (double)R.lx * (double)R.ly;
    for (int s = 0; s < 3; ++s) coverage[s] = (double)h[s] / N;
    const double pairs = (double)h[3], n1 = (double)h[1];
    if (c->model == fskmc::ZGB) *energy = NAN;
    else if (c->model == fskmc::ISING) *energy = -(4.0 * pairs - 8.0 * n1 + 2.0 * N) / N;
    else *energy = -pairs / N;
    for (int r = 0; r < 2 * rmax; ++r) paircorr[r] = (double)h[4 + r] / N;
    return FSKMC_OK;
}

fskmc_status fskmc_stats(fskmc_ctx *c, uint64_t out[5])
{
    if (!c || !out) return FSKMC_EINVAL;
    unsigned long long h[4];
    CK(c, cudaMemcpyAsync(h, c->d_counters, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    out[0] = h[0];
    out[1] = c->windows;
    out[2] = h[1];
    out[3] = h[2];
    out[4] = h[3];
    return FSKMC_OK;
}

fskmc_status fskmc_exact_edge_checks(fskmc_ctx *c, uint64_t *out)
{
    if (!c || !out) return FSKMC_EINVAL;
    unsigned long long h;
    CK(c, cudaMemcpyAsync(&h, c->d_counters + 4, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    *out = h;
    return FSKMC_OK;
}

fskmc_status fskmc_workload(fskmc_ctx *c, int32_t replica, int32_t *out)
{
    if (!c || !out) return FSKMC_EINVAL;
    if (replica < 0 || replica >= c->nrep) return fail(c, FSKMC_EINVAL, "bad replica %d", replica);
    const Replica &R = c->reps[replica];
    CK(c, cudaMemcpyAsync(out, c->d_workload + R.cell_off, sizeof(int32_t) * R.ncx * R.ncy,
                          cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return FSKMC_OK;
}

fskmc_status fskmc_sync(fskmc_ctx *c)
{
    if (!c) return FSKMC_EINVAL;
    CK(c, cudaStreamSynchronize(c->stream));
    return FSKMC_OK;
}

fskmc_status fskmc_schedule(fskmc_scheme scheme, double dt, double T, uint64_t seed,
                            uint32_t replica, uint64_t w0, int32_t *colour, double *h,
                            int64_t cap, int64_t *nwindows)
{
    if (!nwindows) return fail(nullptr, FSKMC_EINVAL, "NULL nwindows");
    if ((int)scheme < 0 || (int)scheme > 3) return fail(nullptr, FSKMC_EINVAL, "unknown scheme %d", (int)scheme);
    if (replica >= (1u << 24)) return fail(nullptr, FSKMC_EINVAL, "replica id must be < 2^24");
    const int64_t n = nsteps(dt, T);
    if (n < 0) return fail(nullptr, FSKMC_EINVAL, "dt must be > 0, T >= 0 and T/dt an integer");
    std::vector<Win> sched;
    build_schedule(scheme, n, dt, seed, replica, w0, sched);
    *nwindows = (int64_t)sched.size();
    if (!colour && !h) return FSKMC_OK;
    if (!colour || !h || cap < (int64_t)sched.size())
        return fail(nullptr, FSKMC_EINVAL, "output arrays missing or too small (%lld windows)",
                    (long long)sched.size());
    for (size_t i = 0; i < sched.size(); ++i) {
        colour[i] = sched[i].colour;
        h[i] = sched[i].h;
    }
    return FSKMC_OK;
}

fskmc_status fskmc_selftest_divide(const double *a, const double *b, int32_t n,
                                   uint32_t *mismatches)
{
    if (!a || !b || !mismatches || n < 0) return fail(nullptr, FSKMC_EINVAL, "bad self-test arguments");
    double *da = nullptr, *db = nullptr;
    unsigned int *dbad = nullptr;
    cudaError_t e = cudaMalloc(&da, sizeof(double) * (size_t)n + 8);
    if (e == cudaSuccess) e = cudaMalloc(&db, sizeof(double) * (size_t)n + 8);
    if (e == cudaSuccess) e = cudaMalloc(&dbad, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemcpy(da, a, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(db, b, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(dbad, 0, sizeof(unsigned int));
    if (e == cudaSuccess) e = fskmc::launch_div_selftest(da, db, n, dbad, nullptr);
    unsigned int bad = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&bad, dbad, sizeof bad, cudaMemcpyDeviceToHost);
    cudaFree(da);
    cudaFree(db);
    cudaFree(dbad);
    if (e != cudaSuccess) return fail(nullptr, FSKMC_ECUDA, "self-test: %s", cudaGetErrorString(e));
    *mismatches = bad;
    return FSKMC_OK;
}

fskmc_status fskmc_selftest_log(const uint64_t *nn, int32_t count, double *out)
{
    if (!nn || !out || count < 0) return fail(nullptr, FSKMC_EINVAL, "bad self-test arguments");
    for (int32_t i = 0; i < count; ++i)
        if (nn[i] < 1 || nn[i] > (1ull << 53)) return fail(nullptr, FSKMC_EINVAL, "n[%d] outside [1, 2^53]", i);
    unsigned long long *dn = nullptr;
    double *dout = nullptr;
    cudaError_t e = cudaMalloc(&dn, sizeof(unsigned long long) * (size_t)count + 8);
    if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(double) * (size_t)count + 8);
    if (e == cudaSuccess) e = cudaMemcpy(dn, nn, sizeof(unsigned long long) * (size_t)count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = fskmc::launch_log_selftest(dn, count, dout, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost);
    cudaFree(dn);
    cudaFree(dout);
    if (e != cudaSuccess) return fail(nullptr, FSKMC_ECUDA, "self-test: %s", cudaGetErrorString(e));
    return FSKMC_OK;
}

fskmc_status fskmc_autotune(int32_t n, const fskmc_lattice *lattices, fskmc_model model,
                            const fskmc_rates *rates, fskmc_scheme scheme, double dt,
                            fskmc_clock clock, fskmc_engine engine, double coverage, uint64_t seed,
                            void *stream, fskmc_cell_shape *best_cell, int32_t *best_wpb,
                            double *best_rate)
{
    if (!lattices || !rates || !best_cell || !best_wpb)
        return fail(nullptr, FSKMC_EINVAL, "NULL argument");
    if (!(dt > 0.0)) return fail(nullptr, FSKMC_EINVAL, "dt must be > 0");
    cudaStream_t s = (cudaStream_t)stream;
    double best = -1.0;
    fskmc_cell_shape bc = {0, 0};
    int bw = 0;
    // square cells in {8, 16, 32}; on a ring, cells of 32..1024 sites
    std::vector<fskmc_cell_shape> shapes;
    if ((int)model == fskmc::ISING1D) {
        for (int q = 32; q <= fskmc::MAX_Q_RING; q <<= 1) shapes.push_back({q, 1});
    } else {
        for (int q : {8, 16, 32}) shapes.push_back({q, q});
    }
    for (const fskmc_cell_shape &shape : shapes) {
        fskmc_ctx *c = nullptr;
        if (make_ctx(n, lattices, model, rates, shape, stream, true, &c) != FSKMC_OK)
            continue;  // this cell size does not fit every lattice
        fskmc_status st = fskmc_set_clock(c, clock);
        if (!st) st = fskmc_set_engine(c, engine);
        if (!st) st = fskmc_init_random(c, seed, coverage);
        for (int wpb : {2, 4, 8}) {
            if (st || fskmc_set_warps_per_block(c, wpb) != FSKMC_OK) break;
            // warm-up step, then a timed run of 4 steps from where it left off
            st = fskmc_run(c, scheme, dt, dt, seed);
            if (st) break;
            uint64_t before[5], after[5];
            if ((st = fskmc_stats(c, before)) != FSKMC_OK) break;
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            cudaEventRecord(a, s);
            st = fskmc_run(c, scheme, dt, 4.0 * dt, seed);
            cudaEventRecord(b, s);
            cudaEventSynchronize(b);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, a, b);
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            if (st || (st = fskmc_stats(c, after)) != FSKMC_OK) break;
            const double rate = ms > 0.0f ? (double)(after[0] - before[0]) / (ms * 1e-3) : 0.0;
            if (rate > best) {
                best = rate;
                bc = shape;
                bw = wpb;
            }
        }
        fskmc_destroy(c);
        if (st) return fail(nullptr, st, "autotune trial failed for cell %dx%d", shape.qx, shape.qy);
    }
    if (best < 0.0) return fail(nullptr, FSKMC_EINVAL, "no candidate cell shape fits every lattice");
    *best_cell = bc;
    *best_wpb = bw;
    if (best_rate) *best_rate = best;
    g_create_error.clear();
    return FSKMC_OK;
}

}  // extern "C"
