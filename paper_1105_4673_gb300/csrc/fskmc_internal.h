// Internal declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace fskmc {

enum Model : int { ADSDES = 0, ISING = 1, DIFFUSION = 2, ZGB = 3, ISING1D = 4 };

constexpr int MAX_CLASSES = 16;
constexpr int MAX_Q = 32;
constexpr int MAX_Q_RING = 1024;  // cell length on a ring (ISING1D)
constexpr int MAX_CELL_SITES = 1024;

// Per-replica description, resident on the device.
struct Replica {
    int32_t lx, ly;      // lattice sides
    int32_t ncx, ncy;    // cells along x and y
    int64_t lat_off;     // byte offset of the replica's lattice in the lattice buffer
                         // (one byte per site, or 32 sites per 32-bit word when packed)
    int32_t cell_off;    // index of the replica's cell 0 in per-cell arrays
    uint32_t rep;        // replica word of the random counters
    double r[MAX_CLASSES];       // class rates, binary64
    uint64_t rq[MAX_CLASSES];    // the rates in fixed point: round(r * 2^qshift)
    float qscale;                // 2^-qshift (binary32 clock path)
    int32_t qshift;
};

// n / d for 0 <= n < 2^16 and 1 <= d <= 2^16 as (n * M) >> 32, M = ceil(2^32 / d).
struct FastDiv {
    uint32_t d;
    uint64_t M;
};
inline FastDiv make_fastdiv(uint32_t d)
{
    FastDiv f;
    f.d = d;
    f.M = ((1ull << 32) + d - 1) / d;
    return f;
}

// Cell shape and the divisions the window kernel needs.
struct CellGeom {
    int32_t qx, qy;
    FastDiv fqx;  // by qx
};
inline CellGeom make_geom(int qx, int qy)
{
    CellGeom g;
    g.qx = qx;
    g.qy = qy;
    g.fqx = make_fastdiv((uint32_t)qx);
    return g;
}

// Arguments of one fractional window over the active cells of one replica.
struct WindowArgs {
    const Replica *reps;       // device array
    int32_t rep_index;         // which replica
    CellGeom geom;             // cell shape
    int32_t colour;            // 0 = E, 1 = O
    uint32_t w;                // global window index
    double h;                  // window length
    uint64_t seed;
    const uint8_t *src;        // lattice at window start (all replicas)
    uint8_t *dst;              // result (== src when updated in place)
    int32_t *workload;         // events per cell in its latest window
    unsigned long long *counters;  // [0] events, [1] ambiguous cell-windows, [2] timeouts
    int32_t packed;            // lattice stored 1 bit per site (spin-flip models)
    const int32_t *order;      // active cells of the window (cell ids) in issue order, or null
    int32_t lanes_per_cell;    // 32: one cell per warp; 4, 8 or 16: grouped (spin-flip models)
    int32_t screen;            // binary64 clock: screened window-edge decisions (edge_screen)
};

// Arguments of one outer window of the nested (two-level) scheme over the
// super-cells of one colour of one replica (fskmc_nested.cu).
struct NestedArgs {
    const Replica *reps;       // device array
    int32_t rep_index;
    CellGeom geom;             // sub-cell shape
    int32_t Qx, Qy;            // super-cell shape (Qx % 2qx == 0, Qy % 2qy == 0)
    int32_t colour;            // outer colour C: 0 = E, 1 = O
    uint32_t w0;               // window index of the first inner window (w_outer * ninner)
    int32_t inner;             // inner schedule: 0 Lie, 1 Strang
    int32_t ninner;            // inner windows per outer window
    double d, dhalf;           // inner step h / n_in and its half
    uint64_t seed;
    uint8_t *lat;              // all replicas, updated in place
    int32_t *workload;         // events per sub-cell in its latest inner window
    unsigned long long *counters;
    int32_t packed;            // 1 bit per site in device memory (then Qx % 32 == 0)
    int32_t screen;            // binary64 clock: screened window-edge decisions
    int32_t super_bytes;       // shared bytes of the staged super-cell (16-byte multiple)
    int32_t lanes;             // lanes per sub-cell: 32 (one per warp) or 8 / 16 (grouped)
};

// Shared-memory bytes of one nested block (super-cell + wpb sub-cell warps),
// and the launch of one outer window (nsuper_active blocks).
size_t nested_smem(int model, int Qx, int Qy, int qx, int qy, int wpb, int lanes);
cudaError_t launch_nested(int model, int fp32, const NestedArgs &a, int nsuper_active, int wpb,
                          cudaStream_t s);

// Shared-memory bytes one warp of the window kernel needs.
size_t window_smem_per_warp(int model, int qx, int qy);
// The two-cells-per-warp ZGB window with the binary32 clock
// (fskmc_zgbpair.cu): whether a cell shape takes it, its shared memory per
// warp, its one-window launch (pairs of active cells, wpb warps per CTA) and
// its persistent kernel (args: PParams by value, int shared bytes per warp).
bool zgb_pair_shape(int qx, int qy);
size_t zgb_pair_smem_per_warp(int qy);
cudaError_t launch_zgb_pair_window(const WindowArgs &a, int nactive, int wpb, cudaStream_t st);
void *zgb_pair_persistent_kernel();
// The rl-cells-per-warp ZGB window (fskmc_zgbquad.cu; rl = 4 or 8): 32-wide
// cells of 2 rl to 32 rows in multiples of rl, binary32 clock; as the
// two-cell calls.
bool zgb_multi_shape(int rl, int qx, int qy);
size_t zgb_multi_smem_per_warp(int rl);
cudaError_t launch_zgb_multi_window(int rl, const WindowArgs &a, int nactive, int wpb, cudaStream_t st);
void *zgb_multi_persistent_kernel(int rl);

// Lanes per cell of the grouped window kernels (several small cells per
// warp, spin-flip models only): the lanes owning the cell's 32-site words,
// rounded up to a power of two and at least the lanes one flip's class
// refresh uses (8 in 2D, 4 on a ring); 32 means the cell takes a whole warp
// (not grouped).
int group_width(int model, int qx, int qy);
// Shared-memory bytes one warp of the grouped kernels needs (0 if not grouped).
size_t group_smem_per_warp(int model, int qx, int qy);
// The grouped kernel for (model, clock, storage, cell shape): plain window
// kernel (args: WindowArgs, int nactive, int stride) or persistent kernel
// (args: PParams by value, int stride), stride = group_smem_per_warp / (32 / W).
void *group_kernel_for(int model, int fp32, bool packed, int qx, int qy, bool persistent);
// The same per clock, for W lanes per cell.
void *group_kernel_f64(int model, bool packed, int lanes, bool persistent);
void *group_kernel_f32(int model, bool packed, int lanes, bool persistent);
cudaError_t launch_group_window(int model, int fp32, const WindowArgs &a, int nactive, int wpb,
                                cudaStream_t s);

// Launch one window (all active cells of a.rep_index).
cudaError_t launch_window(int model, int fp32, const WindowArgs &a, int ncells_active,
                          int warps_per_block, cudaStream_t s);

// Initial states.
cudaError_t launch_init_bernoulli(uint8_t *lat, int lx, int ly, uint64_t seed, double p,
                                  uint32_t rep, cudaStream_t s);
cudaError_t launch_init_bump(uint8_t *lat, int lx, int ly, uint64_t seed, const double *gx,
                             const double *gy, double amp, int species, uint32_t rep,
                             cudaStream_t s);

// Integer observables: out[0..2] state counts, out[3] occupied NN pairs,
// out[4 .. 4+rmax) G_x sums, out[4+rmax .. 4+2 rmax) G_y sums.
cudaError_t launch_observables(const uint8_t *lat, int lx, int ly, int rmax,
                               unsigned long long *out, cudaStream_t s, bool packed = false);

// Bit-packed storage: 32 consecutive sites of a row per 32-bit word, site x
// in bit x % 32 of word y * lx/32 + x/32 (lx a multiple of 32).
cudaError_t launch_pack(const uint8_t *bytes, uint32_t *words, int lx, int ly, cudaStream_t s);
cudaError_t launch_unpack(const uint32_t *words, uint8_t *bytes, int lx, int ly, cudaStream_t s);

// Workload-ordered issue lists (heaviest first by the per-cell event counts
// of each cell's previous window). For replicas r0 .. r0+nrep-1 and the
// colours in [c0, c1]: order[R.cell_off + c * ncells/2 + u] = the u-th
// active cell of colour c in descending workload (bucketed: exact below 64
// events, 8 buckets per power of two above). hist/cursor: scratch of
// ORDER_BUCKETS * nrep * 2 ints each, cleared by the call.
constexpr int ORDER_BUCKETS = 264;
cudaError_t launch_order(const Replica *reps_host, const Replica *reps_dev, int r0, int nrep,
                         int c0, int c1, int qx, int qy, const int32_t *workload, int32_t *order,
                         int32_t *hist, int32_t *cursor, cudaStream_t s);

// Self-test of the window kernel's integer-pipe division against the
// hardware correctly rounded divide: counts disagreeing pairs into *bad.
cudaError_t launch_div_selftest(const double *a, const double *b, int n, unsigned int *bad,
                                cudaStream_t s);

// The window kernels' binary64 -log(n 2^-53) for n[i] in [1, 2^53] into out.
cudaError_t launch_log_selftest(const unsigned long long *n, int count, double *out, cudaStream_t s);

// Validation of a lattice: counts bytes >= nstates into *bad.
cudaError_t launch_validate(const uint8_t *lat, int64_t n, int nstates, unsigned int *bad,
                            cudaStream_t s);

}  // namespace fskmc
