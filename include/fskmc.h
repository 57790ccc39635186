/*
 * fskmc.h -- C ABI of the GB300 fractional-step parallel kinetic Monte Carlo
 * library (Arampatzis, Katsoulakis, Plechac, Taufer, Xu, "Hierarchical
 * fractional-step approximations and parallel kinetic Monte Carlo
 * algorithms", arXiv:1105.4673).
 *
 * The lattice is split into a checkerboard of coarse cells (Section 2.1,
 * Eq. sublatt). In each fractional window every cell of the active colour
 * runs its own serial SSA (Eqs. totalrate and skeleton) for the window length,
 * reading its neighbours' sites as they were when the window began (Section
 * 2.2, Steps 1-3). The colours are composed by Lie (Eq. lie), Strang
 * (Eq. strang) or random (Eq. SLPCS) schedules (Section 3).
 *
 * General rules for every call:
 *  - Calls return a status code; nothing is thrown or aborted across the
 *    ABI. On failure fskmc_last_error() describes the cause.
 *  - A context is used by one host thread at a time.
 *  - The library owns all device memory of a context. Pointers passed in are
 *    borrowed for the duration of the call only.
 *  - Work is queued on the context's CUDA stream (given at creation; NULL
 *    means the legacy default stream). Calls that return data to the host
 *    (fskmc_get_state to host memory, fskmc_observables, fskmc_stats,
 *    fskmc_workload, fskmc_sync) wait for the stream.
 *  - Lattices are periodic lx*ly, one byte per site, row-major: site (x,y)
 *    is byte y*lx+x. Binary models use 0/1 (1 = occupied, or spin +1 for
 *    ISING); ZGB uses 0 empty, 1 A, 2 B.
 *  - Random numbers are Philox4x32-10 (Salmon et al., SC'11) keyed by the
 *    seed, counter (event, window, cell, replica | tag<<24); results depend
 *    on the seed, the window index, the cell shape and the clock precision,
 *    never on launch configuration.
 */
#ifndef FSKMC_H
#define FSKMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fskmc_ctx fskmc_ctx;

typedef enum {
    FSKMC_OK = 0,
    FSKMC_EINVAL = 1,   /* invalid argument (sizes, rates, schedule, pointers) */
    FSKMC_ENOMEM = 2,   /* device or host allocation failed */
    FSKMC_ECUDA = 3,    /* a CUDA call failed (message in fskmc_last_error) */
    FSKMC_ETIMEOUT = 4, /* a bounded device wait gave up (persistent engine) */
    FSKMC_ESTATE = 5    /* call not valid in the context's current state */
} fskmc_status;

/* Models (Section 2 examples; rates in fskmc_rates). */
typedef enum {
    /* adsorption/desorption spin flip, Eq. adsdesrate with nearest-neighbour
       J: r(empty) = ka, r(occupied, n) = kd exp(-betaJ n) */
    FSKMC_ADSDES = 0,
    /* Ising spin-flip Arrhenius dynamics, Eq. Arrhenius at zero spin field
       (U = K n - h, K = 4J, h = 2K): r(0) = ka, r(1, n) = kd exp(-4 betaJ (n-2)) */
    FSKMC_ISING_ARRHENIUS = 1,
    /* ADSDES plus nearest-neighbour hops (Section 2 example 2) of a particle
       with n occupied neighbours onto an empty site: nu exp(-betaJ n) */
    FSKMC_ADSDES_DIFFUSION = 2,
    /* ZGB CO-oxidation (Table COrates): A adsorbs (yA), B2 adsorbs on an
       empty pair ((1-yA)/4 per directed pair), A+B react ((kr/4) per
       directed pair), A desorbs (kd) */
    FSKMC_ZGB = 3,
    /* 1D Ising benchmark of Section 7 (Eq. exactcov1d): a ring of lx sites
       (ly = 1, cells qx x 1, neighbours x-1 and x+1 only) with
       H = -K sum s(x) s(x+1) + h sum s(x), betaJ = beta K and betah = beta h:
       r(0) = ka, r(1, n) = kd exp(-(betaJ n - betah)), n = occupied
       neighbours (0..2); detailed-balanced with H when ka = kd */
    FSKMC_ISING1D = 4
} fskmc_model;

/* Processor communication schedules (Section 3). */
typedef enum {
    FSKMC_LIE = 0,         /* E(dt) O(dt) per step, Eq. lie */
    FSKMC_STRANG = 1,      /* E(dt/2) O(dt) E(dt/2) per step, Eq. strang */
    FSKMC_RANDOM = 2,      /* sub-lattice random schedule, Eq. SLPCS: 2T/dt windows of
                              length dt, colour fair per window */
    FSKMC_RANDOM_ORDER = 3 /* per step (E,O) or (O,E) with probability 1/2, each dt */
} fskmc_scheme;

/* Precision of the per-cell window clock. FP64: lambda, waiting times and
   the class thresholds in binary64, results bit-identical to the CPU
   oracle. FP32: the same integer class counts and member selection, but
   lambda, waiting times and thresholds in binary32 relative to the window
   start (statistically equivalent, not bit-identical). */
typedef enum { FSKMC_CLOCK_FP64 = 0, FSKMC_CLOCK_FP32 = 1 } fskmc_clock;

/* PLAIN: one kernel launch per window (per replica). PERSISTENT: one
   launch runs every window of every replica, cells advancing as soon as
   their neighbours have finished the previous window; launched through a
   CUDA graph. */
typedef enum { FSKMC_ENGINE_PLAIN = 0, FSKMC_ENGINE_PERSISTENT = 1 } fskmc_engine;

/* Largest lattice side (and ring length) any entry point accepts; lx*ly is
   further limited to 2^31 sites. Site coordinates plus a correlation
   distance then stay within 32-bit integers in every kernel. */
#define FSKMC_MAX_SIDE (1 << 30)

typedef struct {
    int32_t lx, ly;    /* lattice sides; lx % (2 qx) == 0 and ly % (2 qy) == 0
                          (ISING1D: ly == 1, a ring of lx sites); each side at most
                          FSKMC_MAX_SIDE, lx*ly at most 2^31 */
    int32_t bitpacked; /* 1: keep the lattice in device memory at 1 bit per site (32 sites of a
                          row per 32-bit word); spin-flip models only, lx % 32 == 0. The ABI
                          still exchanges one byte per site. Results are identical. */
} fskmc_lattice;

typedef struct {
    double ka, kd, betaJ, nu, yA, kr; /* fields a model does not use are ignored */
    double betah;                     /* ISING1D: beta times the external field h */
} fskmc_rates;

typedef struct {
    int32_t qx, qy; /* coarse cell shape, 1..32 each with qx*qy <= 1024 (ISING1D:
                       qy = 1 and qx in 1..1024); {0,0} asks the autotuner to pick
                       a square q in {8,16,32} (ISING1D: qx in {1024, 512, ..., 32}) */
} fskmc_cell_shape;

/*
 * Create a single-lattice context (Section 2.1: lattice, decomposition into
 * qx*qy cells, model rates). The lattice starts empty (all 0).
 * EINVAL: lx or ly not a positive multiple of 2q; q out of range; models
 * with two-site events and q < 2; ADSDES_DIFFUSION with lx < qx+4 or
 * ly < qy+4 (its frozen halo is two sites wide); negative or non-finite
 * rates; yA outside [0,1]; out == NULL.
 * stream: a cudaStream_t (or NULL); the context keeps it, not owns it.
 */
fskmc_status fskmc_create(const fskmc_lattice *lattice, fskmc_model model,
                          const fskmc_rates *rates, fskmc_cell_shape cell,
                          void *stream, fskmc_ctx **out);

/*
 * Create a context holding n independent replicas (the paper's M
 * independent realisations, Section 7) of possibly different sizes and
 * rates, all of the same model and cell shape. Replica r uses r as the
 * replica word of every random counter, so replica r of a batch evolves
 * exactly like a single context whose replica id is r
 * (fskmc_set_replica_id). lattices[n], rates[n]. Same EINVAL rules as
 * fskmc_create, for every replica; also n < 1 or n > 65536.
 */
fskmc_status fskmc_batch_create(int32_t n, const fskmc_lattice *lattices,
                                fskmc_model model, const fskmc_rates *rates,
                                fskmc_cell_shape cell, void *stream, fskmc_ctx **out);

/* Free every resource of the context (waits for its stream). NULL is a no-op. */
void fskmc_destroy(fskmc_ctx *ctx);

/* Last error message of the context (never NULL; "" after success). With
   ctx == NULL: the last error of a failed create call on this thread. */
const char *fskmc_last_error(const fskmc_ctx *ctx);

/* Replica id of a single context (default 0); EINVAL for batches or id >= 2^24. */
fskmc_status fskmc_set_replica_id(fskmc_ctx *ctx, uint32_t id);

fskmc_status fskmc_set_clock(fskmc_ctx *ctx, fskmc_clock clock);
fskmc_status fskmc_set_engine(fskmc_ctx *ctx, fskmc_engine engine);

/* Launch shape of the window kernels: warps per block, 1..16 (a warp runs
   one cell, or several small cells when grouped, below). Results do not
   depend on it. */
fskmc_status fskmc_set_warps_per_block(fskmc_ctx *ctx, int32_t warps);

/* Cells per warp. Spin-flip models (ADSDES, ISING, ISING1D), mode = 1: a
   cell of at most 512 sites takes W = 4, 8 or 16 lanes (its 32-site words
   rounded up to a power of two; at least 8 in 2D, 4 on a ring) and a warp
   runs 32/W cells of the same window in lockstep, so each instruction of
   the event loop (Eqs. totalrate and skeleton per cell) serves 32/W cells.
   ZGB with the binary32 clock and 32-wide cells, mode = 1: eight cells per
   warp (4 lanes each holding eight rows) for rows a multiple of 8 from 16,
   else four (8 lanes, four rows each) for a multiple of 4 from 8, else two
   (16 lanes, two rows each) for an even number from 4 to 32.
   mode = 0: one cell per warp. mode = 2 (default, auto): the same as 1
   (faster in every engine and clock measured). Diffusion, ZGB otherwise,
   and larger cells always take a whole warp. Results (lattices, event
   counts, workloads) do not depend on the mode. EINVAL: mode outside 0..2. */
fskmc_status fskmc_set_cell_grouping(fskmc_ctx *ctx, int32_t mode);

/* Binary64 clock: how the window-edge decision of each event (Eq. skeleton:
   is tau + (-log u_t)/lambda past the window?) is taken. 1 (default): from a
   binary32 estimate of the waiting time on an exact integer clock with a
   running error bound, the binary64 clock kept a few events behind and used
   only for the events the estimate cannot decide (fskmc_exact_edge_checks
   counts them); 0: every decision from the binary64 clock, caught up for
   each event (a slow checking mode). Results (lattices, event counts,
   workloads, ambiguity counts) do not depend on it. No effect with the
   binary32 clock or in the persistent one-cell kernels (two-site models,
   grouping off), which always divide in binary64. EINVAL: on not 0 or 1. */
fskmc_status fskmc_set_edge_screen(fskmc_ctx *ctx, int32_t on);

/* Order in which the active cells of a window are issued (Section 6,
   Eq. wload). The paper rebalances by reshaping the cells so that each
   processor receives equal work; here the cells keep their shape and the
   active cells of a window are handed to the GPU's block scheduler (plain
   engine) or task queue (persistent engine) heaviest first, by their event
   count W(m) in their previous window (longest-processing-time-first list
   scheduling). NATURAL: row-major cell order. WORKLOAD: heaviest first,
   from the counts each cell had when the fskmc_run or fskmc_window call
   began. AUTO (default): WORKLOAD in the plain engine when a window's
   active cells fill the GPU in one wave (8 to 16 per SM; the block scheduler
   then spreads the heaviest cells over the SMs), else NATURAL (with several
   waves the scheduler balances by itself and row-major order keeps
   neighbouring halos in cache; fewer cells make windows too short to pay for
   the ordering; the persistent queue overlaps windows). Results do not
   depend on the order. */
typedef enum {
    FSKMC_ORDER_NATURAL = 0,
    FSKMC_ORDER_WORKLOAD = 1,
    FSKMC_ORDER_AUTO = 2
} fskmc_task_order;
fskmc_status fskmc_set_task_order(fskmc_ctx *ctx, fskmc_task_order order);

/*
 * Nested (two-level) decomposition, Section 5 (Eq. sublatt2, Eq. opdecomp2).
 * The lattice is a checkerboard of super-cells super_cell.qx x super_cell.qy
 * (colours E/O); each super-cell is a checkerboard of the context's cells
 * (here: sub-cells), so L^E_m = L^EE_m + L^EO_m. With nesting on, fskmc_run
 * and fskmc_window run the outer schedule over the super-cell colours
 * (window length h as without nesting), and inside every outer window each
 * super-cell of that colour runs n_inner inner steps of the inner schedule
 * over its sub-cell colours with step d = h / n_inner: LIE EE(d) EO(d),
 * STRANG EE(d/2) EO(d) EE(d/2). Each inner window is a fractional window of
 * the sub-cells of one inner colour (their own serial SSA, neighbours
 * frozen); its draws use window index w * ninner + j (w the outer window
 * index, j the inner window within it, ninner = 2 or 3 times n_inner) and
 * the sub-cell's id. On the GPU a super-cell is one thread block kept in
 * shared memory for the whole outer window, its sub-cells the block's warps;
 * one launch per outer window (the engine setting does not apply); results
 * are those of the CPU oracle's nested run bit for bit (binary64 clock).
 * fskmc_stats counts inner windows; the window index counts outer windows.
 *
 * super_cell {0, 0}: nesting off (the default). EINVAL: a model other than
 * ADSDES and ISING_ARRHENIUS; super-cell sides not multiples of twice the
 * cell sides; lattice sides not multiples of twice the super-cell sides;
 * inner not LIE or STRANG; n_inner < 1; a bit-packed lattice with
 * super_cell.qx not a multiple of 32; a super-cell too large for one block's
 * shared memory.
 */
fskmc_status fskmc_set_nesting(fskmc_ctx *ctx, fskmc_cell_shape super_cell, fskmc_scheme inner,
                               int32_t n_inner);

/* Persistent engine: how many times a cell polls a neighbour's progress
   before giving up (default 2^20; polls back off to one per 4 us, so about
   4 s). A run whose wait gives up returns FSKMC_ETIMEOUT and leaves the
   lattice undefined. */
fskmc_status fskmc_set_spin_limit(fskmc_ctx *ctx, uint32_t polls);

/* Effective cell shape and sizes: out[0]=qx, out[1]=qy, out[2]=replicas,
   out[3]=total cells over replicas, out[4]=warps per block, out[5]=lanes per
   cell the window kernels use with the current engine, clock and grouping
   mode (32: one cell per warp). */
fskmc_status fskmc_info(const fskmc_ctx *ctx, int32_t out[6]);

/*
 * Bernoulli(coverage) initial state of every replica: site i of replica r
 * is 1 iff word 0 of Philox(seed, (i, 0, 0, r | 2<<24)) < coverage * 2^32.
 * EINVAL: coverage outside [0,1].
 */
fskmc_status fskmc_init_random(fskmc_ctx *ctx, uint64_t seed, double coverage);

/*
 * Gaussian-bump pre-coverage: site (x,y) holds `species` with probability
 * amp * g(dx) * g(dy), g(d) = exp(-d^2 / (2 width^2)), d the periodic
 * distance to a centre drawn from Philox(seed, (0, 0xFFFFFFFF, 0, r|3<<24))
 * (x0 = word0 mod lx, y0 = word1 mod ly); empty otherwise (same per-site
 * draw as fskmc_init_random). EINVAL: amp outside [0,1], width <= 0,
 * species not a state of the model.
 */
fskmc_status fskmc_init_bump(fskmc_ctx *ctx, uint64_t seed, double amp, double width,
                             int32_t species);

/* Copy a replica's lattice in (lx*ly bytes, row-major). is_device != 0: src
   is device memory (read on the context's stream). EINVAL: replica out of
   range, NULL src, a byte that is not a state of the model. */
fskmc_status fskmc_set_state(fskmc_ctx *ctx, int32_t replica, const uint8_t *src,
                             int32_t is_device);

/* Copy a replica's lattice out (lx*ly bytes). is_device != 0: dst is device
   memory (written on the stream, not waited for). */
fskmc_status fskmc_get_state(fskmc_ctx *ctx, int32_t replica, uint8_t *dst,
                             int32_t is_device);

/*
 * All replicas' lattices in one copy each way (a batch of M independent
 * realisations, Section 7, moved between host and device without a call
 * per replica). The state buffer holds the replicas back to back in order,
 * replica r's lx*ly bytes (row-major states) from byte offset out[r], each
 * offset a multiple of 256; out[replicas] is the buffer's size in bytes.
 * The bytes between replicas are copied and otherwise unused; they must
 * hold a state of the model like every other byte (0 will do).
 * fskmc_state_layout: out has room for replicas + 1 entries; EINVAL: NULL.
 * fskmc_set_state_all / fskmc_get_state_all: src / dst is a buffer of that
 * size, device memory if is_device != 0. EINVAL: NULL buffer, a bit-packed
 * context (use the per-replica calls), or (set) a byte that is not a state
 * of the model, in which case every lattice is left cleared to 0. get with
 * host memory waits for the copy; with device memory it is only queued on
 * the context's stream.
 */
fskmc_status fskmc_state_layout(const fskmc_ctx *ctx, int64_t *out);
fskmc_status fskmc_set_state_all(fskmc_ctx *ctx, const uint8_t *src, int32_t is_device);
fskmc_status fskmc_get_state_all(fskmc_ctx *ctx, uint8_t *dst, int32_t is_device);

/*
 * Advance every replica by physical time T with fractional windows of
 * length dt under the given schedule (Section 3). The window counter
 * continues across calls, so two runs of T/2 equal one run of T. T/dt must
 * be an integer within 1e-9 relative (EINVAL otherwise, or dt <= 0, T < 0).
 * Asynchronous on the context's stream. ETIMEOUT (persistent engine only):
 * a cell waited too long for a neighbour; the lattice is then undefined.
 */
fskmc_status fskmc_run(fskmc_ctx *ctx, fskmc_scheme scheme, double dt, double T,
                       uint64_t seed);

/*
 * The windows a run of time T would execute (the processor communication
 * schedule of Section 3: Eq. lie, Eq. strang, Eq. SLPCS), starting at global
 * window index w0 for the given replica id: colour[i] (0 = E, 1 = O) and
 * length h[i]. With colour == h == NULL only *nwindows is set. RANDOM draws
 * each window's colour, RANDOM_ORDER each step's order, from bit 0 of word 0
 * of Philox(seed, (0, w, 0, replica | 3<<24)). EINVAL: as fskmc_run, or
 * arrays shorter than *nwindows.
 */
fskmc_status fskmc_schedule(fskmc_scheme scheme, double dt, double T, uint64_t seed,
                            uint32_t replica, uint64_t w0, int32_t *colour, double *h,
                            int64_t cap, int64_t *nwindows);

/* One window of colour (0 = E, 1 = O) and length h at the current window
   index (then incremented), for every replica. EINVAL: h <= 0, colour not 0/1. */
fskmc_status fskmc_window(fskmc_ctx *ctx, int32_t colour, double h, uint64_t seed);

/* Current global window index, and setting it (for resume). */
fskmc_status fskmc_get_window_index(const fskmc_ctx *ctx, uint64_t *w);
fskmc_status fskmc_set_window_index(fskmc_ctx *ctx, uint64_t w);

/*
 * Observables of Section 7 for one replica, from exact integer sums:
 * coverage[3] = fraction of sites in state 0, 1, 2; energy = -(occupied
 * nearest-neighbour pairs)/N for ADSDES, ADSDES_DIFFUSION and ISING1D,
 * -(1/N) sum_<xy> s_x s_y with s = 2 sigma - 1 for ISING, NaN for ZGB;
 * paircorr[2*rmax] = G_x(1..rmax) then G_y(1..rmax), G_e(r) = (1/N) sum_x
 * [sigma(x)=1][sigma(x + r e)=1]. paircorr may be NULL when rmax == 0.
 * A lattice with ly == 1 is a ring: it has no vertical bonds, and its
 * vertical pairs and G_y are 0.
 * EINVAL: rmax < 0, rmax > lx, rmax > ly when ly > 1, NULL coverage/energy.
 */
fskmc_status fskmc_observables(fskmc_ctx *ctx, int32_t replica, double *coverage,
                               double *energy, double *paircorr, int32_t rmax);

/* Counters since creation: out[0] events executed, out[1] windows run,
   out[2] cell-windows whose last waiting time landed within 1e-12
   (relative) of the window edge, out[3] bounded waits that gave up,
   out[4] cell-windows stopped by the kernel's internal consistency check
   (class counts disagreeing with the member masks; always 0 unless the
   library is broken). */
fskmc_status fskmc_stats(fskmc_ctx *ctx, uint64_t out[5]);

/* Window-edge decisions since creation that the binary64 clock took in
   full (*out). The binary64-clock window kernels of the plain engine and
   the grouped persistent kernels take each decision (Eq. skeleton: is
   tau + (-log u_t)/lambda past the window?) from a binary32 estimate of the
   waiting time on an exact integer clock with a running error bound, and
   keep the binary64 clock tau a few events behind; an event whose estimated
   end lies within that bound of the edge (about 2^-20 of the window length)
   is decided from tau in binary64 on the spot. Results are the same either
   way; this counts those decisions, and every decision of the persistent
   one-cell kernels (which divide in binary64 for each event) and of windows
   run with the screen off (fskmc_set_edge_screen). The binary32 clock
   counts none. */
fskmc_status fskmc_exact_edge_checks(fskmc_ctx *ctx, uint64_t *out);

/* Workload W(m) of Eq. wload: events each cell of a replica executed in its
   most recent window, out[ncx*ncy], cell id m = cy*ncx + cx. */
fskmc_status fskmc_workload(fskmc_ctx *ctx, int32_t replica, int32_t *out);

/* Wait until all work queued on the context's stream has finished. */
fskmc_status fskmc_sync(fskmc_ctx *ctx);

/*
 * Self-test of the binary64 window clock's divides. The waiting time
 * -log(u_t)/lambda of the binary64 contract (Eqs. totalrate/skeleton) is
 * divided without the hardware divide, on the integer pipes: a 64-bit
 * reciprocal of the divisor's significand from a binary32 seed and two
 * integer Newton-Raphson steps, the quotient by a multiply, then an exact
 * remainder that corrects it and decides the rounding to nearest even. A
 * binary64 Newton-Raphson variant is kept for comparison. This compares
 * both (and the window kernels' wrapper with its hardware fallback) with
 * the hardware correctly rounded divide on the n pairs (a[i] >= 0, b[i] > 0,
 * host arrays) and writes the number of disagreements to *mismatches (must
 * be 0). Runs on the current device. EINVAL: NULL pointers, n < 0.
 */
fskmc_status fskmc_selftest_divide(const double *a, const double *b, int32_t n,
                                   uint32_t *mismatches);

/*
 * Self-test of the binary64 window clock's logarithm. The waiting-time
 * numerator -log(u_t), u_t = n 2^-53 (Eqs. totalrate/skeleton with the draw
 * of u_t in (0, 1]), is computed by a table-driven logarithm (Tang's
 * reduction); this writes the device's value for each n[i] (host arrays,
 * 1 <= n[i] <= 2^53) to out[i] so that callers can compare it with a host
 * logarithm. Runs on the current device. EINVAL: NULL pointers, count < 0,
 * n[i] out of range.
 */
fskmc_status fskmc_selftest_log(const uint64_t *n, int32_t count, double *out);

/*
 * Autotuner for the batched workload: for every square cell size q in
 * {8, 16, 32} (ISING1D: cells of q x 1 sites, q in {32, 64, ..., 1024})
 * that all n lattices admit and warps per block in {2, 4, 8},
 * builds a scratch batch context (lattices[n], rates[n], model; Bernoulli
 * (coverage) start from seed), runs one warm-up step and times 4 steps of
 * `scheme` with window dt on the given engine and clock (CUDA events on
 * `stream`). Returns the fastest cell shape and warps per block, and its
 * events/s in *best_rate (may be NULL). The cell shape changes the
 * decomposition, hence the approximation (finer Trotter error at larger q,
 * Section 4); warps per block never change results. Errors are reported
 * through fskmc_last_error(NULL). EINVAL: NULL outputs, dt <= 0, no q fits.
 */
fskmc_status fskmc_autotune(int32_t n, const fskmc_lattice *lattices, fskmc_model model,
                            const fskmc_rates *rates, fskmc_scheme scheme, double dt,
                            fskmc_clock clock, fskmc_engine engine, double coverage,
                            uint64_t seed, void *stream, fskmc_cell_shape *best_cell,
                            int32_t *best_wpb, double *best_rate);

/*
 * Observables of a lattice already in device memory, computed without
 * allocating any memory. The paper has no counterpart: this exists for
 * callers that cannot let a library allocate -- applications whose device
 * memory belongs to their own pool (a framework's caching allocator, a
 * pre-reserved arena), and diagnostics that read the state after an
 * out-of-memory error. No context is needed.
 *
 * lattice: device pointer to lx*ly bytes (row-major, states of `model`).
 * stream: cudaStream_t to run on (NULL = legacy default stream); the call
 * waits for it before returning. Outputs as in fskmc_observables (host
 * memory): coverage[3], *energy, paircorr[2*rmax].
 *
 * The integer accumulators live in one fixed device array of
 * 4 + 2*FSKMC_NOALLOC_MAX_RMAX 64-bit words that every GPU loading the
 * library keeps until the process exits; each call clears the part it
 * uses. All calls share that array, so calls that overlap on the GPU (other
 * streams, other host threads) race and give wrong sums: serialise them.
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress, which allocates nothing once the library's device
 * code is loaded), so a device reset or a new primary context is safe.
 *
 * Warm-up: under CUDA's lazy module loading (the default) the first call on
 * a device loads the library's device code, and loading it does allocate
 * device memory. Make one call per device at start-up -- before memory runs
 * short and before any stream capture; later calls allocate neither device
 * nor host heap memory.
 *
 * EINVAL: NULL lattice/coverage/energy (or paircorr with rmax > 0), unknown
 * model, lx or ly < 1 or > FSKMC_MAX_SIDE, lx*ly > 2^31, rmax < 0,
 * rmax > lx, rmax > ly when ly > 1, or rmax > FSKMC_NOALLOC_MAX_RMAX.
 * ECUDA: a CUDA call failed.
 */
#define FSKMC_NOALLOC_MAX_RMAX 256
fskmc_status fskmc_observables_noalloc(const uint8_t *lattice, int32_t lx, int32_t ly,
                                       fskmc_model model, void *stream, double *coverage,
                                       double *energy, double *paircorr, int32_t rmax);

#ifdef __cplusplus
}
#endif
#endif /* FSKMC_H */
