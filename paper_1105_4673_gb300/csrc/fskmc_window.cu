// Fractional-step window kernels of the plain and persistent engines: one
// warp per coarse cell, each running cell_window (fskmc_cell.cuh).
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
#include <algorithm>
#include <cuda/atomic>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "fskmc_cell.cuh"
#include "fskmc_device.cuh"
#include "fskmc_diff32.cuh"
#include "fskmc_zgb32.cuh"
#include "fskmc_internal.h"
#include "fskmc_persistent.h"
#include "philox.cuh"

namespace fskmc {

namespace {

// Plain engine: one launch per window, one warp per active cell of one replica.
// ROWREG: 32-wide ZGB or diffusion cells with the binary32 clock, held in
// registers (zgb32_window, diff32_window); otherwise the generic window
// (cell_window).
// Held to 64 registers (two 512-thread blocks per SM): with more warps
// resident the latency of one event's chain hides better (16384^2 ZGB:
// +2-8%; the binary64 forms spill a few words and still gain).
template <int MODEL, typename CLK, bool PACKED, bool ROWREG = false>
__global__ void __launch_bounds__(512, 2) fs_window_kernel(WindowArgs a, int nactive, int smem_per_warp)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int g = blockIdx.x * (blockDim.x >> 5) + wib;
    if (g >= nactive) return;
    const Replica &R = a.reps[a.rep_index];
    int cx, cy;
    if (a.order) {  // heaviest-first issue list
        const int m = a.order[g];
        cy = m / R.ncx;
        cx = m - cy * R.ncx;
    } else {
        const int half = R.ncx >> 1;
        cy = g / half;
        cx = 2 * (g % half) + ((a.colour + cy) & 1);
    }
    const uint8_t *src = a.src + R.lat_off;
    uint8_t *dst = a.dst + R.lat_off;
    if (a.src != a.dst) {
        // the inactive neighbour whose unwritten sites this warp copies:
        // right of an E cell, below an O cell
        int ncx2 = a.colour == 0 ? (cx + 1) % R.ncx : cx;
        int ncy2 = a.colour == 0 ? cy : (cy + 1) % R.ncy;
        copy_unwritten<false>(src, dst, R.lx, R.ly, a.geom.qx, a.geom.qy, ncx2, ncy2, a.colour, lane);
    }
    bool amb = false, bad = false;
    uint32_t nexact = 0;
    uint32_t e;
    if constexpr (ROWREG && MODEL == DIFFUSION)
        e = diff32_window<false>(smem + (size_t)wib * smem_per_warp, R, a.geom, cell_at(R, a.geom, cx, cy),
                                 a.colour, a.w, a.h, a.seed, src, dst, lane, &bad);
    else if constexpr (ROWREG)
        e = zgb32_window<false>(smem + (size_t)wib * smem_per_warp, R, a.geom, cell_at(R, a.geom, cx, cy),
                                a.colour, a.w, a.h, a.seed, src, dst, lane, &bad);
    else
        e = cell_window<MODEL, CLK, false, PACKED>(smem + (size_t)wib * smem_per_warp, R, a.geom,
                                                   cell_at(R, a.geom, cx, cy), a.colour, a.w, a.h, a.screen != 0,
                                                   a.seed, src, dst, lane, &amb, &bad, &nexact);
    if (lane == 0) {
        a.workload[R.cell_off + cy * R.ncx + cx] = (int32_t)e;
        atomicAdd(&a.counters[0], (unsigned long long)e);
        if (amb) atomicAdd(&a.counters[1], 1ull);
        if (bad) atomicAdd(&a.counters[3], 1ull);
        if (nexact) atomicAdd(&a.counters[4], (unsigned long long)nexact);
    }
}

// ---------------------------------------------------------------------------
// Persistent engine. One launch runs every window of every replica; tasks
// are dequeued from one global counter, window-major, and a task waits only
// on tasks that precede it in that order, so a dequeued task's prerequisites
// are always held by running warps.
// In-place models (spin flip, ZGB): tasks are the active cells only.
//   epoch[m] = 1 + the last window in which cell m was active. Active (m, i)
//   needs epoch[m] >= 1 + (m's previous active window) and, for each edge
//   neighbour n, epoch[n] >= 1 + (n's last active window before i): then no
//   site m reads or writes is being written or read by anyone else.
// Ping-pong model (diffusion): every cell has a task in every window, active
//   cells first. epoch[m] = i + 1 once every read and write of m's sites for
//   windows <= i is done. Active (m, i) waits on its 3x3 neighbourhood at
//   epoch >= i; inactive (m, i) does the same, copies its unwritten sites,
//   then waits until its 4 active edge neighbours reach epoch i + 1.
// Every wait polls at most spin_limit times; on expiry the warp raises the
// abort flag, counts a timeout and the whole launch drains.
// ---------------------------------------------------------------------------

// Held to 64 registers (four 256-thread blocks per SM), as the plain kernel.
// The parameters are a kernel argument (constant bank), so the loop reads
// them without holding them in registers.
template <int MODEL, typename CLK, bool PACKED, bool ROWREG = false>
__global__ void __launch_bounds__(256, 4) fs_persistent_kernel(const __grid_constant__ PParams P,
                                                               int smem_per_warp)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    uint8_t *wsm = smem + (size_t)wib * smem_per_warp;
    const bool pingpong = P.lat2 != nullptr;
    const bool inplace = P.inplace != 0;
    // One task per active cell and window; with ping-pong storage the task
    // also copies the unwritten sites of the inactive cell to its right
    // (each inactive cell is the right neighbour of exactly one active cell).
    const int per_window = P.total_active;
    const unsigned long long total = (unsigned long long)P.nwin * (unsigned long long)per_window;

    // In-place models with the binary64 clock: the next task is dequeued
    // while this one runs, which hides the round trip to the much-contended
    // queue counter (tasks wait only on tasks of earlier windows, all
    // dequeued before it, so holding one cannot block them). The binary32
    // clock's shorter tasks and the ping-pong model's dense copy tasks run
    // better without it.
    const bool prefetch = inplace && sizeof(CLK) == 8;
    unsigned long long t_next = 0;
    if (prefetch && lane == 0) t_next = atomicAdd(P.queue, 1ull);
    for (;;) {
        unsigned long long t = 0;
        if (prefetch) {
            t = __shfl_sync(0xffffffffu, t_next, 0);
            if (t >= total) break;
            if (lane == 0) t_next = atomicAdd(P.queue, 1ull);
        } else {
            if (lane == 0) t = atomicAdd(P.queue, 1ull);
            t = __shfl_sync(0xffffffffu, t, 0);
            if (t >= total) break;
        }
        int ab = 0;
        if (lane == 0) ab = *(volatile int32_t *)P.abort_flag;
        if (__shfl_sync(0xffffffffu, ab, 0)) break;
        const int i = (int)(t / (unsigned long long)per_window);
        const int u = (int)(t % (unsigned long long)per_window);
        const int2 rk = P.cell_rk[u];
        const int r = rk.x;
        const int k = rk.y;
        const Replica &R = P.reps[r];
        const int64_t widx = P.colour_per_replica ? (int64_t)r * P.nwin + i : i;
        const int ccol = P.colour[widx];
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
        const int slot = R.cell_off + m;
        uint8_t *cur = (pingpong && (i & 1)) ? P.lat2 : P.lat;
        uint8_t *nxt = pingpong ? ((i & 1) ? P.lat : P.lat2) : cur;
        cur += R.lat_off;
        nxt += R.lat_off;

        bool ok = true;
        if (inplace) {
            // epoch[c] = 1 + the last window in which cell c was active.
            // Lane 0: this cell's previous active window; lanes 1..4: the
            // edge neighbours' last active window before this one.
            // A ring (one row of cells) has no vertical neighbours.
            const int2 pv = P.prev[widx];
            const int ex = lane == 1 ? 1 : (lane == 3 ? -1 : 0);
            const int ey = lane == 2 ? 1 : (lane == 4 ? -1 : 0);
            const int dcx = (cx + ex + R.ncx) % R.ncx, dcy = (cy + ey + R.ncy) % R.ncy;
            const int target = (lane == 0 ? pv.x : pv.y) + 1;
            const bool dep = lane < 5 && target > 0 && !(ey != 0 && R.ncy == 1);
            ok = wait_epochs(ep, dcy * R.ncx + dcx, dep, target, P, lane);
        } else {
            // ping-pong: epoch[c] = 1 + the last window whose work on cell c
            // is complete (an active cell's window, an inactive cell's
            // copy). The active cell and the inactive cell to its right each
            // need their 3x3 neighbourhood done with the previous window: the
            // 4 x 3 cells from one left of this cell to two right of it.
            const int ddx = (lane & 3) - 1, ddy = (lane >> 2) - 1;
            const int dcx = (cx + ddx + R.ncx) % R.ncx, dcy = (cy + ddy + R.ncy) % R.ncy;
            ok = wait_epochs(ep, dcy * R.ncx + dcx, lane < 12, i, P, lane);
        }
        if (!ok) break;
        bool amb = false, bad = false;
        uint32_t nexact = 0;
        uint32_t e;
        if constexpr (ROWREG && MODEL == DIFFUSION)
            e = diff32_window<true>(wsm, R, P.geom, cell_at(R, P.geom, cx, cy), ccol, P.w0 + (uint32_t)i,
                                    P.h[i], P.seed, cur, nxt, lane, &bad);
        else if constexpr (ROWREG)
            e = zgb32_window<true>(wsm, R, P.geom, cell_at(R, P.geom, cx, cy), ccol, P.w0 + (uint32_t)i,
                                   P.h[i], P.seed, cur, nxt, lane, &bad);
        else
            e = cell_window<MODEL, CLK, true, PACKED>(wsm, R, P.geom, cell_at(R, P.geom, cx, cy), ccol,
                                                      P.w0 + (uint32_t)i, P.h[i], P.screen != 0, P.seed,
                                                      cur, nxt, lane, &amb, &bad, &nexact);
        if (lane == 0) {
            P.workload[slot] = (int32_t)e;
            atomicAdd(&P.counters[0], (unsigned long long)e);
            if (amb) atomicAdd(&P.counters[1], 1ull);
            if (bad) atomicAdd(&P.counters[3], 1ull);
            if (nexact) atomicAdd(&P.counters[4], (unsigned long long)nexact);
        }
        if (pingpong) {
            // the inactive cell to the right. It publishes its window as soon
            // as its copy is done: whoever next reads or overwrites the sites
            // its active edge neighbours write into it (its edge band, its
            // corners) waits on those neighbours too, since every task waits
            // on the 3x3 neighbourhood of the cells it works on and the cells
            // reading this cell's corners have the writers of those corners
            // as edge neighbours.
            copy_unwritten<true>(cur, nxt, R.lx, R.ly, P.geom.qx, P.geom.qy, (cx + 1) % R.ncx, cy, ccol, lane);
        }
        // the warp barrier orders every lane's writes before lane 0's release
        // store (release is cumulative), which publishes them
        __syncwarp();
        if (lane == 0) {
            cuda::atomic_ref<int32_t, cuda::thread_scope_device> ea(P.epoch[slot]);
            ea.store(i + 1, cuda::memory_order_release);
        }
        if (pingpong && lane == 1) {
            cuda::atomic_ref<int32_t, cuda::thread_scope_device> eb(P.epoch[R.cell_off + cy * R.ncx + (cx + 1) % R.ncx]);
            eb.store(i + 1, cuda::memory_order_release);
        }
    }
}

template <int MODEL>
cudaError_t launch_model(int fp32, const WindowArgs &a, int nactive, int wpb, cudaStream_t st)
{
    if (a.lanes_per_cell < 32) {
        // ZGB: two 32-wide cells per warp (binary32 clock); the spin-flip
        // models: the grouped kernels
        if constexpr (MODEL == ZGB) {
            const int rl = 32 / a.lanes_per_cell;  // cells per warp
            if (fp32 && (rl == 4 || rl == 8) && zgb_multi_shape(rl, a.geom.qx, a.geom.qy))
                return launch_zgb_multi_window(rl, a, nactive, wpb, st);
            if (!fp32 || a.lanes_per_cell != 16 || !zgb_pair_shape(a.geom.qx, a.geom.qy)) return cudaErrorInvalidValue;
            return launch_zgb_pair_window(a, nactive, wpb, st);
        }
        return launch_group_window(MODEL, fp32, a, nactive, wpb, st);
    }
    int spw = make_layout<MODEL>(a.geom.qx, a.geom.qy).bytes;
    if constexpr (MODEL == ZGB) spw = std::max(spw, zgb32_smem(a.geom.qy));  // either window fits
    if constexpr (MODEL == DIFFUSION) spw = std::max(spw, diff32_smem(a.geom.qy));
    size_t smem = (size_t)spw * wpb;
    int blocks = (nactive + wpb - 1) / wpb;
    if (blocks == 0) return cudaSuccess;
    void (*kern)(WindowArgs, int, int) = nullptr;
    if constexpr (is_spin_flip<MODEL>()) {
        if (a.packed) kern = fp32 ? fs_window_kernel<MODEL, float, true> : fs_window_kernel<MODEL, double, true>;
    }
    if constexpr (MODEL == ZGB || MODEL == DIFFUSION) {
        if (fp32 && a.geom.qx == 32 && a.geom.qy >= 2) kern = fs_window_kernel<MODEL, float, false, true>;
    }
    if (!kern) kern = fp32 ? fs_window_kernel<MODEL, float, false> : fs_window_kernel<MODEL, double, false>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<blocks, 32 * wpb, smem, st>>>(a, nactive, spw);
    return cudaGetLastError();
}

template <int MODEL>
void *persistent_kernel_ptr(int fp32, bool packed, int qx, int qy)
{
    if constexpr (MODEL == ZGB || MODEL == DIFFUSION) {
        if (fp32 && qx == 32 && qy >= 2) return (void *)fs_persistent_kernel<MODEL, float, false, true>;
    }
    if constexpr (is_spin_flip<MODEL>()) {
        if (packed)
            return fp32 ? (void *)fs_persistent_kernel<MODEL, float, true>
                        : (void *)fs_persistent_kernel<MODEL, double, true>;
    }
    return fp32 ? (void *)fs_persistent_kernel<MODEL, float, false>
                : (void *)fs_persistent_kernel<MODEL, double, false>;
}

void *persistent_kernel_for(int model, int fp32, bool packed, int qx, int qy)
{
    switch (model) {
    case ADSDES: return persistent_kernel_ptr<ADSDES>(fp32, packed, qx, qy);
    case ISING: return persistent_kernel_ptr<ISING>(fp32, packed, qx, qy);
    case DIFFUSION: return persistent_kernel_ptr<DIFFUSION>(fp32, false, qx, qy);
    case ZGB: return persistent_kernel_ptr<ZGB>(fp32, false, qx, qy);
    case ISING1D: return persistent_kernel_ptr<ISING1D>(fp32, packed, qx, qy);
    }
    return nullptr;
}

}  // namespace

size_t window_smem_per_warp(int model, int qx, int qy)
{
    switch (model) {
    case ADSDES: return make_layout<ADSDES>(qx, qy).bytes;
    case ISING: return make_layout<ISING>(qx, qy).bytes;
    case DIFFUSION: return std::max(make_layout<DIFFUSION>(qx, qy).bytes, diff32_smem(qy));
    case ZGB: return std::max(make_layout<ZGB>(qx, qy).bytes, zgb32_smem(qy));
    case ISING1D: return make_layout<ISING1D>(qx, qy).bytes;
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
    case ISING1D: return launch_model<ISING1D>(fp32, a, nactive, wpb, st);
    }
    return cudaErrorInvalidValue;
}

// Device buffers of the persistent engine and the graph that launches it:
// reset the per-cell epochs and the queue, then run the persistent kernel.
struct PersistentState {
    int model = -1, fp32 = -1, wpb = -1, grid = 0, packed = -1, lanes = -1;
    // the kernel node of the graph, whose PParams argument is set before each launch
    cudaGraphNode_t knode = nullptr;
    void *kern = nullptr;
    int spw = 0;
    size_t smem = 0;
    int32_t *d_epoch = nullptr;
    unsigned long long *d_queue = nullptr;  // [0] queue, [1] abort flag (low word)
    int32_t *d_prefix = nullptr;
    int2 *d_cell_rk = nullptr;
    int8_t *d_colour = nullptr;
    size_t colour_cap = 0;
    int2 *d_prev = nullptr;
    size_t prev_cap = 0;
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
    cudaFree(st->d_epoch);
    cudaFree(st->d_queue);
    cudaFree(st->d_prefix);
    cudaFree(st->d_cell_rk);
    cudaFree(st->d_colour);
    cudaFree(st->d_prev);
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
        PCK(cudaMalloc(&st->d_epoch, sizeof(int32_t) * (size_t)run.total_cells));
        PCK(cudaMalloc(&st->d_queue, 2 * sizeof(unsigned long long)));
        PCK(cudaMalloc(&st->d_prefix, sizeof(int32_t) * (size_t)(run.nrep + 1)));
        PCK(cudaMallocHost(&st->h_abort, sizeof(int32_t)));
        std::vector<int32_t> pre(run.nrep + 1, 0);
        for (int r = 0; r < run.nrep; ++r)
            pre[r + 1] = pre[r] + run.reps_host[r].ncx * run.reps_host[r].ncy / 2;
        PCK(cudaMemcpyAsync(st->d_prefix, pre.data(), sizeof(int32_t) * pre.size(),
                            cudaMemcpyHostToDevice, s));
        // a -> (replica, index within it): one load per task instead of a search
        std::vector<int2> rk((size_t)std::max(pre[run.nrep], 1));
        for (int r = 0; r < run.nrep; ++r)
            for (int k = 0; k < pre[r + 1] - pre[r]; ++k) rk[(size_t)pre[r] + k] = make_int2(r, k);
        PCK(cudaMalloc(&st->d_cell_rk, sizeof(int2) * rk.size()));
        PCK(cudaMemcpyAsync(st->d_cell_rk, rk.data(), sizeof(int2) * rk.size(), cudaMemcpyHostToDevice, s));
        PCK(cudaStreamSynchronize(s));  // the host vectors go out of scope
        st->total_cells = run.total_cells;
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
    // last earlier window of the same and of the other colour, per window
    std::vector<int2> prev(ncol);
    const int nsched = run.colour_per_replica ? run.nrep : 1;
    for (int r = 0; r < nsched; ++r) {
        int last[2] = {-1, -1};
        for (int64_t i = 0; i < run.nwin; ++i) {
            const int c = run.colour[(size_t)r * run.nwin + i];
            prev[(size_t)r * run.nwin + i] = make_int2(last[c], last[1 - c]);
            last[c] = (int)i;
        }
    }
    if (ncol > st->prev_cap) {
        cudaFree(st->d_prev);
        st->d_prev = nullptr;
        PCK(cudaMalloc(&st->d_prev, sizeof(int2) * ncol));
        st->prev_cap = ncol;
    }
    PCK(cudaMemcpyAsync(st->d_prev, prev.data(), sizeof(int2) * ncol, cudaMemcpyHostToDevice, s));
    PCK(cudaMemcpyAsync(st->d_colour, run.colour, ncol, cudaMemcpyHostToDevice, s));
    PCK(cudaMemcpyAsync(st->d_h, run.h, sizeof(double) * (size_t)run.nwin, cudaMemcpyHostToDevice, s));
    PParams P;
    P.reps = run.reps_dev;
    P.nrep = run.nrep;
    P.geom = make_geom(run.qx, run.qy);
    P.lat = run.lat;
    P.lat2 = run.lat2;
    P.workload = run.workload;
    P.counters = run.counters;
    P.act_prefix = st->d_prefix;
    P.cell_rk = st->d_cell_rk;
    P.total_cells = run.total_cells;
    P.total_active = run.total_cells / 2;
    P.colour = st->d_colour;
    P.colour_per_replica = run.colour_per_replica ? 1 : 0;
    P.prev = st->d_prev;
    P.order = run.order;
    P.inplace = run.lat2 == nullptr ? 1 : 0;
    P.screen = run.screen ? 1 : 0;
    P.h = st->d_h;
    P.nwin = run.nwin;
    P.w0 = (uint32_t)run.w0;
    P.seed = run.seed;
    P.spin_limit = run.spin_limit;
    P.epoch = st->d_epoch;
    P.queue = st->d_queue;
    P.abort_flag = reinterpret_cast<int32_t *>(st->d_queue + 1);
    // (Re)build the graph when the kernel variant or launch shape changes;
    // otherwise set this run's parameters on its kernel node.
    if (st->model != run.model || st->fp32 != run.fp32 || st->wpb != run.wpb ||
        st->packed != (int)run.packed || st->lanes != run.lanes_per_cell) {
        if (st->exec) { cudaGraphExecDestroy(st->exec); st->exec = nullptr; }
        if (st->graph) { cudaGraphDestroy(st->graph); st->graph = nullptr; }
        // grouped kernel (several cells per warp: ZGB's two-cell kernel or
        // the spin-flip models' groups) or one cell per warp; the kernel's
        // int argument is the per-cell (spin-flip groups) or per-warp shared
        // memory
        const bool grouped = run.lanes_per_cell < 32;
        const bool zpair = grouped && run.model == ZGB;
        const int zrl = 32 / run.lanes_per_cell;  // cells per warp
        const bool zquad = zpair && (zrl == 4 || zrl == 8);
        if (zpair && !(run.fp32 && (zquad ? zgb_multi_shape(zrl, run.qx, run.qy) : zgb_pair_shape(run.qx, run.qy)))) {
            *msg = "multi-cell ZGB kernel: binary32 clock, 32-wide cells of a suitable number of rows";
            return cudaErrorInvalidValue;
        }
        void *kern = zquad     ? zgb_multi_persistent_kernel(zrl)
                     : zpair   ? zgb_pair_persistent_kernel()
                     : grouped ? group_kernel_for(run.model, run.fp32, run.packed, run.qx, run.qy, true)
                               : persistent_kernel_for(run.model, run.fp32, run.packed, run.qx, run.qy);
        if (!kern) { *msg = "no persistent kernel for this model and cell width"; return cudaErrorInvalidValue; }
        const int wbytes = zquad     ? (int)zgb_multi_smem_per_warp(zrl)
                           : zpair   ? (int)zgb_pair_smem_per_warp(run.qy)
                           : grouped ? (int)group_smem_per_warp(run.model, run.qx, run.qy)
                                     : (int)window_smem_per_warp(run.model, run.qx, run.qy);
        const int spw = (grouped && !zpair) ? wbytes / (32 / run.lanes_per_cell) : wbytes;
        const size_t smem = (size_t)wbytes * run.wpb;
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
        int spw_arg = spw;
        void *args[] = {(void *)&P, (void *)&spw_arg};
        cudaLaunchKernel(kern, dim3(st->grid), dim3(32 * run.wpb), args, smem, cs);
        cudaError_t ce = cudaStreamEndCapture(cs, &st->graph);
        cudaStreamDestroy(cs);
        if (ce != cudaSuccess) { *msg = "graph capture"; return ce; }
        PCK(cudaGraphInstantiate(&st->exec, st->graph, 0));
        size_t nn = 0;
        PCK(cudaGraphGetNodes(st->graph, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        PCK(cudaGraphGetNodes(st->graph, nodes.data(), &nn));
        st->knode = nullptr;
        for (cudaGraphNode_t n : nodes) {
            cudaGraphNodeType ty;
            PCK(cudaGraphNodeGetType(n, &ty));
            if (ty == cudaGraphNodeTypeKernel) st->knode = n;
        }
        if (!st->knode) { *msg = "graph capture: no kernel node"; return cudaErrorUnknown; }
        st->kern = kern;
        st->spw = spw;
        st->smem = smem;
        st->model = run.model;
        st->fp32 = run.fp32;
        st->wpb = run.wpb;
        st->packed = (int)run.packed;
        st->lanes = run.lanes_per_cell;
    } else {
        int spw_arg = st->spw;
        void *args[] = {(void *)&P, (void *)&spw_arg};
        cudaKernelNodeParams kp = {};
        kp.func = st->kern;
        kp.gridDim = dim3(st->grid);
        kp.blockDim = dim3(32 * st->wpb);
        kp.sharedMemBytes = (unsigned)st->smem;
        kp.kernelParams = args;
        kp.extra = nullptr;
        PCK(cudaGraphExecKernelNodeSetParams(st->exec, st->knode, &kp));
    }
    PCK(cudaGraphLaunch(st->exec, s));
    PCK(cudaMemcpyAsync(st->h_abort, P.abort_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PCK(cudaStreamSynchronize(s));
    if (*st->h_abort) { *msg = "a bounded wait gave up"; return cudaErrorTimeout; }
    return cudaSuccess;
}

__global__ void div_selftest_kernel(const double *a, const double *b, int n, unsigned int *bad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const double y = __ddiv_rn(a[i], b[i]);
        const double x = div_rn(a[i], b[i]);
        bool slow, slow2;
        double z = div_newton(a[i], b[i], slow);
        if (slow) z = y;  // the caller's fallback
        double u = div_int(a[i], b[i], slow2);
        if (slow2) u = y;
        if (__double_as_longlong(x) != __double_as_longlong(y)) atomicAdd(bad, 1u);
        if (__double_as_longlong(z) != __double_as_longlong(y)) atomicAdd(bad, 1u);
        if (__double_as_longlong(u) != __double_as_longlong(y)) atomicAdd(bad, 1u);
    }
}

__global__ void log_selftest_kernel(const unsigned long long *nn, int n, double *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = neg_log_u53(nn[i]);
}

cudaError_t launch_log_selftest(const unsigned long long *nn, int n, double *out, cudaStream_t s)
{
    if (n > 0) log_selftest_kernel<<<(n + 255) / 256, 256, 0, s>>>(nn, n, out);
    return cudaGetLastError();
}

cudaError_t launch_div_selftest(const double *a, const double *b, int n, unsigned int *bad,
                                cudaStream_t s)
{
    if (n > 0) div_selftest_kernel<<<(n + 255) / 256, 256, 0, s>>>(a, b, n, bad);
    return cudaGetLastError();
}

}  // namespace fskmc
