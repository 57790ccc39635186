// Kernels of the RL-cells-per-warp ZGB window (fskmc_zgb32x4.cuh; RL = 4 or
// 8): 32-wide cells whose rows are a multiple of RL, from 2 RL to 32, with
// the binary32 clock.
//
// fs_zgbq_window_kernel<RL>: one fractional window (Eqs. totalrate and
// skeleton on every active cell), warp g running the window's active cells
// RL g .. RL g + RL - 1 (in issue order when one is given).
// fs_zgbq_persistent_kernel<RL>: the persistent engine of fskmc_window.cu
// for this window, a task being RL consecutive active cells of one window;
// each cell waits on its own prerequisites (its previous active window, its
// edge neighbours' last active window before this one) with the bounded,
// backed-off polls of wait_epochs, and publishes its own epoch.
#include <cuda/atomic>
#include <cuda_runtime.h>

#include "fskmc_device.cuh"
#include "fskmc_internal.h"
#include "fskmc_zgb32x4.cuh"
#include "philox.cuh"

namespace fskmc {

namespace {

// The events of the warp's RL cells to counter 0 and their failures to
// counter 3 (lane 0; every lane calls it; W lanes per cell).
template <int W>
__device__ __forceinline__ void zgbq_count(unsigned long long *counters, int lane, bool valid, uint32_t e, bool bad)
{
    constexpr unsigned leads = W == 8 ? 0x01010101u : 0x11111111u;  // lane 0 of every cell
    const uint32_t evs = __reduce_add_sync(0xffffffffu, (valid && (lane & (W - 1)) == 0) ? e : 0u);
    const unsigned bads = __ballot_sync(0xffffffffu, bad) & leads;
    if (lane == 0) {
        atomicAdd(&counters[0], (unsigned long long)evs);
        if (bads) atomicAdd(&counters[3], (unsigned long long)__popc(bads));
    }
}

// Held to 64 registers (as the other one-window kernels) with four cells
// per warp, to 72 with eight (a small spill; 28 warps per SM with two-warp
// blocks: faster than 80 registers without the spill, or 64 with more).
template <int RL>
__global__ void __maxnreg__(RL == 8 ? 72 : 64) fs_zgbq_window_kernel(WindowArgs a, int nactive, int smem_per_warp)
{
    constexpr int W = 32 / RL;
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int g = blockIdx.x * (blockDim.x >> 5) + wib;
    if (RL * g >= nactive) return;
    const int cidx = RL * g + lane / W;
    const bool valid = cidx < nactive;
    const Replica &R = a.reps[a.rep_index];
    int cx = 0, cy = 0;
    if (valid) {
        if (a.order) {  // heaviest-first issue list
            const int m = a.order[cidx];
            cy = m / R.ncx;
            cx = m - cy * R.ncx;
        } else {
            const int half = R.ncx >> 1;
            cy = cidx / half;
            cx = 2 * (cidx % half) + ((a.colour + cy) & 1);
        }
    }
    bool bad = false;
    const uint32_t e = zgbm_window<RL, false>(smem + (size_t)wib * smem_per_warp, R, a.geom,
                                              cell_at(R, a.geom, cx, cy), valid, a.colour, a.w, a.h, a.seed,
                                              a.src + R.lat_off, a.dst + R.lat_off, lane, &bad);
    if ((lane & (W - 1)) == 0 && valid) a.workload[R.cell_off + cy * R.ncx + cx] = (int32_t)e;
    zgbq_count<W>(a.counters, lane, valid, e, bad);
}

// Held to 64 registers with four cells per warp, to 72 with eight (as the
// one-window kernel).
template <int RL>
__global__ void __maxnreg__(RL == 8 ? 72 : 64) fs_zgbq_persistent_kernel(const __grid_constant__ PParams P,
                                                                    int smem_per_warp)
{
    constexpr int W = 32 / RL;
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int gl = lane & (W - 1);  // lane within the cell's group
    uint8_t *wsm = smem + (size_t)wib * smem_per_warp;
    const int per_window = P.total_active;
    const int chunks = (per_window + RL - 1) / RL;
    const unsigned long long total = (unsigned long long)P.nwin * (unsigned long long)chunks;
    for (;;) {
        // the dequeue and the abort flag in one round trip
        unsigned long long t = 0;
        int ab = 0;
        if (lane == 0) {
            t = atomicAdd(P.queue, 1ull);
            ab = *(volatile int32_t *)P.abort_flag;
        }
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= total || __shfl_sync(0xffffffffu, ab, 0)) break;
        const int i = (int)(t / (unsigned long long)chunks);
        const int u = RL * (int)(t % (unsigned long long)chunks) + lane / W;
        const bool valid = u < per_window;
        int r = 0, k = 0;
        if (valid) {
            const int2 rk = P.cell_rk[u];
            r = rk.x;
            k = rk.y;
        }
        const Replica &R = P.reps[r];
        const int64_t widx = P.colour_per_replica ? (int64_t)r * P.nwin + i : i;
        const int ccol = P.colour[widx];
        int cx = 0, cy = 0;
        if (valid) {
            if (P.order) {
                const int mo = P.order[R.cell_off + ccol * ((R.ncx >> 1) * R.ncy) + k];
                cy = mo / R.ncx;
                cx = mo - cy * R.ncx;
            } else {
                const int half = R.ncx >> 1;
                cy = k / half;
                cx = 2 * (k % half) + ((ccol + cy) & 1);
            }
        }
        const int slot = R.cell_off + cy * R.ncx + cx;
        // epoch[c] = 1 + the last window in which cell c was active.
        // Dependency 0: the cell's previous active window; 1..4: the edge
        // neighbours' last active window before this one; lane gl of a group
        // waits on dependencies gl, gl + W.
        {
            const int2 pv = P.prev[widx];
            bool ok = true;
#pragma unroll
            for (int d0 = 0; d0 < 5; d0 += W) {
                const int d = d0 + gl;
                const int ex = d == 1 ? 1 : (d == 3 ? -1 : 0);
                const int ey = d == 2 ? 1 : (d == 4 ? -1 : 0);
                const int dcx = (cx + ex + R.ncx) % R.ncx, dcy = (cy + ey + R.ncy) % R.ncy;
                const int target = (d == 0 ? pv.x : pv.y) + 1;
                const bool dep = valid && d < 5 && target > 0 && !(ey != 0 && R.ncy == 1);
                if (ok) ok = wait_epochs(P.epoch + R.cell_off, dcy * R.ncx + dcx, dep, target, P, lane);
            }
            if (!ok) break;
        }
        bool bad = false;
        const uint32_t e = zgbm_window<RL, true>(wsm, R, P.geom, cell_at(R, P.geom, cx, cy), valid, ccol,
                                                 P.w0 + (uint32_t)i, P.h[i], P.seed, P.lat + R.lat_off,
                                                 P.lat + R.lat_off, lane, &bad);
        if (gl == 0 && valid) P.workload[slot] = (int32_t)e;
        zgbq_count<W>(P.counters, lane, valid, e, bad);
        // the warp barrier orders every lane's writes before the release
        // stores of the groups' lane 0 (release is cumulative), which
        // publish them
        __syncwarp();
        if (gl == 0 && valid) {
            cuda::atomic_ref<int32_t, cuda::thread_scope_device> ea(P.epoch[slot]);
            ea.store(i + 1, cuda::memory_order_release);
        }
    }
}

}  // namespace

size_t zgb_multi_smem_per_warp(int rl)
{
    return (size_t)zgbm_warp_smem(rl);
}

bool zgb_multi_shape(int rl, int qx, int qy)
{
    return (rl == 4 || rl == 8) && zgbm_shape_ok(rl, qx, qy);
}

cudaError_t launch_zgb_multi_window(int rl, const WindowArgs &a, int nactive, int wpb, cudaStream_t st)
{
    const int groups = (nactive + rl - 1) / rl;
    const int blocks = (groups + wpb - 1) / wpb;
    if (blocks == 0) return cudaSuccess;
    const int spw = (int)zgb_multi_smem_per_warp(rl);
    const size_t smem = (size_t)spw * wpb;
    void (*kern)(WindowArgs, int, int) = rl == 8 ? fs_zgbq_window_kernel<8> : fs_zgbq_window_kernel<4>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<blocks, 32 * wpb, smem, st>>>(a, nactive, spw);
    return cudaGetLastError();
}

void *zgb_multi_persistent_kernel(int rl)
{
    return rl == 8 ? (void *)fs_zgbq_persistent_kernel<8> : (void *)fs_zgbq_persistent_kernel<4>;
}

}  // namespace fskmc
