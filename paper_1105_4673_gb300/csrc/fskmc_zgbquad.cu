// Kernels of the four-cells-per-warp ZGB window (fskmc_zgb32x4.cuh): 32-wide
// cells whose rows are a multiple of 4, from 8 to 32, with the binary32
// clock.
//
// fs_zgbq_window_kernel: one fractional window (Eqs. totalrate and skeleton
// on every active cell), warp g running the window's active cells 4g ..
// 4g + 3 (in issue order when one is given).
// fs_zgbq_persistent_kernel: the persistent engine of fskmc_window.cu for
// this window, a task being four consecutive active cells of one window;
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

// The events of the warp's four cells to counter 0 and their failures to
// counter 3 (lane 0; every lane calls it).
__device__ __forceinline__ void zgbq_count(unsigned long long *counters, int lane, bool valid, uint32_t e, bool bad)
{
    const uint32_t evs = __reduce_add_sync(0xffffffffu, (valid && (lane & 7) == 0) ? e : 0u);
    const unsigned bads = __ballot_sync(0xffffffffu, bad) & 0x01010101u;
    if (lane == 0) {
        atomicAdd(&counters[0], (unsigned long long)evs);
        if (bads) atomicAdd(&counters[3], (unsigned long long)__popc(bads));
    }
}

// Held to 64 registers (as the other one-window kernels).
__global__ void __launch_bounds__(512, 2) fs_zgbq_window_kernel(WindowArgs a, int nactive, int smem_per_warp)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int g = blockIdx.x * (blockDim.x >> 5) + wib;
    if (4 * g >= nactive) return;
    const int cidx = 4 * g + (lane >> 3);
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
    const uint32_t e = zgb32x4_window<false>(smem + (size_t)wib * smem_per_warp, R, a.geom,
                                             cell_at(R, a.geom, cx, cy), valid, a.colour, a.w, a.h, a.seed,
                                             a.src + R.lat_off, a.dst + R.lat_off, lane, &bad);
    if ((lane & 7) == 0 && valid) a.workload[R.cell_off + cy * R.ncx + cx] = (int32_t)e;
    zgbq_count(a.counters, lane, valid, e, bad);
}

// Held to 64 registers (four 256-thread blocks per SM).
__global__ void __launch_bounds__(256, 4) fs_zgbq_persistent_kernel(const __grid_constant__ PParams P,
                                                                    int smem_per_warp)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int gl = lane & 7;  // lane within the cell's group
    uint8_t *wsm = smem + (size_t)wib * smem_per_warp;
    const int per_window = P.total_active;
    const int chunks = (per_window + 3) >> 2;
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
        const int u = 4 * (int)(t % (unsigned long long)chunks) + (lane >> 3);
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
        // epoch[c] = 1 + the last window in which cell c was active. Lane 0
        // of a group: its cell's previous active window; lanes 1..4: the
        // edge neighbours' last active window before this one.
        {
            const int2 pv = P.prev[widx];
            const int ex = gl == 1 ? 1 : (gl == 3 ? -1 : 0);
            const int ey = gl == 2 ? 1 : (gl == 4 ? -1 : 0);
            const int dcx = (cx + ex + R.ncx) % R.ncx, dcy = (cy + ey + R.ncy) % R.ncy;
            const int target = (gl == 0 ? pv.x : pv.y) + 1;
            const bool dep = valid && gl < 5 && target > 0 && !(ey != 0 && R.ncy == 1);
            if (!wait_epochs(P.epoch + R.cell_off, dcy * R.ncx + dcx, dep, target, P, lane)) break;
        }
        bool bad = false;
        const uint32_t e = zgb32x4_window<true>(wsm, R, P.geom, cell_at(R, P.geom, cx, cy), valid, ccol,
                                                P.w0 + (uint32_t)i, P.h[i], P.seed, P.lat + R.lat_off,
                                                P.lat + R.lat_off, lane, &bad);
        if (gl == 0 && valid) P.workload[slot] = (int32_t)e;
        zgbq_count(P.counters, lane, valid, e, bad);
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

size_t zgb_quad_smem_per_warp()
{
    return (size_t)zgbq_warp_smem();
}

bool zgb_quad_shape(int qx, int qy)
{
    return zgbq_shape_ok(qx, qy);
}

cudaError_t launch_zgb_quad_window(const WindowArgs &a, int nactive, int wpb, cudaStream_t st)
{
    const int quads = (nactive + 3) / 4;
    const int blocks = (quads + wpb - 1) / wpb;
    if (blocks == 0) return cudaSuccess;
    const int spw = (int)zgb_quad_smem_per_warp();
    const size_t smem = (size_t)spw * wpb;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(fs_zgbq_window_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    fs_zgbq_window_kernel<<<blocks, 32 * wpb, smem, st>>>(a, nactive, spw);
    return cudaGetLastError();
}

void *zgb_quad_persistent_kernel()
{
    return (void *)fs_zgbq_persistent_kernel;
}

}  // namespace fskmc
