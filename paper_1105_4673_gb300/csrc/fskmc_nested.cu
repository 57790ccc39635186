// Nested (two-level) fractional-step windows, Section 5 (Eq. sublatt2,
// Eq. opdecomp2), for the spin-flip models.
//
// The paper lays its two levels of decomposition onto the hardware of its
// time: super-cells onto GPUs, sub-cells onto threads. Here the two levels
// are the GB300's own: a super-cell is one thread block, its sub-cells are
// that block's warps. One launch runs one outer window (one super-cell
// colour C, length h) of one replica:
//   1. every block stages its super-cell and a one-site halo into shared
//      memory (the halo belongs to super-cells of the other colour, which
//      are frozen for the whole outer window);
//   2. it runs the inner schedule there -- n_in inner steps of Lie
//      (EE(d) EO(d)) or Strang (EE(d/2) EO(d) EE(d/2)), d = h/n_in -- where
//      in each inner window its warps run the sub-cells of one inner colour
//      (cell_window, staging from and writing back to the shared super-cell;
//      a warp takes the next sub-cell when it finishes one), with a block
//      barrier between inner windows;
//   3. it writes the super-cell back once.
// Same-colour sub-cells of one super-cell share no edge, and sub-cells of
// different super-cells of one colour meet at most at a corner, so for
// nearest-neighbour spin flips every inner window is exact (Eq. exact) and
// the result equals the oracle's orc_fs2_run bit for bit (binary64 clock):
// the same draws, keyed by the inner window index w_outer * ninner + j and
// the sub-cell's id in the global sub-cell grid.
#include <cuda_runtime.h>

#include "fskmc_cell.cuh"
#include "fskmc_internal.h"

namespace fskmc {

namespace {

template <int MODEL, typename CLK, bool PACKED>
__global__ void __launch_bounds__(512) fs_nested_kernel(NestedArgs a, int smem_per_warp)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const Replica &R = a.reps[a.rep_index];
    const int Qx = a.Qx, Qy = a.Qy, qx = a.geom.qx, qy = a.geom.qy;
    const int BW = Qx + 2, BH = Qy + 2;
    uint8_t *sup = smem;
    uint8_t *wsm = smem + a.super_bytes + (size_t)(threadIdx.x >> 5) * smem_per_warp;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

    // this block's super-cell: the g-th of colour C in row-major order
    const int nscx = R.lx / Qx;
    const int half = nscx >> 1;
    const int scy = blockIdx.x / half;
    const int scx = 2 * (blockIdx.x - scy * half) + ((a.colour + scy) & 1);
    const int X0 = scx * Qx, Y0 = scy * Qy;
    const int lx = R.lx, ly = R.ly;

    // 1. stage the super-cell and its halo (periodic wrap)
    {
        int by = 0, bx = threadIdx.x;
        while (bx >= BW) { bx -= BW; ++by; }
        for (int i = threadIdx.x; i < BW * BH; i += blockDim.x) {
            int gy = Y0 - 1 + by, gx = X0 - 1 + bx;
            gy += (gy < 0) ? ly : 0; gy -= (gy >= ly) ? ly : 0;
            gx += (gx < 0) ? lx : 0; gx -= (gx >= lx) ? lx : 0;
            if (PACKED) {
                const uint32_t *w32 = reinterpret_cast<const uint32_t *>(a.lat + R.lat_off) +
                                      (int64_t)gy * (lx >> 5) + (gx >> 5);
                sup[i] = (uint8_t)((*w32 >> (gx & 31)) & 1u);
            } else {
                sup[i] = a.lat[R.lat_off + (int64_t)gy * lx + gx];
            }
            bx += blockDim.x;
            while (bx >= BW) { bx -= BW; ++by; }
        }
    }
    __syncthreads();

    // 2. the inner windows
    const int rx = Qx / qx, ry = Qy / qy;  // sub-cells per super-cell side (even)
    const int per_row = rx >> 1;           // sub-cells of one inner colour per sub-cell row
    const int nact = per_row * ry;
    const int nsx = R.lx / qx;             // the global sub-cell grid
    for (int j = 0; j < a.ninner; ++j) {
        const int p = a.inner == 0 ? (j & 1) : j % 3;
        const int cin = a.inner == 0 ? p : (p == 1);
        const double len = (a.inner == 0 || p == 1) ? a.d : a.dhalf;
        for (int u = wib; u < nact; u += nwarps) {
            const int ly_ = u / per_row;
            const int lx_ = 2 * (u - ly_ * per_row) + ((cin + ly_) & 1);
            const int sx = scx * rx + lx_, sy = scy * ry + ly_;
            const uint32_t m = (uint32_t)(sy * nsx + sx);
            const CellAt at{1 + lx_ * qx, 1 + ly_ * qy, BW, BH, m};
            bool amb = false, bad = false;
            uint32_t nexact = 0;
            const uint32_t e = cell_window<MODEL, CLK, false, false>(
                wsm, R, a.geom, at, cin, a.w0 + (uint32_t)j, len, a.screen != 0, a.seed, sup, sup, lane,
                &amb, &bad, &nexact);
            if (lane == 0) {
                a.workload[R.cell_off + m] = (int32_t)e;
                atomicAdd(&a.counters[0], (unsigned long long)e);
                if (amb) atomicAdd(&a.counters[1], 1ull);
                if (bad) atomicAdd(&a.counters[3], 1ull);
                if (nexact) atomicAdd(&a.counters[4], (unsigned long long)nexact);
            }
            __syncwarp();
        }
        __syncthreads();
    }

    // 3. write the super-cell back
    if (PACKED) {
        // Qx is a multiple of 32: the super-cell's words are its own
        uint32_t *dst = reinterpret_cast<uint32_t *>(a.lat + R.lat_off);
        const int nwr = Qx >> 5;
        for (int t = threadIdx.x; t < Qy * nwr; t += blockDim.x) {
            const int row = t / nwr, wi = t - row * nwr;
            const uint8_t *b = sup + (row + 1) * BW + 1 + 32 * wi;
            uint32_t bits = 0u;
#pragma unroll 8
            for (int k = 0; k < 32; ++k) bits |= (uint32_t)(b[k] & 1u) << k;
            dst[(int64_t)(Y0 + row) * (lx >> 5) + (X0 >> 5) + wi] = bits;
        }
    } else {
        int row = 0, col = threadIdx.x;
        while (col >= Qx) { col -= Qx; ++row; }
        for (int i = threadIdx.x; i < Qx * Qy; i += blockDim.x) {
            a.lat[R.lat_off + (int64_t)(Y0 + row) * lx + X0 + col] = sup[(row + 1) * BW + 1 + col];
            col += blockDim.x;
            while (col >= Qx) { col -= Qx; ++row; }
        }
    }
}

template <int MODEL>
cudaError_t launch_nested_model(int fp32, const NestedArgs &a, int nsuper_active, int wpb,
                                cudaStream_t st)
{
    if (nsuper_active == 0) return cudaSuccess;
    void (*kern)(NestedArgs, int) = nullptr;
    if (a.packed) kern = fp32 ? fs_nested_kernel<MODEL, float, true> : fs_nested_kernel<MODEL, double, true>;
    else kern = fp32 ? fs_nested_kernel<MODEL, float, false> : fs_nested_kernel<MODEL, double, false>;
    const int spw = make_layout<MODEL>(a.geom.qx, a.geom.qy).bytes;
    const size_t smem = (size_t)a.super_bytes + (size_t)spw * wpb;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<nsuper_active, 32 * wpb, smem, st>>>(a, spw);
    return cudaGetLastError();
}

}  // namespace

size_t nested_smem(int model, int Qx, int Qy, int qx, int qy, int wpb)
{
    const size_t sup = (size_t)(((Qx + 2) * (Qy + 2) + 15) & ~15);
    switch (model) {
    case ADSDES: return sup + (size_t)make_layout<ADSDES>(qx, qy).bytes * wpb;
    case ISING: return sup + (size_t)make_layout<ISING>(qx, qy).bytes * wpb;
    }
    return 0;
}

cudaError_t launch_nested(int model, int fp32, const NestedArgs &a, int nsuper_active, int wpb,
                          cudaStream_t st)
{
    switch (model) {
    case ADSDES: return launch_nested_model<ADSDES>(fp32, a, nsuper_active, wpb, st);
    case ISING: return launch_nested_model<ISING>(fp32, a, nsuper_active, wpb, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fskmc
