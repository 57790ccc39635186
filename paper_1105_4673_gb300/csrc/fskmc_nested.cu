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
// the sub-cell's id in the global sub-cell grid. Sub-cells of at most 512
// sites run several to a warp (group_window, W lanes each), as in the
// one-level grouped kernels; larger ones one per warp (cell_window).
#include <cuda_runtime.h>

#include "fskmc_cell.cuh"
#include "fskmc_group.cuh"
#include "fskmc_internal.h"

namespace fskmc {

namespace {

// The block's super-cell: the g-th of colour C in row-major order.
struct SuperAt {
    int scx, scy, X0, Y0;
};

__device__ __forceinline__ SuperAt super_at(const Replica &R, const NestedArgs &a)
{
    const int half = (R.lx / a.Qx) >> 1;
    const int scy = blockIdx.x / half;
    const int scx = 2 * (blockIdx.x - scy * half) + ((a.colour + scy) & 1);
    return SuperAt{scx, scy, scx * a.Qx, scy * a.Qy};
}

// Stage the super-cell and its one-site halo (periodic wrap) into sup.
template <bool PACKED>
__device__ void stage_super(uint8_t *sup, const Replica &R, const NestedArgs &a, const SuperAt &S)
{
    const int BW = a.Qx + 2, BH = a.Qy + 2, lx = R.lx, ly = R.ly;
    int by = 0, bx = threadIdx.x;
    while (bx >= BW) { bx -= BW; ++by; }
    for (int i = threadIdx.x; i < BW * BH; i += blockDim.x) {
        int gy = S.Y0 - 1 + by, gx = S.X0 - 1 + bx;
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

// Write the super-cell (without its halo) back from sup.
template <bool PACKED>
__device__ void write_super(const uint8_t *sup, const Replica &R, const NestedArgs &a, const SuperAt &S)
{
    const int Qx = a.Qx, Qy = a.Qy, BW = Qx + 2, lx = R.lx;
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
            dst[(int64_t)(S.Y0 + row) * (lx >> 5) + (S.X0 >> 5) + wi] = bits;
        }
    } else {
        int row = 0, col = threadIdx.x;
        while (col >= Qx) { col -= Qx; ++row; }
        for (int i = threadIdx.x; i < Qx * Qy; i += blockDim.x) {
            a.lat[R.lat_off + (int64_t)(S.Y0 + row) * lx + S.X0 + col] = sup[(row + 1) * BW + 1 + col];
            col += blockDim.x;
            while (col >= Qx) { col -= Qx; ++row; }
        }
    }
}

// Inner window j: its sub-cell colour and length.
__device__ __forceinline__ void inner_window(const NestedArgs &a, int j, int &cin, double &len)
{
    const int p = a.inner == 0 ? (j & 1) : j % 3;
    cin = a.inner == 0 ? p : (p == 1);
    len = (a.inner == 0 || p == 1) ? a.d : a.dhalf;
}

// The u-th sub-cell of inner colour cin in the super-cell: its origin in
// the staged super-cell and its id in the global sub-cell grid.
__device__ __forceinline__ CellAt sub_at(const Replica &R, const NestedArgs &a, const SuperAt &S, int cin, int u)
{
    const int qx = a.geom.qx, qy = a.geom.qy, rx = a.Qx / qx, ry = a.Qy / qy;
    const int per_row = rx >> 1;
    const int ly_ = u / per_row;
    const int lx_ = 2 * (u - ly_ * per_row) + ((cin + ly_) & 1);
    const int sx = S.scx * rx + lx_, sy = S.scy * ry + ly_;
    return CellAt{1 + lx_ * qx, 1 + ly_ * qy, a.Qx + 2, a.Qy + 2, (uint32_t)(sy * (R.lx / qx) + sx)};
}

// One sub-cell per warp (cell_window).
template <int MODEL, typename CLK, bool PACKED>
__global__ void __launch_bounds__(512) fs_nested_kernel(NestedArgs a, int smem_per_warp)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const Replica &R = a.reps[a.rep_index];
    uint8_t *sup = smem;
    uint8_t *wsm = smem + a.super_bytes + (size_t)(threadIdx.x >> 5) * smem_per_warp;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const SuperAt S = super_at(R, a);
    stage_super<PACKED>(sup, R, a, S);
    __syncthreads();
    const int nact = (a.Qx / a.geom.qx) * (a.Qy / a.geom.qy) / 2;
    for (int j = 0; j < a.ninner; ++j) {
        int cin;
        double len;
        inner_window(a, j, cin, len);
        for (int u = wib; u < nact; u += nwarps) {
            const CellAt at = sub_at(R, a, S, cin, u);
            bool amb = false, bad = false;
            uint32_t nexact = 0;
            const uint32_t e = cell_window<MODEL, CLK, false, false>(
                wsm, R, a.geom, at, cin, a.w0 + (uint32_t)j, len, a.screen != 0, a.seed, sup, sup, lane,
                &amb, &bad, &nexact);
            if (lane == 0) {
                a.workload[R.cell_off + at.m] = (int32_t)e;
                atomicAdd(&a.counters[0], (unsigned long long)e);
                if (amb) atomicAdd(&a.counters[1], 1ull);
                if (bad) atomicAdd(&a.counters[3], 1ull);
                if (nexact) atomicAdd(&a.counters[4], (unsigned long long)nexact);
            }
            __syncwarp();
        }
        __syncthreads();
    }
    write_super<PACKED>(sup, R, a, S);
}

// GC = 32/W sub-cells per warp (group_window, W lanes each).
template <int MODEL, typename CLK, bool PACKED, int W>
__global__ void __launch_bounds__(512) fs_nested_group_kernel(NestedArgs a, int stride)
{
    constexpr int GC = 32 / W;
    extern __shared__ __align__(16) uint8_t smem[];
    const Replica &R = a.reps[a.rep_index];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    uint8_t *sup = smem;
    uint8_t *csm = smem + a.super_bytes + (size_t)(wib * GC + lane / W) * stride;
    const GLayout Lo = make_glayout<MODEL>(a.geom.qx, a.geom.qy, W);
    const SuperAt S = super_at(R, a);
    stage_super<PACKED>(sup, R, a, S);
    __syncthreads();
    const int nact = (a.Qx / a.geom.qx) * (a.Qy / a.geom.qy) / 2;
    for (int j = 0; j < a.ninner; ++j) {
        int cin;
        double len;
        inner_window(a, j, cin, len);
        for (int u0 = wib * GC; u0 < nact; u0 += nwarps * GC) {
            const int u = u0 + lane / W;
            const bool valid = u < nact;
            const CellAt at = sub_at(R, a, S, cin, valid ? u : u0);
            uint32_t ev, nexact;
            bool amb, bad;
            group_window<MODEL, CLK, false, false, W>(csm, Lo, R, a.geom, valid, at, a.w0 + (uint32_t)j, len,
                                                      a.screen != 0, a.seed, sup, sup, lane, &ev, &amb, &bad,
                                                      &nexact);
            if (valid && (lane & (W - 1)) == 0) a.workload[R.cell_off + at.m] = (int32_t)ev;
            add_counters<W>(a.counters, lane, valid, ev, amb, bad, nexact);
        }
        __syncthreads();
    }
    write_super<PACKED>(sup, R, a, S);
}

template <int MODEL>
cudaError_t launch_nested_model(int fp32, const NestedArgs &a, int nsuper_active, int wpb,
                                cudaStream_t st)
{
    if (nsuper_active == 0) return cudaSuccess;
    void (*kern)(NestedArgs, int) = nullptr;
    int arg;  // per-warp shared bytes (one sub-cell per warp) or per-group stride
    if (a.lanes == 8 || a.lanes == 16) {
        if (a.lanes == 8) {
            if (a.packed) kern = fp32 ? fs_nested_group_kernel<MODEL, float, true, 8> : fs_nested_group_kernel<MODEL, double, true, 8>;
            else kern = fp32 ? fs_nested_group_kernel<MODEL, float, false, 8> : fs_nested_group_kernel<MODEL, double, false, 8>;
        } else {
            if (a.packed) kern = fp32 ? fs_nested_group_kernel<MODEL, float, true, 16> : fs_nested_group_kernel<MODEL, double, true, 16>;
            else kern = fp32 ? fs_nested_group_kernel<MODEL, float, false, 16> : fs_nested_group_kernel<MODEL, double, false, 16>;
        }
        arg = make_glayout<MODEL>(a.geom.qx, a.geom.qy, a.lanes).stride;
    } else {
        if (a.packed) kern = fp32 ? fs_nested_kernel<MODEL, float, true> : fs_nested_kernel<MODEL, double, true>;
        else kern = fp32 ? fs_nested_kernel<MODEL, float, false> : fs_nested_kernel<MODEL, double, false>;
        arg = make_layout<MODEL>(a.geom.qx, a.geom.qy).bytes;
    }
    const size_t smem = nested_smem(MODEL, a.Qx, a.Qy, a.geom.qx, a.geom.qy, wpb, a.lanes);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<nsuper_active, 32 * wpb, smem, st>>>(a, arg);
    return cudaGetLastError();
}

}  // namespace

size_t nested_smem(int model, int Qx, int Qy, int qx, int qy, int wpb, int lanes)
{
    const size_t sup = (size_t)(((Qx + 2) * (Qy + 2) + 15) & ~15);
    const bool grouped = lanes == 8 || lanes == 16;
    switch (model) {
    case ADSDES:
        return sup + (size_t)wpb * (grouped ? (size_t)make_glayout<ADSDES>(qx, qy, lanes).stride * (32 / lanes)
                                            : (size_t)make_layout<ADSDES>(qx, qy).bytes);
    case ISING:
        return sup + (size_t)wpb * (grouped ? (size_t)make_glayout<ISING>(qx, qy, lanes).stride * (32 / lanes)
                                            : (size_t)make_layout<ISING>(qx, qy).bytes);
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
