// Host side of the grouped window kernels (fskmc_group.cuh; instantiated in
// fskmc_group_f64.cu and fskmc_group_f32.cu): widths, shared-memory sizes,
// kernel choice and the plain engine's launch.
#include <cuda_runtime.h>

#include "fskmc_group.cuh"

namespace fskmc {

namespace {

int group_stride(int model, int qx, int qy, int W)
{
    switch (model) {
    case ADSDES: return make_glayout<ADSDES>(qx, qy, W).stride;
    case ISING: return make_glayout<ISING>(qx, qy, W).stride;
    case ISING1D: return make_glayout<ISING1D>(qx, qy, W).stride;
    }
    return 0;
}

}  // namespace

int group_width(int model, int qx, int qy)
{
    if (model != ADSDES && model != ISING && model != ISING1D) return 32;
    const int nl = (qx * qy + 31) / 32;
    int w = model == ISING1D ? 4 : 8;
    while (w < nl) w <<= 1;
    return w;
}

size_t group_smem_per_warp(int model, int qx, int qy)
{
    const int W = group_width(model, qx, qy);
    if (W >= 32) return 0;
    return (size_t)group_stride(model, qx, qy, W) * (size_t)(32 / W);
}

void *group_kernel_for(int model, int fp32, bool packed, int qx, int qy, bool persistent)
{
    const int W = group_width(model, qx, qy);
    if (W >= 32) return nullptr;
    return fp32 ? group_kernel_f32(model, packed, W, persistent) : group_kernel_f64(model, packed, W, persistent);
}

cudaError_t launch_group_window(int model, int fp32, const WindowArgs &a, int nactive, int wpb,
                                cudaStream_t st)
{
    void *kern = group_kernel_for(model, fp32, a.packed != 0, a.geom.qx, a.geom.qy, false);
    if (!kern) return cudaErrorInvalidValue;
    wpb = wpb < 8 ? wpb : 8;  // the grouped kernels are built for up to 256 threads per block
    const int W = group_width(model, a.geom.qx, a.geom.qy);
    const int cells_per_warp = 32 / W;
    const int stride = group_stride(model, a.geom.qx, a.geom.qy, W);
    const size_t smem = (size_t)stride * cells_per_warp * wpb;
    const int nwarps = (nactive + cells_per_warp - 1) / cells_per_warp;
    const int blocks = (nwarps + wpb - 1) / wpb;
    if (blocks == 0) return cudaSuccess;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    void *args[] = {(void *)&a, (void *)&nactive, (void *)&stride};
    return cudaLaunchKernel(kern, dim3(blocks), dim3(32 * wpb), args, smem, st);
}

}  // namespace fskmc
