// Grouped window kernels (fskmc_group.cuh) instantiated for the binary32
// clock; split from the other clock so that the two compile in parallel.
#include "fskmc_group.cuh"

namespace fskmc {

namespace {

template <int MODEL, bool PACKED>
void *kernel_m(int W, bool persistent)
{
    using CLK = float;
    if constexpr (MODEL == ISING1D) {
        if (W == 4) return persistent ? (void *)fs_group_persistent_kernel<MODEL, CLK, PACKED, 4>
                                      : (void *)fs_group_kernel<MODEL, CLK, PACKED, 4>;
    }
    if (W == 8) return persistent ? (void *)fs_group_persistent_kernel<MODEL, CLK, PACKED, 8>
                                  : (void *)fs_group_kernel<MODEL, CLK, PACKED, 8>;
    if (W == 16) return persistent ? (void *)fs_group_persistent_kernel<MODEL, CLK, PACKED, 16>
                                   : (void *)fs_group_kernel<MODEL, CLK, PACKED, 16>;
    return nullptr;
}

template <int MODEL>
void *kernel_p(bool packed, int W, bool persistent)
{
    return packed ? kernel_m<MODEL, true>(W, persistent) : kernel_m<MODEL, false>(W, persistent);
}

}  // namespace

void *group_kernel_f32(int model, bool packed, int lanes, bool persistent)
{
    switch (model) {
    case ADSDES: return kernel_p<ADSDES>(packed, lanes, persistent);
    case ISING: return kernel_p<ISING>(packed, lanes, persistent);
    case ISING1D: return kernel_p<ISING1D>(packed, lanes, persistent);
    }
    return nullptr;
}

}  // namespace fskmc
