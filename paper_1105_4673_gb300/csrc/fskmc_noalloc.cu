// fskmc_observables_noalloc: the observables of a lattice that already sits
// in device memory, computed without allocating anything.
//
// Some callers cannot let a library allocate device memory: applications
// whose device memory is owned by their own pool (a framework's caching
// allocator, a pre-reserved arena in a long-running service) must not have
// cudaMalloc/cudaFree called behind their back, and a monitoring hook that
// reads the state after an out-of-memory error has no memory left to get.
// This entry point serves them: its integer accumulators live in a fixed,
// file-scope device array that every GPU loading the library holds until
// the process exits. Once the library's device code is loaded on a device
// (the first call there, under lazy module loading) a call allocates
// neither device nor host heap memory.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "fskmc.h"
#include "fskmc_internal.h"

namespace {

// Room for the observables kernel's accumulators: 3 state counts, the pair
// count and 2 * rmax correlation sums, rmax <= FSKMC_NOALLOC_MAX_RMAX.
constexpr int kMaxSlots = 4 + 2 * FSKMC_NOALLOC_MAX_RMAX;
static __device__ __align__(256) unsigned long long g_obs_scratch[kMaxSlots];

// Device address of the scratch array on the current device. Looked up on
// every call (cheap once the module is loaded, and no allocation), so a
// device reset or a re-created primary context never leaves a stale
// address; the host-side symbol itself is not a device address and is never
// handed to a kernel.
cudaError_t scratch_address(void **out)
{
    return cudaGetSymbolAddress(out, g_obs_scratch);
}

}  // namespace

extern "C" fskmc_status fskmc_observables_noalloc(const uint8_t *lattice, int32_t lx, int32_t ly,
                                                  fskmc_model model, void *stream,
                                                  double *coverage, double *energy,
                                                  double *paircorr, int32_t rmax)
{
    if (!lattice || !coverage || !energy) return FSKMC_EINVAL;
    if ((int)model < 0 || (int)model > 4) return FSKMC_EINVAL;
    if (lx < 1 || ly < 1 || lx > FSKMC_MAX_SIDE || ly > FSKMC_MAX_SIDE ||
        (int64_t)lx * ly > ((int64_t)1 << 31))
        return FSKMC_EINVAL;
    if (rmax < 0 || rmax > FSKMC_NOALLOC_MAX_RMAX || rmax > lx || (ly > 1 && rmax > ly))
        return FSKMC_EINVAL;
    if (rmax > 0 && !paircorr) return FSKMC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    void *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return FSKMC_ECUDA;
    unsigned long long *acc = static_cast<unsigned long long *>(scratch);
    const int n = 4 + 2 * rmax;
    // the array keeps the previous call's sums: clear the part this call uses
    if (cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * n, s) != cudaSuccess) return FSKMC_ECUDA;
    if (fskmc::launch_observables(lattice, lx, ly, rmax, acc, s) != cudaSuccess) return FSKMC_ECUDA;
    unsigned long long h[kMaxSlots];
    if (cudaMemcpyAsync(h, acc, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return FSKMC_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FSKMC_ECUDA;
    const double N = (double)lx * (double)ly;
    for (int k = 0; k < 3; ++k) coverage[k] = (double)h[k] / N;
    const double pairs = (double)h[3], n1 = (double)h[1];
    if ((int)model == fskmc::ZGB) *energy = NAN;
    else if ((int)model == fskmc::ISING) *energy = -(4.0 * pairs - 8.0 * n1 + 2.0 * N) / N;
    else *energy = -pairs / N;
    for (int r = 0; r < 2 * rmax; ++r) paircorr[r] = (double)h[4 + r] / N;
    return FSKMC_OK;
}
