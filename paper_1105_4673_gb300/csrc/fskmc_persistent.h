// Persistent engine: one launch runs every window of every replica.
#pragma once
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "fskmc_internal.h"

namespace fskmc {

// Everything one persistent run needs (host-side view).
struct PersistentRun {
    int model, fp32, qx, qy, nrep, wpb;
    const Replica *reps_host;
    const Replica *reps_dev;
    uint8_t *lat;                 // state at run start (all replicas)
    uint8_t *lat2;                // ping-pong partner (diffusion) or nullptr
    int32_t *workload;
    unsigned long long *counters;
    int32_t total_cells;
    const int8_t *colour;         // [nwin] or [nrep * nwin] when colour_per_replica
    bool colour_per_replica;
    const double *h;              // [nwin]
    int64_t nwin;
    uint64_t w0, seed;
    uint32_t spin_limit;          // polls before a wait gives up
    bool packed;                  // bit-packed lattice (spin-flip models)
    const int32_t *order;         // device: active cells per replica and colour, heaviest
                                  // first (see launch_order), or null for row-major order
    int lanes_per_cell;           // 32, or the width of the grouped kernel (spin-flip models)
    bool screen;                  // binary64 clock: screened window-edge decisions
};

struct PersistentState;  // device buffers and the captured CUDA graph

// Queue the run on the stream and wait for it; returns cudaErrorTimeout
// (with *msg set) if a bounded wait gave up.
cudaError_t persistent_run(PersistentState **st, const PersistentRun &run, cudaStream_t s,
                           std::string *msg);
void persistent_free(PersistentState *st);

}  // namespace fskmc
