// batch.h -- the batched multi-request step kernel used by the solve server.
#pragma once

#include <cuda_runtime.h>

#include "mmfd_internal.h"

namespace mmfd {

constexpr int kBatchTileX = 64;
constexpr int kBatchTileY = 4;

// One admitted request in a batched launch (device-resident table, one entry per request).
struct BatchItem {
    Geom g;
    void* lev[3];          // level buffers (ghosted layout)
    int nlev;              // 2 or 3
    int cur;               // buffer holding level t at the start of the tick
    long long steps_left;  // steps this request still needs at the start of the tick
    long long step0;       // steps done before the tick (stochastic-rounding counter)
    const void* coef;      // device copy of the request's Coef<T>
    long long tile0;       // first flat tile index of this request in the launch
    int tx, ty, tz;        // tiles along x, y, z
    int sr;                // stochastic rounding on
    unsigned long long seed;
};

// Advance every request in the table by step j of the tick (requests with steps_left <= j
// are skipped).  Grid-stride over the flat tile space; one node per thread.
using BatchFn = cudaError_t (*)(const BatchItem* items, int nitems, long long total_tiles, int j, int grid,
                                cudaStream_t s);
BatchFn find_batch(int lat, int pde, int levels, int st);

// All S steps of a tick for every request in the table in one persistent launch: a device-resident
// work queue of (step j, tile t) items, claimed in order through ctl[0]; a tile of step j > 0
// first waits (bounded, about a second) until every tile of its request's step j - 1 is done
// (ctl[2 + r] counts request r's finished tiles).  On a timeout the kernel sets ctl[1] (the other
// CTAs stop) and KERR_QUEUE_TIMEOUT in *err.  ctl holds 2 + nitems zeroed words per launch.
// stall_bias is added to every wait's target count: 0, or (for the failure-detection test) a
// count no tile reaches, so that every wait runs out.
constexpr int KERR_QUEUE_TIMEOUT = 2;   // device flag code (KERR_TMA_TIMEOUT is 1)
using QueueFn = cudaError_t (*)(const BatchItem* items, int nitems, long long total_tiles, int S, unsigned* ctl,
                                int* err, unsigned stall_bias, cudaStream_t s);
QueueFn find_batch_queue(int lat, int pde, int levels, int st);

inline long long batch_tiles(const Geom& g, int* tx, int* ty, int* tz) {
    *tx = (g.nx + kBatchTileX - 1) / kBatchTileX;
    *ty = (g.ny + kBatchTileY - 1) / kBatchTileY;
    *tz = g.nz;
    return (long long)(*tx) * (*ty) * (*tz);
}

}  // namespace mmfd
