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

inline long long batch_tiles(const Geom& g, int* tx, int* ty, int* tz) {
    *tx = (g.nx + kBatchTileX - 1) / kBatchTileX;
    *ty = (g.ny + kBatchTileY - 1) / kBatchTileY;
    *tz = g.nz;
    return (long long)(*tx) * (*ty) * (*tz);
}

}  // namespace mmfd
