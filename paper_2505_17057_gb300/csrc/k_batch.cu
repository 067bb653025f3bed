// k_batch.cu -- batched, persistent (grid-stride) MMFD step over many requests of one kernel
// class (lattice, PDE, levels, storage) with uneven grids packed into one launch.
#include "batch.h"
#include "k_direct.cuh"

namespace mmfd {

template <int LAT, int PDE, int LEVELS, int ST>
__global__ void __launch_bounds__(256) k_batch(const BatchItem* __restrict__ items, int nitems,
                                               long long total_tiles, int j) {
    using T = typename Storage<ST>::T;
    for (long long t = blockIdx.x; t < total_tiles; t += gridDim.x) {
        int lo = 0, hi = nitems - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (items[mid].tile0 <= t) lo = mid;
            else hi = mid - 1;
        }
        const BatchItem& it = items[lo];
        if (j >= it.steps_left) continue;
        const Geom g = it.g;
        const long long lt = t - it.tile0;
        const int bx = (int)(lt % it.tx);
        const int by = (int)((lt / it.tx) % it.ty);
        const int bz = (int)(lt / ((long long)it.tx * it.ty));
        const int x = bx * kBatchTileX + (int)(threadIdx.x % kBatchTileX);
        const int y = by * kBatchTileY + (int)(threadIdx.x / kBatchTileX);
        const int nl = it.nlev;
        const int c = (it.cur + j) % nl;
        const int prev = nl == 3 ? (c + 2) % 3 : c;
        const int next = nl == 2 ? 1 - c : (c + 1) % 3;
        StepExtra ex;
        ex.seed = it.seed;
        ex.step = it.step0 + j + 1;
        ex.sr = it.sr;
        if (x < g.nx && y < g.ny)
            direct_node<LAT, PDE, LEVELS, ST>(g, it.lev[c], it.lev[prev], it.lev[next],
                                              *static_cast<const Coef<T>*>(it.coef), ex, x, y, bz);
    }
}

template <int LAT, int PDE, int LEVELS, int ST>
cudaError_t launch_batch(const BatchItem* items, int nitems, long long total, int j, int grid, cudaStream_t s) {
    k_batch<LAT, PDE, LEVELS, ST><<<grid, kBatchTileX * kBatchTileY, 0, s>>>(items, nitems, total, j);
    return cudaGetLastError();
}

namespace {
template <int LAT, int PDE>
BatchFn pick_ls(int levels, int st) {
    if (levels == 2) {
        if (st == ST_F64) return launch_batch<LAT, PDE, 2, ST_F64>;
        if (st == ST_F32) return launch_batch<LAT, PDE, 2, ST_F32>;
        if (st == ST_BF16) return launch_batch<LAT, PDE, 2, ST_BF16>;
    } else if (levels == 3) {
        if (st == ST_F64) return launch_batch<LAT, PDE, 3, ST_F64>;
        if (st == ST_F32) return launch_batch<LAT, PDE, 3, ST_F32>;
        if (st == ST_BF16) return launch_batch<LAT, PDE, 3, ST_BF16>;
    }
    return nullptr;
}
}  // namespace

BatchFn find_batch(int lat, int pde, int levels, int st) {
    switch (lat) {
    case LAT_D2Q5: return pde == PDE_LCDE ? pick_ls<LAT_D2Q5, PDE_LCDE>(levels, st) : nullptr;
    case LAT_D3Q7: return pde == PDE_LCDE ? pick_ls<LAT_D3Q7, PDE_LCDE>(levels, st) : nullptr;
    case LAT_D2Q9:
        if (pde == PDE_LCDE) return pick_ls<LAT_D2Q9, PDE_LCDE>(levels, st);
        if (pde == PDE_NCDE) return pick_ls<LAT_D2Q9, PDE_NCDE>(levels, st);
        if (pde == PDE_NSE) return pick_ls<LAT_D2Q9, PDE_NSE>(levels, st);
        return nullptr;
    case LAT_D3Q19:
        if (pde == PDE_LCDE) return pick_ls<LAT_D3Q19, PDE_LCDE>(levels, st);
        if (pde == PDE_NCDE) return pick_ls<LAT_D3Q19, PDE_NCDE>(levels, st);
        if (pde == PDE_NSE) return pick_ls<LAT_D3Q19, PDE_NSE>(levels, st);
        return nullptr;
    }
    return nullptr;
}

}  // namespace mmfd
