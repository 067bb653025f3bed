// k_batch.cu -- batched, persistent (grid-stride) MMFD step over many requests of one kernel
// class (lattice, PDE, levels, storage) with uneven grids packed into one launch.
#include "batch.h"
#include "k_direct.cuh"
#include "tma.cuh"

namespace mmfd {

// The request holding flat tile t (tables are ordered by tile0).
__device__ __forceinline__ int batch_item_of(const BatchItem* __restrict__ items, int nitems, long long t) {
    int lo = 0, hi = nitems - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].tile0 <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Step j of the tick for tile lt of request it: one node per thread.
template <int LAT, int PDE, int LEVELS, int ST>
__device__ __forceinline__ void batch_tile(const BatchItem& it, long long lt, int j) {
    using T = typename Storage<ST>::T;
    const Geom g = it.g;
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

template <int LAT, int PDE, int LEVELS, int ST>
__global__ void __launch_bounds__(256) k_batch(const BatchItem* __restrict__ items, int nitems,
                                               long long total_tiles, int j) {
    for (long long t = blockIdx.x; t < total_tiles; t += gridDim.x) {
        const BatchItem& it = items[batch_item_of(items, nitems, t)];
        if (j >= it.steps_left) continue;
        batch_tile<LAT, PDE, LEVELS, ST>(it, t - it.tile0, j);
    }
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// The device-resident work queue (batch.h).  Items q = j * total_tiles + t are claimed in
// increasing order, so every item a tile waits for (its request's step j - 1) was claimed
// earlier by a CTA that is running and waits only on still earlier items: the queue cannot
// deadlock, whatever number of CTAs is resident.  The producer side of a tile is the pattern of
// a grid barrier: the tile's stores, a CTA barrier, then one thread's fence and counter
// increment; the consumer side an acquire load of the counter by one thread, then a CTA barrier
// before any thread reads the level (the acquire also makes this SM's L1 drop stale lines).
template <int LAT, int PDE, int LEVELS, int ST>
__global__ void __launch_bounds__(256) k_batch_queue(const BatchItem* __restrict__ items, int nitems,
                                                     long long total_tiles, int S, unsigned* __restrict__ ctl,
                                                     int* __restrict__ err, unsigned stall_bias) {
    __shared__ int s_go, s_item, s_j;
    __shared__ long long s_lt;
    const long long nq = total_tiles * S;
    for (;;) {
        if (threadIdx.x == 0) {
            const long long q = (long long)atomicAdd(&ctl[0], 1u);
            int go = 0, r = 0, j = 0;
            long long lt = 0;
            if (q < nq && *reinterpret_cast<volatile unsigned*>(&ctl[1]) == 0u) {
                j = (int)(q / total_tiles);
                const long long t = q - (long long)j * total_tiles;
                r = batch_item_of(items, nitems, t);
                const BatchItem& it = items[r];
                lt = t - it.tile0;
                go = j >= it.steps_left ? 2 : 1;     // 2: the request is done, nothing to wait for
                if (go == 1 && j > 0) {
                    const unsigned need = (unsigned)((long long)it.tx * it.ty * it.tz * j) + stall_bias;
                    const long long t0 = clock64();
                    while (ld_acquire_gpu(&ctl[2 + r]) < need) {
                        if (*reinterpret_cast<volatile unsigned*>(&ctl[1]) != 0u || clock64() - t0 > kWaitBudgetCycles) {
                            atomicExch(&ctl[1], 1u);
                            atomicExch(err, KERR_QUEUE_TIMEOUT);
                            go = 0;
                            break;
                        }
                        __nanosleep(100);
                    }
                    __threadfence();
                }
            }
            s_go = go;
            s_item = r;
            s_j = j;
            s_lt = lt;
        }
        __syncthreads();
        const int go = s_go;
        if (go == 0) break;
        if (go == 1) batch_tile<LAT, PDE, LEVELS, ST>(items[s_item], s_lt, s_j);
        __syncthreads();   // the tile's stores are done (and thread 0 may overwrite the shared slots)
        if (go == 1 && threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&ctl[2 + s_item], 1u);
        }
    }
}

template <int LAT, int PDE, int LEVELS, int ST>
cudaError_t launch_batch_queue(const BatchItem* items, int nitems, long long total, int S, unsigned* ctl, int* err,
                               unsigned stall_bias, cudaStream_t s) {
    auto kern = k_batch_queue<LAT, PDE, LEVELS, ST>;
    static int resident = 0;
    if (resident == 0) {
        int per_sm = 0, dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0);
        if (e != cudaSuccess) return e;
        resident = (per_sm > 0 ? per_sm : 1) * sms;
    }
    const long long nq = total * S;
    const int grid = nq < resident ? (int)nq : resident;
    kern<<<grid, 256, 0, s>>>(items, nitems, total, S, ctl, err, stall_bias);
    return cudaGetLastError();
}

template <int LAT, int PDE, int LEVELS, int ST>
cudaError_t launch_batch(const BatchItem* items, int nitems, long long total, int j, int grid, cudaStream_t s) {
    k_batch<LAT, PDE, LEVELS, ST><<<grid, kBatchTileX * kBatchTileY, 0, s>>>(items, nitems, total, j);
    return cudaGetLastError();
}

namespace {
template <int LAT, int PDE>
QueueFn pick_q(int levels, int st) {
    if (levels == 2) {
        if (st == ST_F64) return launch_batch_queue<LAT, PDE, 2, ST_F64>;
        if (st == ST_F32) return launch_batch_queue<LAT, PDE, 2, ST_F32>;
        if (st == ST_BF16) return launch_batch_queue<LAT, PDE, 2, ST_BF16>;
    } else if (levels == 3) {
        if (st == ST_F64) return launch_batch_queue<LAT, PDE, 3, ST_F64>;
        if (st == ST_F32) return launch_batch_queue<LAT, PDE, 3, ST_F32>;
        if (st == ST_BF16) return launch_batch_queue<LAT, PDE, 3, ST_BF16>;
    }
    return nullptr;
}

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

QueueFn find_batch_queue(int lat, int pde, int levels, int st) {
    switch (lat) {
    case LAT_D2Q5: return pde == PDE_LCDE ? pick_q<LAT_D2Q5, PDE_LCDE>(levels, st) : nullptr;
    case LAT_D3Q7: return pde == PDE_LCDE ? pick_q<LAT_D3Q7, PDE_LCDE>(levels, st) : nullptr;
    case LAT_D2Q9:
        if (pde == PDE_LCDE) return pick_q<LAT_D2Q9, PDE_LCDE>(levels, st);
        if (pde == PDE_NCDE) return pick_q<LAT_D2Q9, PDE_NCDE>(levels, st);
        if (pde == PDE_NSE) return pick_q<LAT_D2Q9, PDE_NSE>(levels, st);
        return nullptr;
    case LAT_D3Q19:
        if (pde == PDE_LCDE) return pick_q<LAT_D3Q19, PDE_LCDE>(levels, st);
        if (pde == PDE_NCDE) return pick_q<LAT_D3Q19, PDE_NCDE>(levels, st);
        if (pde == PDE_NSE) return pick_q<LAT_D3Q19, PDE_NSE>(levels, st);
        return nullptr;
    }
    return nullptr;
}

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
