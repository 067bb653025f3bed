// k_util.cu -- layout conversion (dense user arrays <-> ghosted storage) and deterministic
// FP64 reductions (sum, max |v|, non-finite count, GRE of Sec. IV and max-norm).
#include <cuda_bf16.h>

#include "kernels.h"
#include "stencil.cuh"

namespace mmfd {

namespace {

constexpr int kRedBlocks = 608;   // 4 x 152 SMs
constexpr int kRedThreads = 256;

template <int ST>
__device__ __forceinline__ double load_st(const void* base, long long i, double ref) {
    using Tr = Storage<ST>;
    return (double)Tr::load(static_cast<const typename Tr::S*>(base) + i, (typename Tr::T)ref);
}

// Layout kernels walk rows (blockIdx.y over y + z ny, grid-stride) and columns (threads), so no
// per-element division is needed; only edge nodes take the ghost-image path.
template <int ST>
__global__ void k_pack(Geom g, const void* __restrict__ src, int src_dtype, void* __restrict__ dst, double ref) {
    using Tr = Storage<ST>;
    using S = typename Tr::S;
    using T = typename Tr::T;
    S* d = static_cast<S*>(dst);
    const long long rows = (long long)g.ny * g.nz;
    for (long long r = blockIdx.y; r < rows; r += gridDim.y) {
        const int y = (int)(r % g.ny);
        const int z = (int)(r / g.ny);
        const long long base = r * g.nx;
        for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < g.nx; x += gridDim.x * blockDim.x) {
            const long long i = base + x;
            const double v = src_dtype == 0 ? static_cast<const double*>(src)[i] : (double)static_cast<const float*>(src)[i];
            const S sv = Tr::pack((T)v, (T)ref, 0u);
            const bool edge = x < g.gx || x >= g.nx - g.gx || y == 0 || y == g.ny - 1 ||
                              (g.dim == 3 && (z == 0 || z == g.nz - 1));
            if (!edge) {
                d[g.at(x, y, z)] = sv;
            } else if (g.dim == 3) {
                store_with_ghosts<3>(d, g, x, y, z, sv);
            } else {
                store_with_ghosts<2>(d, g, x, y, z, sv);
            }
        }
    }
}

template <int ST>
__global__ void k_unpack(Geom g, const void* __restrict__ src, double ref, void* __restrict__ dst, int dst_dtype) {
    const long long rows = (long long)g.ny * g.nz;
    for (long long r = blockIdx.y; r < rows; r += gridDim.y) {
        const int y = (int)(r % g.ny);
        const int z = (int)(r / g.ny);
        const long long base = r * g.nx;
        const long long sbase = g.at(0, y, z);
        for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < g.nx; x += gridDim.x * blockDim.x) {
            const double v = load_st<ST>(src, sbase + x, ref);
            if (dst_dtype == 0)
                static_cast<double*>(dst)[base + x] = v;
            else
                static_cast<float*>(dst)[base + x] = (float)v;
        }
    }
}

struct Acc4 {
    double a, b, c, d;
};

__device__ __forceinline__ Acc4 combine(int op, Acc4 x, Acc4 y) {
    if (op == 1) return {fmax(x.a, y.a), 0, 0, 0};
    if (op == 3) return {x.a + y.a, x.b + y.b, fmax(x.c, y.c), fmax(x.d, y.d)};
    return {x.a + y.a, 0, 0, 0};
}

// Fixed-order block reduction: block b covers rows b, b + nblocks, ... (row = y + z ny) and, in
// each row, columns threadIdx.x, + blockDim.x, ...; it reduces through shared memory in a fixed
// tree, so the result is bitwise reproducible.
template <int ST>
__global__ void __launch_bounds__(kRedThreads) k_reduce_parts(Geom g, const void* __restrict__ lev, double fref,
                                                              int op, const void* __restrict__ ref, int ref_dtype,
                                                              Acc4* __restrict__ parts) {
    __shared__ Acc4 sh[kRedThreads];
    const long long rows = (long long)g.ny * g.nz;
    Acc4 acc = {0, 0, 0, 0};
    const int cop = op == 2 ? 0 : op;
    for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
        const int y = (int)(r % g.ny);
        const int z = (int)(r / g.ny);
        const long long sbase = g.at(0, y, z);
        const long long dbase = r * g.nx;
        for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
            const double v = load_st<ST>(lev, sbase + x, fref);
            Acc4 e;
            if (op == 0) {
                e = {v, 0, 0, 0};
            } else if (op == 1) {
                e = {fabs(v), 0, 0, 0};
            } else if (op == 2) {
                e = {isfinite(v) ? 0.0 : 1.0, 0, 0, 0};
            } else {
                const long long i = dbase + x;
                const double rv = ref_dtype == 0 ? static_cast<const double*>(ref)[i] : (double)static_cast<const float*>(ref)[i];
                e = {fabs(v - rv), fabs(rv), fabs(v - rv), fabs(rv)};
                if (!isfinite(v)) e = {INFINITY, fabs(rv), INFINITY, fabs(rv)};
            }
            acc = combine(cop, acc, e);
        }
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kRedThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = combine(cop, sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) parts[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(kRedThreads) k_reduce_final(const Acc4* __restrict__ parts, int nparts, int op,
                                                              double* __restrict__ out) {
    __shared__ Acc4 sh[kRedThreads];
    Acc4 acc = {0, 0, 0, 0};
    const int cop = op == 2 ? 0 : op;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc = combine(cop, acc, parts[i]);
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kRedThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = combine(cop, sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sh[0].a;
        out[1] = sh[0].b;
        out[2] = sh[0].c;
        out[3] = sh[0].d;
    }
}

dim3 grid_rows(const Geom& g) {
    const long long rows = (long long)g.ny * g.nz;
    const int bx = (g.nx + 255) / 256 < 64 ? (g.nx + 255) / 256 : 64;
    const long long by = rows < 65535 ? rows : 65535;
    return dim3(bx, (unsigned)by, 1);
}

}  // namespace

cudaError_t launch_pack(const Geom& g, int st, const void* src, int src_dtype, void* dst_level, int field,
                        double ref, cudaStream_t s) {
    const dim3 blocks = grid_rows(g);
    char* dst = static_cast<char*>(dst_level) + (size_t)field * g.fs * g.es;
    if (st == ST_F64) k_pack<ST_F64><<<blocks, 256, 0, s>>>(g, src, src_dtype, dst, ref);
    else if (st == ST_F32) k_pack<ST_F32><<<blocks, 256, 0, s>>>(g, src, src_dtype, dst, ref);
    else k_pack<ST_BF16><<<blocks, 256, 0, s>>>(g, src, src_dtype, dst, ref);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const Geom& g, int st, const void* src_level, int field, double ref, void* dst,
                          int dst_dtype, cudaStream_t s) {
    const dim3 blocks = grid_rows(g);
    const char* src = static_cast<const char*>(src_level) + (size_t)field * g.fs * g.es;
    if (st == ST_F64) k_unpack<ST_F64><<<blocks, 256, 0, s>>>(g, src, ref, dst, dst_dtype);
    else if (st == ST_F32) k_unpack<ST_F32><<<blocks, 256, 0, s>>>(g, src, ref, dst, dst_dtype);
    else k_unpack<ST_BF16><<<blocks, 256, 0, s>>>(g, src, ref, dst, dst_dtype);
    return cudaGetLastError();
}

int reduce_parts_needed() { return kRedBlocks * 4; }  // doubles (Acc4 per block)

cudaError_t launch_reduce(const Geom& g, int st, const void* level, int field, double fref, int op,
                          const void* ref, int ref_dtype, double* d_partials, int nparts, double* d_out,
                          cudaStream_t s) {
    (void)nparts;
    const char* lev = static_cast<const char*>(level) + (size_t)field * g.fs * g.es;
    Acc4* parts = reinterpret_cast<Acc4*>(d_partials);
    if (st == ST_F64) k_reduce_parts<ST_F64><<<kRedBlocks, kRedThreads, 0, s>>>(g, lev, fref, op, ref, ref_dtype, parts);
    else if (st == ST_F32) k_reduce_parts<ST_F32><<<kRedBlocks, kRedThreads, 0, s>>>(g, lev, fref, op, ref, ref_dtype, parts);
    else k_reduce_parts<ST_BF16><<<kRedBlocks, kRedThreads, 0, s>>>(g, lev, fref, op, ref, ref_dtype, parts);
    k_reduce_final<<<1, kRedThreads, 0, s>>>(parts, kRedBlocks, op, d_out);
    return cudaGetLastError();
}

}  // namespace mmfd
