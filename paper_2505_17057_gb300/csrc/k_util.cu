// k_util.cu -- layout conversion (dense user arrays <-> ghosted storage) and deterministic
// FP64 reductions (sum, max |v|, non-finite count, GRE of Sec. IV and max-norm).
#include <cuda_bf16.h>

#include <type_traits>

#include "kernels.h"
#include "stencil.cuh"

namespace mmfd {

namespace {

constexpr int kRedBlocks = 608;   // 4 x 152 SMs
constexpr int kRedThreads = 256;

// Value of a stored element: the reference plus the stored offset, formed in FP64 so that an
// FP32 / BF16 offset comes back exactly (FP64 levels hold values, ref 0).
template <int ST>
__device__ __forceinline__ double load_st(const void* base, long long i, double ref) {
    using Tr = Storage<ST>;
    return ref + (double)Tr::raw(static_cast<const typename Tr::S*>(base) + i);
}

// Four consecutive values of a dense FP64 / FP32 source row, 16-byte aligned.
__device__ __forceinline__ void ld4_src(const void* src, int dtype, long long i, double v[4]) {
    if (dtype == 0) {
        const double2 a = *reinterpret_cast<const double2*>(static_cast<const double*>(src) + i);
        const double2 b = *reinterpret_cast<const double2*>(static_cast<const double*>(src) + i + 2);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    } else {
        const float4 a = *reinterpret_cast<const float4*>(static_cast<const float*>(src) + i);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    }
}

// Four consecutive stored values starting at a 16-byte aligned slot.
template <int ST>
__device__ __forceinline__ void ld4_st(const void* base, long long i, double ref, double v[4]) {
    using Tr = Storage<ST>;
    using S = typename Tr::S;
    const S* p = static_cast<const S*>(base) + i;
    if constexpr (ST == ST_F32) {
        // FP32 levels hold v - ref: the value is ref + stored, formed in FP64 (as load_st)
        const float4 a = *reinterpret_cast<const float4*>(p);
        v[0] = ref + (double)a.x; v[1] = ref + (double)a.y; v[2] = ref + (double)a.z; v[3] = ref + (double)a.w;
    } else if constexpr (ST == ST_F64) {
        const double2 a = *reinterpret_cast<const double2*>(p);
        const double2 b = *reinterpret_cast<const double2*>(p + 2);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = ref + (double)Tr::raw(p + k);
    }
}

// Vector pack: rows as in k_pack, four consecutive columns per thread (nx a multiple of 4 and a
// 16-byte aligned source); the source may be device memory or page-locked host memory read
// directly over the host link.  F32: an FP32 source into FP32 / BF16 storage with a reference
// that FP32 holds exactly; the offset is then formed in FP32, which rounds to the same value as
// the FP64 difference (the exact difference of two FP32 values fits in FP64 unless their
// exponents are more than 29 apart, and then both round to the larger operand).  FP64 runs at a
// sixtieth of the FP32 rate on this part, so the FP64 form made a 16.8M-value upload
// arithmetic-bound (94 against about 25 us at 4096^2).
template <int ST, bool F32 = false>
__global__ void k_pack4(Geom g, const void* __restrict__ src, int src_dtype, void* __restrict__ dst, double ref,
                        long long r_lo, long long r_hi) {
    using Tr = Storage<ST>;
    using S = typename Tr::S;
    using T = typename Tr::T;
    S* d = static_cast<S*>(dst);
    const int nq = g.nx >> 2;
    for (long long r = r_lo + blockIdx.y; r < r_hi; r += gridDim.y) {
        const int y = (int)(r % g.ny);
        const int z = (int)(r / g.ny);
        const bool yedge = y == 0 || y == g.ny - 1 || (g.dim == 3 && (z == 0 || z == g.nz - 1));
        for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
            const int x = q << 2;
            S sv[4];
            if constexpr (F32) {
                static_assert(ST != ST_F64, "FP64 storage keeps the FP64 path");
                const float4 a = *reinterpret_cast<const float4*>(static_cast<const float*>(src) + (r - r_lo) * g.nx + x);
                const float rf = (float)ref;
                sv[0] = Tr::pack_raw(a.x - rf, 0u);
                sv[1] = Tr::pack_raw(a.y - rf, 0u);
                sv[2] = Tr::pack_raw(a.z - rf, 0u);
                sv[3] = Tr::pack_raw(a.w - rf, 0u);
            } else {
                double v[4];
                ld4_src(src, src_dtype, (r - r_lo) * g.nx + x, v);
#pragma unroll
                for (int k = 0; k < 4; ++k) sv[k] = Tr::pack_raw((T)(v[k] - ref), 0u);   // offset formed in FP64
            }
            const bool edge = yedge || x < g.gx || x + 3 >= g.nx - g.gx;
            if (!edge) {
                S* p = d + g.at(x, y, z);
                if constexpr (ST == ST_F32) {
                    *reinterpret_cast<float4*>(p) = make_float4(sv[0], sv[1], sv[2], sv[3]);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) p[k] = sv[k];
                }
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (g.dim == 3) store_with_ghosts<3>(d, g, x + k, y, z, sv[k]);
                    else store_with_ghosts<2>(d, g, x + k, y, z, sv[k]);
                }
            }
        }
    }
}

// Layout kernels walk rows (blockIdx.y over y + z ny, grid-stride) and columns (threads), so no
// per-element division is needed; only edge nodes take the ghost-image path.
template <int ST>
__global__ void k_pack(Geom g, const void* __restrict__ src, int src_dtype, void* __restrict__ dst, double ref,
                       long long r_lo, long long r_hi) {
    using Tr = Storage<ST>;
    using S = typename Tr::S;
    using T = typename Tr::T;
    S* d = static_cast<S*>(dst);
    for (long long r = r_lo + blockIdx.y; r < r_hi; r += gridDim.y) {
        const int y = (int)(r % g.ny);
        const int z = (int)(r / g.ny);
        const long long base = (r - r_lo) * g.nx;
        for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < g.nx; x += gridDim.x * blockDim.x) {
            const long long i = base + x;
            const double v = src_dtype == 0 ? static_cast<const double*>(src)[i] : (double)static_cast<const float*>(src)[i];
            const S sv = Tr::pack_raw((T)(v - ref), 0u);   // offset formed in FP64, rounded once
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
__global__ void k_unpack(Geom g, const void* __restrict__ src, double ref, void* __restrict__ dst, int dst_dtype,
                         long long r_lo, long long r_hi) {
    for (long long r = r_lo + blockIdx.y; r < r_hi; r += gridDim.y) {
        const int y = (int)(r % g.ny);
        const int z = (int)(r / g.ny);
        const long long base = (r - r_lo) * g.nx;
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

// Rows [r_lo, r_hi) (r = y + z ny) of every field of a level to / from dense buffers in one launch
// (blockIdx.z = field): the halo-row exchange of a slab decomposition moves a few rows per step,
// so the launch count matters more than the bandwidth.
struct RowBufs {
    const void* src[4];
    void* dst[4];
    double ref[4];
};

template <int ST>
__global__ void k_rows_pack(Geom g, RowBufs b, int src_dtype, void* __restrict__ level, long long r_lo, long long r_hi) {
    using Tr = Storage<ST>;
    using S = typename Tr::S;
    using T = typename Tr::T;
    const int f = blockIdx.z;
    S* d = static_cast<S*>(level) + (size_t)f * g.fs;
    const double ref = b.ref[f];
    for (long long r = r_lo + blockIdx.y; r < r_hi; r += gridDim.y) {
        const int y = (int)(r % g.ny);
        const int z = (int)(r / g.ny);
        const long long base = (r - r_lo) * g.nx;
        for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < g.nx; x += gridDim.x * blockDim.x) {
            const long long i = base + x;
            const double v = src_dtype == 0 ? static_cast<const double*>(b.src[f])[i] : (double)static_cast<const float*>(b.src[f])[i];
            const S sv = Tr::pack_raw((T)(v - ref), 0u);
            if (g.dim == 3) store_with_ghosts<3>(d, g, x, y, z, sv);
            else store_with_ghosts<2>(d, g, x, y, z, sv);
        }
    }
}

template <int ST>
__global__ void k_rows_unpack(Geom g, RowBufs b, int dst_dtype, const void* __restrict__ level, long long r_lo,
                              long long r_hi) {
    const int f = blockIdx.z;
    const char* src = static_cast<const char*>(level) + (size_t)f * g.fs * g.es;
    const double ref = b.ref[f];
    for (long long r = r_lo + blockIdx.y; r < r_hi; r += gridDim.y) {
        const int y = (int)(r % g.ny);
        const int z = (int)(r / g.ny);
        const long long base = (r - r_lo) * g.nx;
        const long long sbase = g.at(0, y, z);
        for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < g.nx; x += gridDim.x * blockDim.x) {
            const double v = load_st<ST>(src, sbase + x, ref);
            if (dst_dtype == 0)
                static_cast<double*>(b.dst[f])[base + x] = v;
            else
                static_cast<float*>(b.dst[f])[base + x] = (float)v;
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
// The operation is a template parameter (0 sum, 1 max |v|, 2 non-finite count, 3 error norms):
// with a run-time switch in the element loop every element paid for all four accumulators.
template <int ST, int OPT>
__global__ void __launch_bounds__(kRedThreads) k_reduce_parts(Geom g, const void* __restrict__ lev, double fref,
                                                              const void* __restrict__ ref, int ref_dtype,
                                                              Acc4* __restrict__ parts) {
    constexpr int op = OPT;
    __shared__ Acc4 sh[kRedThreads];
    const long long rows = (long long)g.ny * g.nz;
    Acc4 acc = {0, 0, 0, 0};
    constexpr int cop = op == 2 ? 0 : op;
    const bool vec = OPT != 3 && (g.nx & 3) == 0;
    for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
        const int y = (int)(r % g.ny);
        const int z = (int)(r / g.ny);
        const long long sbase = g.at(0, y, z);
        const long long dbase = r * g.nx;
        if (vec) {
            // four columns per thread per pass (the row starts on a 16-byte boundary)
            for (int x = threadIdx.x << 2; x < g.nx; x += blockDim.x << 2) {
                double v[4];
                ld4_st<ST>(lev, sbase + x, fref, v);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if constexpr (OPT == 0) acc.a += v[k];
                    else if constexpr (OPT == 1) acc.a = fmax(acc.a, fabs(v[k]));
                    else if constexpr (OPT == 2) acc.a += isfinite(v[k]) ? 0.0 : 1.0;
                }
            }
            continue;
        }
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

namespace {

// The boundary ring of a grid (nodes with x = 0 / nx - 1, y = 0 / ny - 1, and z = 0 / nz - 1 in
// 3D), enumerated face by face without repeats: in 3D the two z faces whole, then the two y faces
// between them, then the two x faces between those; in 2D the y faces and then the x faces.
__host__ __device__ inline long long ring_nodes(const Geom& g) {
    const long long zn = g.dim == 3 ? g.nz - 2 : 1;
    return (g.dim == 3 ? 2ll * g.nx * g.ny : 0ll) + 2ll * g.nx * zn + 2ll * (g.ny - 2) * zn;
}

template <typename E>
__global__ void k_ring_copy(Geom g, const E* __restrict__ src, E* __restrict__ dst, long long count) {
    const long long zn = g.dim == 3 ? g.nz - 2 : 1;
    const int z0 = g.dim == 3 ? 1 : 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        long long k = i;
        int x, y, z;
        const long long zface = g.dim == 3 ? (long long)g.nx * g.ny : 0;
        const long long yface = (long long)g.nx * zn;
        const long long xface = (long long)(g.ny - 2) * zn;
        if (k < 2 * zface) {
            z = k < zface ? 0 : g.nz - 1;
            const long long r = k % zface;
            x = (int)(r % g.nx);
            y = (int)(r / g.nx);
        } else if ((k -= 2 * zface) < 2 * yface) {
            y = k < yface ? 0 : g.ny - 1;
            const long long r = k % yface;
            x = (int)(r % g.nx);
            z = z0 + (int)(r / g.nx);
        } else {
            k -= 2 * yface;
            x = k < xface ? 0 : g.nx - 1;
            const long long r = k % xface;
            y = 1 + (int)(r % (g.ny - 2));
            z = z0 + (int)(r / (g.ny - 2));
        }
        const long long at = g.at(x, y, z);
        for (int f = 0; f < g.nf; ++f) dst[(long long)f * g.fs + at] = src[(long long)f * g.fs + at];
    }
}

}  // namespace

cudaError_t launch_ring_copy(const Geom& g, const void* src_level, void* dst_level, cudaStream_t s) {
    const long long count = ring_nodes(g);
    if (count <= 0) return cudaSuccess;
    const int blocks = (int)((count + 255) / 256 < 1184 ? (count + 255) / 256 : 1184);
    if (g.es == 8) k_ring_copy<unsigned long long><<<blocks, 256, 0, s>>>(g, static_cast<const unsigned long long*>(src_level), static_cast<unsigned long long*>(dst_level), count);
    else if (g.es == 4) k_ring_copy<unsigned int><<<blocks, 256, 0, s>>>(g, static_cast<const unsigned int*>(src_level), static_cast<unsigned int*>(dst_level), count);
    else k_ring_copy<unsigned short><<<blocks, 256, 0, s>>>(g, static_cast<const unsigned short*>(src_level), static_cast<unsigned short*>(dst_level), count);
    return cudaGetLastError();
}

cudaError_t launch_pack(const Geom& g, int st, const void* src, int src_dtype, void* dst_level, int field,
                        double ref, cudaStream_t s, long long r_lo, long long r_hi) {
    if (r_hi < 0) r_hi = (long long)g.ny * g.nz;
    if (r_hi <= r_lo) return cudaSuccess;
    dim3 blocks = grid_rows(g);
    if ((long long)blocks.y > r_hi - r_lo) blocks.y = (unsigned)(r_hi - r_lo);
    char* dst = static_cast<char*>(dst_level) + (size_t)field * g.fs * g.es;
    if ((g.nx & 3) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0 && g.nx >= 8) {
        const dim3 b4((unsigned)((g.nx / 4 + 255) / 256 < 64 ? (g.nx / 4 + 255) / 256 : 64), blocks.y, 1);
        const bool f32 = src_dtype == 1 && (double)(float)ref == ref;   // 1: FP32 (MMFD_DT_F32)
        if (st == ST_F64) k_pack4<ST_F64><<<b4, 256, 0, s>>>(g, src, src_dtype, dst, ref, r_lo, r_hi);
        else if (st == ST_F32 && f32) k_pack4<ST_F32, true><<<b4, 256, 0, s>>>(g, src, src_dtype, dst, ref, r_lo, r_hi);
        else if (st == ST_F32) k_pack4<ST_F32><<<b4, 256, 0, s>>>(g, src, src_dtype, dst, ref, r_lo, r_hi);
        else if (f32) k_pack4<ST_BF16, true><<<b4, 256, 0, s>>>(g, src, src_dtype, dst, ref, r_lo, r_hi);
        else k_pack4<ST_BF16><<<b4, 256, 0, s>>>(g, src, src_dtype, dst, ref, r_lo, r_hi);
        return cudaGetLastError();
    }
    if (st == ST_F64) k_pack<ST_F64><<<blocks, 256, 0, s>>>(g, src, src_dtype, dst, ref, r_lo, r_hi);
    else if (st == ST_F32) k_pack<ST_F32><<<blocks, 256, 0, s>>>(g, src, src_dtype, dst, ref, r_lo, r_hi);
    else k_pack<ST_BF16><<<blocks, 256, 0, s>>>(g, src, src_dtype, dst, ref, r_lo, r_hi);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const Geom& g, int st, const void* src_level, int field, double ref, void* dst,
                          int dst_dtype, cudaStream_t s, long long r_lo, long long r_hi) {
    if (r_hi < 0) r_hi = (long long)g.ny * g.nz;
    if (r_hi <= r_lo) return cudaSuccess;
    dim3 blocks = grid_rows(g);
    if ((long long)blocks.y > r_hi - r_lo) blocks.y = (unsigned)(r_hi - r_lo);
    const char* src = static_cast<const char*>(src_level) + (size_t)field * g.fs * g.es;
    if (st == ST_F64) k_unpack<ST_F64><<<blocks, 256, 0, s>>>(g, src, ref, dst, dst_dtype, r_lo, r_hi);
    else if (st == ST_F32) k_unpack<ST_F32><<<blocks, 256, 0, s>>>(g, src, ref, dst, dst_dtype, r_lo, r_hi);
    else k_unpack<ST_BF16><<<blocks, 256, 0, s>>>(g, src, ref, dst, dst_dtype, r_lo, r_hi);
    return cudaGetLastError();
}

cudaError_t launch_rows(const Geom& g, int st, bool pack, const void* const* bufs, int nf, int dtype, void* level,
                        const double* refs, long long r_lo, long long r_hi, cudaStream_t s) {
    if (nf < 1 || nf > 4) return cudaErrorInvalidValue;
    if (r_hi <= r_lo) return cudaSuccess;
    RowBufs b{};
    for (int f = 0; f < nf; ++f) {
        if (pack) b.src[f] = bufs[f];
        else b.dst[f] = const_cast<void*>(bufs[f]);
        b.ref[f] = refs[f];
    }
    const long long rows = r_hi - r_lo;
    const dim3 blocks((unsigned)((g.nx + 255) / 256 < 64 ? (g.nx + 255) / 256 : 64),
                      (unsigned)(rows < 65535 ? rows : 65535), (unsigned)nf);
    if (pack) {
        if (st == ST_F64) k_rows_pack<ST_F64><<<blocks, 256, 0, s>>>(g, b, dtype, level, r_lo, r_hi);
        else if (st == ST_F32) k_rows_pack<ST_F32><<<blocks, 256, 0, s>>>(g, b, dtype, level, r_lo, r_hi);
        else k_rows_pack<ST_BF16><<<blocks, 256, 0, s>>>(g, b, dtype, level, r_lo, r_hi);
    } else {
        if (st == ST_F64) k_rows_unpack<ST_F64><<<blocks, 256, 0, s>>>(g, b, dtype, level, r_lo, r_hi);
        else if (st == ST_F32) k_rows_unpack<ST_F32><<<blocks, 256, 0, s>>>(g, b, dtype, level, r_lo, r_hi);
        else k_rows_unpack<ST_BF16><<<blocks, 256, 0, s>>>(g, b, dtype, level, r_lo, r_hi);
    }
    return cudaGetLastError();
}

int reduce_parts_needed() { return kRedBlocks * 4; }  // doubles (Acc4 per block)

cudaError_t launch_reduce(const Geom& g, int st, const void* level, int field, double fref, int op,
                          const void* ref, int ref_dtype, double* d_partials, int nparts, double* d_out,
                          cudaStream_t s) {
    (void)nparts;
    const char* lev = static_cast<const char*>(level) + (size_t)field * g.fs * g.es;
    Acc4* parts = reinterpret_cast<Acc4*>(d_partials);
    auto parts_kernel = [&](auto stc) -> void {
        constexpr int SC = decltype(stc)::value;
        switch (op) {
            case 0: k_reduce_parts<SC, 0><<<kRedBlocks, kRedThreads, 0, s>>>(g, lev, fref, ref, ref_dtype, parts); break;
            case 1: k_reduce_parts<SC, 1><<<kRedBlocks, kRedThreads, 0, s>>>(g, lev, fref, ref, ref_dtype, parts); break;
            case 2: k_reduce_parts<SC, 2><<<kRedBlocks, kRedThreads, 0, s>>>(g, lev, fref, ref, ref_dtype, parts); break;
            default: k_reduce_parts<SC, 3><<<kRedBlocks, kRedThreads, 0, s>>>(g, lev, fref, ref, ref_dtype, parts); break;
        }
    };
    if (st == ST_F64) parts_kernel(std::integral_constant<int, ST_F64>{});
    else if (st == ST_F32) parts_kernel(std::integral_constant<int, ST_F32>{});
    else parts_kernel(std::integral_constant<int, ST_BF16>{});
    k_reduce_final<<<1, kRedThreads, 0, s>>>(parts, kRedBlocks, op, d_out);
    return cudaGetLastError();
}

}  // namespace mmfd
