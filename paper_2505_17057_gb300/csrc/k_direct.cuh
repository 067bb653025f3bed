// k_direct.cuh -- one node per thread MMFD update (any grid shape, any lattice/PDE).
// Neighbours are read straight from the ghosted layout through the L1/L2 caches; every
// output is written to its interior slot and its periodic ghost images.
#pragma once

#include <type_traits>

#include "kernels.h"
#include "stencil.cuh"

namespace mmfd {

template <int P, int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (P < N) {
        f(std::integral_constant<int, P>{});
        static_for<P + 1, N>(f);
    }
}

// Source term of level l at node c0 (weights folded on the host, see SrcCoef): SRC 1 reads S
// only (M_1F = 0 or S u), SRC 2 also the M_1F components.  Source levels are read-only for
// the whole launch, so they go through the read-only data path.
template <int LAT, int SRC, typename T>
__device__ __forceinline__ T source_level(const Geom& g, const T* __restrict__ src, const SrcCoef<T>& w, int l,
                                          long long c0) {
    constexpr int NP = lat_npair(LAT);
    constexpr int D = lat_dim(LAT);
    T acc = w.W0[l] * __ldg(src + c0);
    static_for<0, NP>([&](auto pc) {
        constexpr int P = decltype(pc)::value;
        const long long off = pair_offset<LAT>(g, P);
        acc += w.Wp[l][P] * __ldg(src + c0 + off) + w.Wm[l][P] * __ldg(src + c0 - off);
        if constexpr (SRC == 2) {
#pragma unroll
            for (int a = 0; a < D; ++a)
                if (pair_e(LAT, P, a) != 0) {
                    const T* m = src + (long long)(1 + a) * g.fs;
                    acc += w.M[l][P][a] * (__ldg(m + c0 + off) - __ldg(m + c0 - off));
                }
        }
    });
    return acc;
}

// The update of one node (x, y, z): reads levels t (in0) and t - dt (in1) in the ghosted
// layout, writes level t + dt (out) and its periodic ghost images.  Shared by the one-solve
// kernel below and the batched multi-request kernel, so a request computes the same bits
// alone and inside a batch.
// With SRC != 0 the source terms of `sa` are added before the store.
template <int LAT, int PDE, int LEVELS, int ST, int SRC = 0>
__device__ __forceinline__ void direct_node(const Geom& g, const void* __restrict__ in0v,
                                            const void* __restrict__ in1v, void* __restrict__ outv,
                                            const Coef<typename Storage<ST>::T>& cf, const StepExtra& ex,
                                            int x, int y, int z,
                                            const SrcArgs<typename Storage<ST>::T>* sa = nullptr) {
    using Tr = Storage<ST>;
    using S = typename Tr::S;
    using T = typename Tr::T;
    constexpr int D = lat_dim(LAT);
    constexpr int NP = lat_npair(LAT);
    constexpr int NF = pde_nf(PDE, LAT);
    const long long c0 = g.at(x, y, z);
    T acc[NF];
#pragma unroll
    for (int i = 0; i < NF; ++i) acc[i] = T(0);

#pragma unroll
    for (int l = 0; l < LEVELS - 1; ++l) {
        const S* in = static_cast<const S*>(l == 0 ? in0v : in1v);
        if constexpr (PDE == PDE_LCDE) {
            // f_j^eq = phi ubar_j (Eq. (TforMMFD-0)): the update is a fixed linear stencil.
            T s = cf.W0[l] * kload<ST, PDE>(in + c0, cf.ref[0]);
            static_for<0, NP>([&](auto pc) {
                constexpr int P = decltype(pc)::value;
                const long long off = pair_offset<LAT>(g, P);
                s += cf.Wp[l][P] * kload<ST, PDE>(in + c0 + off, cf.ref[0]) + cf.Wm[l][P] * kload<ST, PDE>(in + c0 - off, cf.ref[0]);
            });
            acc[0] += s;
        } else {
            T f[NF];
#pragma unroll
            for (int i = 0; i < NF; ++i) f[i] = kload<ST, PDE>(in + i * g.fs + c0, cf.ref[i]);
            Basis<LAT, PDE, T> b0;
            b0.init(f, cf);
            acc[0] += cf.a0[l] * b0.A() + cf.ap[l] * b0.rest(cf);
            if constexpr (PDE == PDE_NSE) {
#pragma unroll
                for (int a = 0; a < D; ++a) acc[1 + a] += cf.ab0[l] * b0.mom(a);
            }
            static_for<0, NP>([&](auto pc) {
                constexpr int P = decltype(pc)::value;
                const long long off = pair_offset<LAT>(g, P);
                T fp[NF], fm[NF];
#pragma unroll
                for (int i = 0; i < NF; ++i) {
                    fp[i] = kload<ST, PDE>(in + i * g.fs + c0 + off, cf.ref[i]);
                    fm[i] = kload<ST, PDE>(in + i * g.fs + c0 - off, cf.ref[i]);
                }
                Basis<LAT, PDE, T> bp, bm;
                bp.init(fp, cf);
                bm.init(fm, cf);
                T Ep, Op, Em, Om;
                bp.template eo<P>(cf, Ep, Op);
                bm.template eo<P>(cf, Em, Om);
                acc[0] += cf.ap[l] * (Ep + Em) + cf.am[l] * (Op - Om);
                if constexpr (PDE == PDE_NSE) {
                    const T dm = cf.abm[l] * (Ep - Em) + cf.abp[l] * (Op + Om);
#pragma unroll
                    for (int a = 0; a < D; ++a)
                        if (pair_e(LAT, P, a) != 0) acc[1 + a] += T(pair_e(LAT, P, a)) * cf.fmom[a] * dm;
                }
            });
        }
    }
    if constexpr (SRC != 0) {
#pragma unroll
        for (int l = 0; l < LEVELS - 1; ++l) acc[0] += source_level<LAT, SRC, T>(g, sa->s[l], sa->w, l, c0);
    }
    S* out = static_cast<S*>(outv);
    const long long node = ((long long)z * g.ny + y) * g.nx + x;
#pragma unroll
    for (int i = 0; i < NF; ++i) {
        const unsigned rnd = ex.sr ? sr_bits(ex.seed, ex.step, node, i) : 0u;
        store_with_ghosts<D>(out + i * g.fs, g, x, y, z, kpack<ST, PDE>(acc[i], cf.ref[i], rnd));
    }
}

template <int LAT, int PDE, int LEVELS, int ST>
__global__ void __launch_bounds__(256) k_direct(Geom g, const void* __restrict__ in0v,
                                                const void* __restrict__ in1v, void* __restrict__ outv,
                                                Coef<typename Storage<ST>::T> cf, StepExtra ex) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    direct_node<LAT, PDE, LEVELS, ST>(g, in0v, in1v, outv, cf, ex, x, y, z);
}

template <int LAT, int PDE, int LEVELS, int ST>
cudaError_t launch_direct(const LaunchArgs& a) {
    using T = typename Storage<ST>::T;
    dim3 block(64, 4, 1);
    dim3 grid((a.g.nx + block.x - 1) / block.x, (a.g.ny + block.y - 1) / block.y, a.g.nz);
    k_direct<LAT, PDE, LEVELS, ST><<<grid, block, 0, a.stream>>>(a.g, a.in0, a.in1, a.out,
                                                                  *static_cast<const Coef<T>*>(a.coef), a.ex);
    return cudaGetLastError();
}

template <int LAT, int PDE, int LEVELS, int ST, int SRC>
__global__ void __launch_bounds__(256) k_direct_src(Geom g, const void* __restrict__ in0v,
                                                    const void* __restrict__ in1v, void* __restrict__ outv,
                                                    Coef<typename Storage<ST>::T> cf, StepExtra ex,
                                                    const __grid_constant__ SrcArgs<typename Storage<ST>::T> sa) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    direct_node<LAT, PDE, LEVELS, ST, SRC>(g, in0v, in1v, outv, cf, ex, x, y, z, &sa);
}

template <int LAT, int PDE, int LEVELS, int ST, int SRC>
cudaError_t launch_direct_src(const LaunchArgs& a) {
    using T = typename Storage<ST>::T;
    SrcArgs<T> sa;
    sa.s[0] = static_cast<const T*>(a.src[0]);
    sa.s[1] = static_cast<const T*>(LEVELS == 3 ? a.src[1] : a.src[0]);
    sa.w = *static_cast<const SrcCoef<T>*>(a.src_coef);
    dim3 block(64, 4, 1);
    dim3 grid((a.g.nx + block.x - 1) / block.x, (a.g.ny + block.y - 1) / block.y, a.g.nz);
    k_direct_src<LAT, PDE, LEVELS, ST, SRC><<<grid, block, 0, a.stream>>>(
        a.g, a.in0, a.in1, a.out, *static_cast<const Coef<T>*>(a.coef), a.ex, sa);
    return cudaGetLastError();
}

}  // namespace mmfd
