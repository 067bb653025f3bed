// k_march2d.cuh -- 2D MMFD step: row-marching CTAs fed by a TMA shared-memory ring.
//
// A CTA owns a strip of NW * 128 columns and H rows.  Each warp owns 128 columns (4
// consecutive nodes per lane).  Thread 0 streams the input rows y0-1 .. y0+H of every stored
// field and input level through an NSTAGE-deep ring: one cp.async.bulk.tensor.2d box of
// 128 + 2 * (16 bytes) columns per warp, per field, per row, completing on the stage's
// mbarrier.  Every input row is read from shared memory once and pushed into register
// accumulators of the three output rows it touches (r-1, r, r+1) -- the paired central form
// of the MMFD update (see mmfd_internal.h).  After row r the accumulators of row r-1 are
// complete and are stored with 16-byte vector stores (plus periodic ghost images at the
// domain edges).  Waits are bounded: on timeout the CTA records KERR_TMA_TIMEOUT in the
// solver's device flag, waits (bounded) for its own copies still in flight, and exits.
#pragma once

#include <type_traits>

#include "k_direct.cuh"
#include "kernels.h"
#include "stencil.cuh"
#include "tma.cuh"

namespace mmfd {

constexpr int kLaneNodes = 4;
constexpr int kWarpCols = 32 * kLaneNodes;

template <int ST>
struct MarchCfg {
    static constexpr int ES = (int)sizeof(typename Storage<ST>::S);
    static constexpr int ALIGN = 16 / ES;                        // halo elements per side
    static constexpr int BOXW = kWarpCols + 2 * ALIGN;           // TMA box width (elements)
    static constexpr int SLOT = ((BOXW * ES + 127) / 128) * 128; // bytes per (warp, field) slot
};

// Four consecutive values of storage type S from shared memory (aligned) into T.
template <int ST>
__device__ __forceinline__ void lds4(const unsigned char* p, typename Storage<ST>::T ref, typename Storage<ST>::T v[4]) {
    if constexpr (ST == ST_F32) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else if constexpr (ST == ST_F64) {
        const double2 a = *reinterpret_cast<const double2*>(p);
        const double2 b = *reinterpret_cast<const double2*>(p + 16);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    } else {
        const uint2 q = *reinterpret_cast<const uint2*>(p);
        v[0] = ref + __uint_as_float(q.x << 16);
        v[1] = ref + __uint_as_float(q.x & 0xffff0000u);
        v[2] = ref + __uint_as_float(q.y << 16);
        v[3] = ref + __uint_as_float(q.y & 0xffff0000u);
    }
}

template <int ST>
__device__ __forceinline__ void stg4(void* p, const typename Storage<ST>::S s[4]) {
    if constexpr (ST == ST_F32) {
        *reinterpret_cast<float4*>(p) = make_float4(s[0], s[1], s[2], s[3]);
    } else if constexpr (ST == ST_F64) {
        reinterpret_cast<double2*>(p)[0] = make_double2(s[0], s[1]);
        reinterpret_cast<double2*>(p)[1] = make_double2(s[2], s[3]);
    } else {
        const unsigned lo = (unsigned)__bfloat16_as_ushort(s[0]) | ((unsigned)__bfloat16_as_ushort(s[1]) << 16);
        const unsigned hi = (unsigned)__bfloat16_as_ushort(s[2]) | ((unsigned)__bfloat16_as_ushort(s[3]) << 16);
        *reinterpret_cast<uint2*>(p) = make_uint2(lo, hi);
    }
}

template <int LAT, int PDE, int LEVELS, int ST, int NW, int NSTAGE>
__global__ void __launch_bounds__(NW * 32) k_march2d(const __grid_constant__ TmapSet maps, Geom g,
                                                     void* __restrict__ outv, Coef<typename Storage<ST>::T> cf,
                                                     StepExtra ex, int H, int* __restrict__ err) {
    using Tr = Storage<ST>;
    using S = typename Tr::S;
    using T = typename Tr::T;
    using Cfg = MarchCfg<ST>;
    constexpr int NF = pde_nf(PDE, LAT);
    constexpr int NIN = NF * (LEVELS - 1);
    constexpr int NP = lat_npair(LAT);
    constexpr int D = 2;

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    unsigned char* ring = smem + 128;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int x0 = blockIdx.x * (NW * kWarpCols);
    const int y0 = blockIdx.y * H;
    const int heff = min(H, g.ny - y0);
    const int nrows = heff + 2;
    constexpr uint32_t kTx = (uint32_t)(NIN * NW * Cfg::BOXW * Cfg::ES);

    auto slot = [&](int s, int q, int w) -> unsigned char* {
        return ring + (size_t)((s * NIN + q) * NW + w) * Cfg::SLOT;
    };
    auto issue = [&](int i) {
        const int s = i % NSTAGE;
        mbar_arrive_expect_tx(&full[s], kTx);
        const int prow = y0 + i;  // padded row of input row y0 - 1 + i
#pragma unroll
        for (int q = 0; q < NIN; ++q)
#pragma unroll
            for (int w = 0; w < NW; ++w) tma_load_2d(slot(s, q, w), &maps.m[q], &full[s], x0 + w * kWarpCols, prow);
    };

    if (threadIdx.x == 0) {
#pragma unroll
        for (int s = 0; s < NSTAGE; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
#pragma unroll
        for (int q = 0; q < NIN; ++q) tma_prefetch_desc(&maps.m[q]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int first = nrows < NSTAGE ? nrows : NSTAGE;
        for (int i = 0; i < first; ++i) issue(i);
    }

    T accP[kLaneNodes][NF], accC[kLaneNodes][NF], accN[kLaneNodes][NF];
#pragma unroll
    for (int k = 0; k < kLaneNodes; ++k)
#pragma unroll
        for (int f = 0; f < NF; ++f) accP[k][f] = accC[k][f] = accN[k][f] = T(0);

    const int xb = x0 + warp * kWarpCols + lane * kLaneNodes;  // first node of this lane
    S* out = static_cast<S*>(outv);
    int i = 0;
    bool failed = false;
    for (; i < nrows; ++i) {
        const int s = i % NSTAGE;
        const bool ok = mbar_wait_bounded(&full[s], (uint32_t)((i / NSTAGE) & 1));
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
#pragma unroll
        for (int l = 0; l < LEVELS - 1; ++l) {
            // raw fields of the 6 nodes xb-1 .. xb+4 of this input row
            T raw[6][NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const unsigned char* base = slot(s, l * NF + f, warp);
                const S* sp = reinterpret_cast<const S*>(base);
                T v4[4];
                lds4<ST>(base + (size_t)(Cfg::ALIGN + lane * kLaneNodes) * Cfg::ES, cf.ref[f], v4);
                raw[0][f] = Tr::load(sp + Cfg::ALIGN + lane * kLaneNodes - 1, cf.ref[f]);
                raw[1][f] = v4[0];
                raw[2][f] = v4[1];
                raw[3][f] = v4[2];
                raw[4][f] = v4[3];
                raw[5][f] = Tr::load(sp + Cfg::ALIGN + lane * kLaneNodes + 4, cf.ref[f]);
            }
            static_for<0, 6>([&](auto cc) {
                constexpr int C = decltype(cc)::value - 1;  // node offset -1 .. 4
                if constexpr (PDE == PDE_LCDE) {
                    const T phi = raw[C + 1][0];
                    if constexpr (C >= 0 && C < 4) accC[C][0] += cf.W0[l] * phi;
                    static_for<0, NP>([&](auto pc) {
                        constexpr int P = decltype(pc)::value;
                        constexpr int EX = pair_e(LAT, P, 0), EY = pair_e(LAT, P, 1);
                        constexpr int TP = C - EX, TM = C + EX;
                        if constexpr (TP >= 0 && TP < 4) {
                            if constexpr (EY == 1) accP[TP][0] += cf.Wp[l][P] * phi;
                            else accC[TP][0] += cf.Wp[l][P] * phi;
                        }
                        if constexpr (TM >= 0 && TM < 4) {
                            if constexpr (EY == 1) accN[TM][0] += cf.Wm[l][P] * phi;
                            else accC[TM][0] += cf.Wm[l][P] * phi;
                        }
                    });
                } else {
                    Basis<LAT, PDE, T> b;
                    b.init(raw[C + 1], cf);
                    if constexpr (C >= 0 && C < 4) {
                        accC[C][0] += cf.a0[l] * b.A() + cf.ap[l] * b.rest(cf);
                        if constexpr (PDE == PDE_NSE) {
#pragma unroll
                            for (int a = 0; a < D; ++a) accC[C][1 + a] += cf.ab0[l] * b.mom(a);
                        }
                    }
                    static_for<0, NP>([&](auto pc) {
                        constexpr int P = decltype(pc)::value;
                        constexpr int EX = pair_e(LAT, P, 0), EY = pair_e(LAT, P, 1);
                        constexpr int TP = C - EX, TM = C + EX;
                        constexpr bool HP = TP >= 0 && TP < 4, HM = TM >= 0 && TM < 4;
                        if constexpr (HP || HM) {
                            T E, O;
                            b.template eo<P>(cf, E, O);
                            const T sE = cf.ap[l] * E, sO = cf.am[l] * O;
                            T mE = T(0), mO = T(0);
                            if constexpr (PDE == PDE_NSE) {
                                mE = cf.abm[l] * E;
                                mO = cf.abp[l] * O;
                            }
                            auto add = [&](T (&acc)[kLaneNodes][NF], int node, T sv, T mv) {
                                acc[node][0] += sv;
                                if constexpr (PDE == PDE_NSE) {
                                    if constexpr (EX != 0) acc[node][1] += T(EX) * cf.fmom[0] * mv;
                                    if constexpr (EY != 0) acc[node][2] += T(EY) * cf.fmom[1] * mv;
                                }
                            };
                            if constexpr (HP) {
                                if constexpr (EY == 1) add(accP, TP, sE + sO, mO + mE);
                                else add(accC, TP, sE + sO, mO + mE);
                            }
                            if constexpr (HM) {
                                if constexpr (EY == 1) add(accN, TM, sE - sO, mO - mE);
                                else add(accC, TM, sE - sO, mO - mE);
                            }
                        }
                    });
                }
            });
        }
        // row y0 - 1 + i - 1 is complete
        if (i >= 2) {
            const int yo = y0 + i - 2;
            const long long nb = (long long)yo * g.nx;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                S sv[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const unsigned rnd = ex.sr ? sr_bits(ex.seed, ex.step, nb + xb + k, f) : 0u;
                    sv[k] = Tr::pack(accP[k][f], cf.ref[f], rnd);
                }
                S* fo = out + (size_t)f * g.fs;
                const bool interior = xb > 0 && xb + 3 < g.nx - 1 && yo > 0 && yo < g.ny - 1;
                if (interior) {
                    stg4<ST>(fo + g.at(xb, yo, 0), sv);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (xb + k < g.nx) store_with_ghosts<2>(fo, g, xb + k, yo, 0, sv[k]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kLaneNodes; ++k)
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                accP[k][f] = accC[k][f];
                accC[k][f] = accN[k][f];
                accN[k][f] = T(0);
            }
        __syncthreads();  // every warp is done with stage s
        if (threadIdx.x == 0 && i + NSTAGE < nrows) {
            fence_proxy_async_smem();
            issue(i + NSTAGE);
        }
    }
    if (failed) {
        if (threadIdx.x == 0) {
            atomicExch(err, KERR_TMA_TIMEOUT);
            const int last = min(nrows, i + NSTAGE);
            for (int j = i; j < last; ++j) mbar_wait_bounded(&full[j % NSTAGE], (uint32_t)((j / NSTAGE) & 1));
        }
        __syncthreads();
    }
}

template <int ST, int LEVELS, int NF, int NW, int NSTAGE>
constexpr size_t march2d_smem() {
    return 128 + (size_t)NSTAGE * NF * (LEVELS - 1) * NW * MarchCfg<ST>::SLOT;
}

template <int LAT, int PDE, int LEVELS, int ST, int NW, int NSTAGE>
cudaError_t launch_march2d_t(const LaunchArgs& a) {
    using T = typename Storage<ST>::T;
    constexpr int NF = pde_nf(PDE, LAT);
    constexpr size_t smem = march2d_smem<ST, LEVELS, NF, NW, NSTAGE>();
    auto kern = k_march2d<LAT, PDE, LEVELS, ST, NW, NSTAGE>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int H = a.H > 0 ? a.H : 64;
    dim3 grid((a.g.nx + NW * kWarpCols - 1) / (NW * kWarpCols), (a.g.ny + H - 1) / H, 1);
    kern<<<grid, NW * 32, smem, a.stream>>>(*a.maps, a.g, a.out, *static_cast<const Coef<T>*>(a.coef), a.ex, H,
                                             a.err);
    return cudaGetLastError();
}

}  // namespace mmfd
