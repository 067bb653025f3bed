// k_march2d.cuh -- 2D MMFD step: row-marching warps, each fed by its own TMA shared-memory ring.
//
// A warp owns items of 128 columns x H rows (4 consecutive nodes per lane).  Its lane 0
// streams the input rows y0-1 .. y0+H of every stored field and input level through a private
// NSTAGE-deep ring: one cp.async.bulk.tensor.2d box of 128 + 2 x (16 bytes) columns per field
// per row, completing on the stage's mbarrier.  Every input row is read from shared memory
// once and pushed into register accumulators of the three output rows it touches
// (r-1, r, r+1) -- the paired central form of the MMFD update (see mmfd_internal.h).  After
// row r the accumulators of row r-1 are complete and are stored with vector stores (plus the
// periodic ghost images at the domain edges).  No CTA-wide barrier is used after start-up.
// Waits are bounded: on timeout the warp records KERR_TMA_TIMEOUT in the solver's device flag,
// waits (bounded) for its own copies still in flight, and exits.
#pragma once

#include <type_traits>

#include "k_direct.cuh"
#include "kernels.h"
#include "pack2.cuh"
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

// Work decomposition: an item is (128-column warp strip, H-row segment).  Every warp walks its
// own sequence of items (item = global warp id, + total warps, ...) as one stream of input
// rows; lane 0 keeps NSTAGE rows of that stream in flight through the warp's private ring, so
// the prefetch runs across item boundaries and warps never wait for one another.
struct RowCursor {
    int item;  // current item
    int row;   // input row index within the item (0 .. nrows - 1)
};

__device__ __forceinline__ int march_item_rows(int item, int strips, int H, int ny) {
    const int seg = item / strips;
    return min(H, ny - seg * H) + 2;
}

template <int LAT, int PDE, int LEVELS, int ST, int NW, int NSTAGE>
__global__ void __launch_bounds__(NW * 32) k_march2d(const __grid_constant__ TmapSet maps, Geom g,
                                                     void* __restrict__ outv, Coef<typename Storage<ST>::T> cf,
                                                     StepExtra ex, int H, int nitems, int* __restrict__ err) {
    using Tr = Storage<ST>;
    using S = typename Tr::S;
    using T = typename Tr::T;
    using Cfg = MarchCfg<ST>;
    constexpr int NF = pde_nf(PDE, LAT);
    constexpr int NIN = NF * (LEVELS - 1);
    constexpr int NP = lat_npair(LAT);
    constexpr int D = 2;
    constexpr uint32_t kTx = (uint32_t)(NIN * Cfg::BOXW * Cfg::ES);
    constexpr size_t kRingBytes = (size_t)NSTAGE * NIN * Cfg::SLOT;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations must sit on 128-byte boundaries whatever the dynamic-smem base is
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem) + warp * NSTAGE;
    unsigned char* ring = smem + 128 * ((NW * NSTAGE * 8 + 127) / 128) + warp * kRingBytes;

    const int strips = (g.nx + kWarpCols - 1) / kWarpCols;
    const int wstride = gridDim.x * NW;
    const int wid = blockIdx.x * NW + warp;
    if (wid >= nitems) return;

    auto slot = [&](int s, int q) -> unsigned char* { return ring + (size_t)(s * NIN + q) * Cfg::SLOT; };

    // producer (lane 0): row stream cursor and count of rows issued
    RowCursor pc{wid, 0};
    long long issued = 0;
    auto issue_next = [&]() {
        if (pc.item >= nitems) return;
        const int s = (int)(issued % NSTAGE);
        mbar_arrive_expect_tx(&full[s], kTx);
        const int xcol = (pc.item % strips) * kWarpCols;             // padded column of the box
        const int prow = (pc.item / strips) * H + pc.row;            // padded row of input row y0 - 1 + row
#pragma unroll
        for (int q = 0; q < NIN; ++q) tma_load_2d(slot(s, q), &maps.m[q], &full[s], xcol, prow);
        ++issued;
        if (++pc.row == march_item_rows(pc.item, strips, H, g.ny)) {
            pc.item += wstride;
            pc.row = 0;
        }
    };

    if (lane == 0) {
#pragma unroll
        for (int s = 0; s < NSTAGE; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
#pragma unroll
        for (int q = 0; q < NIN; ++q) tma_prefetch_desc(&maps.m[q]);
        for (int k = 0; k < NSTAGE; ++k) issue_next();
    }
    __syncwarp();

    // Accumulators of the three output rows r-1, r, r+1 this lane is building.  Each holds
    // the lane's 4 nodes as two packed pairs: pair 0 = nodes (0, 2), pair 1 = nodes (1, 3).
    using V = typename Pair2<T>::type;
    V acc0[2][NF], acc1[2][NF], acc2[2][NF];
    S* out = static_cast<S*>(outv);
    long long consumed = 0;
    bool failed = false;

    // Push one input row into (P = row r-1, Cr = row r, N = row r+1) and, when row r-1 is
    // complete, store it and clear it (it becomes the next "row r+1").
    auto row_body = [&](int i, int y0, int xb, V (&P)[2][NF], V (&Cr)[2][NF], V (&N)[2][NF]) -> bool {
        const int s = (int)(consumed % NSTAGE);
        const bool ok = mbar_wait_bounded(&full[s], (uint32_t)((consumed / NSTAGE) & 1));
        if (__any_sync(0xffffffffu, !ok)) return false;
#pragma unroll
        for (int l = 0; l < LEVELS - 1; ++l) {
            // input groups of node offsets: A = (-1, 1), B = (0, 2), C = (1, 3), D = (2, 4)
            V grp[4][NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const unsigned char* base = slot(s, l * NF + f);
                const S* sp = reinterpret_cast<const S*>(base);
                T v4[4];
                lds4<ST>(base + (size_t)(Cfg::ALIGN + lane * kLaneNodes) * Cfg::ES, cf.ref[f], v4);
                const T left = Tr::load(sp + Cfg::ALIGN + lane * kLaneNodes - 1, cf.ref[f]);
                const T right = Tr::load(sp + Cfg::ALIGN + lane * kLaneNodes + 4, cf.ref[f]);
                grp[0][f] = mk2(left, v4[1]);
                grp[1][f] = mk2(v4[0], v4[2]);
                grp[2][f] = mk2(v4[1], v4[3]);
                grp[3][f] = mk2(v4[2], right);
            }
            static_for<0, 4>([&](auto gc) {
                constexpr int G = decltype(gc)::value;
                constexpr int SX = G - 1;  // x offset of the group's first node
                const V* in = grp[G];
                if constexpr (PDE == PDE_LCDE) {
                    const V phi = in[0];
                    if constexpr (SX == 0 || SX == 1) Cr[SX][0] = fma2(bc2(cf.W0[l]), phi, Cr[SX][0]);
                    static_for<0, NP>([&](auto pcc) {
                        constexpr int P_ = decltype(pcc)::value;
                        constexpr int EX = pair_e(LAT, P_, 0), EY = pair_e(LAT, P_, 1);
                        constexpr int OP = SX - EX, OM = SX + EX;
                        if constexpr (OP == 0 || OP == 1) {
                            if constexpr (EY == 1) P[OP][0] = fma2(bc2(cf.Wp[l][P_]), phi, P[OP][0]);
                            else Cr[OP][0] = fma2(bc2(cf.Wp[l][P_]), phi, Cr[OP][0]);
                        }
                        if constexpr (OM == 0 || OM == 1) {
                            if constexpr (EY == 1) N[OM][0] = fma2(bc2(cf.Wm[l][P_]), phi, N[OM][0]);
                            else Cr[OM][0] = fma2(bc2(cf.Wm[l][P_]), phi, Cr[OM][0]);
                        }
                    });
                } else {
                    // packed basis of the group (arguments of Eq. (3-3))
                    V A, B[2], m2v, uxx, uyy, uxy;
                    if constexpr (PDE == PDE_NSE) {
                        A = in[0];
                        B[0] = in[1];
                        B[1] = in[2];
                        uxx = mul2(in[1], in[1]);
                        uyy = mul2(in[2], in[2]);
                        uxy = mul2(in[1], in[2]);
                    } else {
                        const V phi = in[0];
                        A = phi;
                        m2v = fma2(fma2(fma2(fma2(bc2(cf.m2[4]), phi, bc2(cf.m2[3])), phi, bc2(cf.m2[2])), phi,
                                        bc2(cf.m2[1])), phi, bc2(cf.m2[0]));
#pragma unroll
                        for (int a = 0; a < D; ++a)
                            B[a] = fma2(fma2(fma2(bc2(cf.flux[a][3]), phi, bc2(cf.flux[a][2])), phi,
                                             bc2(cf.flux[a][1])), phi, bc2(cf.flux[a][0]));
                    }
                    if constexpr (SX == 0 || SX == 1) {
                        V rest;
                        if constexpr (PDE == PDE_NSE)
                            rest = fma2(bc2(cf.rC[1]), uyy, fma2(bc2(cf.rC[0]), uxx, mul2(bc2(cf.rA), A)));
                        else
                            rest = fma2(bc2(cf.rM2), m2v, mul2(bc2(cf.rPhi), A));
                        Cr[SX][0] = fma2(bc2(cf.ap[l]), rest, fma2(bc2(cf.a0[l]), A, Cr[SX][0]));
                        if constexpr (PDE == PDE_NSE) {
                            Cr[SX][1] = fma2(bc2(cf.ab0[l]), B[0], Cr[SX][1]);
                            Cr[SX][2] = fma2(bc2(cf.ab0[l]), B[1], Cr[SX][2]);
                        }
                    }
                    static_for<0, NP>([&](auto pcc) {
                        constexpr int P_ = decltype(pcc)::value;
                        constexpr int EX = pair_e(LAT, P_, 0), EY = pair_e(LAT, P_, 1);
                        constexpr int OP = SX - EX, OM = SX + EX;
                        constexpr bool HP = (OP == 0 || OP == 1), HM = (OM == 0 || OM == 1);
                        if constexpr (HP || HM) {
                            V E, O;
                            if constexpr (PDE == PDE_NSE) {
                                E = fma2(bc2(cf.eC[P_][1]), uyy, fma2(bc2(cf.eC[P_][0]), uxx, mul2(bc2(cf.eA[P_]), A)));
                                if constexpr (EX * EY != 0) E = fma2(bc2(cf.eC[P_][3]), uxy, E);
                            } else {
                                E = fma2(bc2(cf.eM2[P_]), m2v, mul2(bc2(cf.ePhi[P_]), A));
                            }
                            if constexpr (EX != 0 && EY != 0)
                                O = fma2(bc2(cf.oB[P_][1]), B[1], mul2(bc2(cf.oB[P_][0]), B[0]));
                            else if constexpr (EX != 0)
                                O = mul2(bc2(cf.oB[P_][0]), B[0]);
                            else
                                O = mul2(bc2(cf.oB[P_][1]), B[1]);
                            const V sE = mul2(bc2(cf.ap[l]), E);
                            auto push = [&](V (&acc)[2][NF], int o, bool plus) {
                                // scalar / rho: a+ E +- a- O
                                acc[o][0] = plus ? fma2(bc2(cf.am[l]), O, add2(acc[o][0], sE))
                                                 : fma2(bc2(-cf.am[l]), O, add2(acc[o][0], sE));
                                if constexpr (PDE == PDE_NSE) {
                                    // momentum: e_a (c_a / rho0) (abar+ O +- abar- E)
                                    const V mv = plus ? fma2(bc2(cf.abm[l]), E, mul2(bc2(cf.abp[l]), O))
                                                      : fma2(bc2(-cf.abm[l]), E, mul2(bc2(cf.abp[l]), O));
                                    if constexpr (EX != 0) acc[o][1] = fma2(bc2(T(EX) * cf.fmom[0]), mv, acc[o][1]);
                                    if constexpr (EY != 0) acc[o][2] = fma2(bc2(T(EY) * cf.fmom[1]), mv, acc[o][2]);
                                }
                            };
                            if constexpr (HP) {
                                if constexpr (EY == 1) push(P, OP, true);
                                else push(Cr, OP, true);
                            }
                            if constexpr (HM) {
                                if constexpr (EY == 1) push(N, OM, false);
                                else push(Cr, OM, false);
                            }
                        }
                    });
                }
            });
        }
        ++consumed;
        __syncwarp();  // every lane is done reading stage s
        if (lane == 0) {
            fence_proxy_async_smem();
            issue_next();
        }
        // row y0 - 1 + i - 1 is complete
        if (i >= 2 && xb < g.nx) {
            const int yo = y0 + i - 2;
            const long long nb = (long long)yo * g.nx;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const T vals[4] = {lo(P[0][f]), lo(P[1][f]), hi(P[0][f]), hi(P[1][f])};
                S sv[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const unsigned rnd = ex.sr ? sr_bits(ex.seed, ex.step, nb + xb + k, f) : 0u;
                    sv[k] = Tr::pack(vals[k], cf.ref[f], rnd);
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
        for (int o = 0; o < 2; ++o)
#pragma unroll
            for (int f = 0; f < NF; ++f) P[o][f] = bc2(T(0));
        return true;
    };

    for (int item = wid; item < nitems && !failed; item += wstride) {
        const int x0 = (item % strips) * kWarpCols;
        const int y0 = (item / strips) * H;
        const int nrows = march_item_rows(item, strips, H, g.ny);
        const int xb = x0 + lane * kLaneNodes;
#pragma unroll
        for (int o = 0; o < 2; ++o)
#pragma unroll
            for (int f = 0; f < NF; ++f) acc0[o][f] = acc1[o][f] = acc2[o][f] = bc2(T(0));
        // rows rotate through the three accumulator sets without register moves
        for (int i = 0; i < nrows && !failed; i += 3) {
            if (!row_body(i, y0, xb, acc0, acc1, acc2)) { failed = true; break; }
            if (i + 1 < nrows && !row_body(i + 1, y0, xb, acc1, acc2, acc0)) { failed = true; break; }
            if (i + 2 < nrows && !row_body(i + 2, y0, xb, acc2, acc0, acc1)) { failed = true; break; }
        }
    }
    if (failed && lane == 0) {
        atomicExch(err, KERR_TMA_TIMEOUT);
        // wait (bounded) for every copy this warp issued but did not consume
        for (long long k = consumed; k < issued; ++k)
            mbar_wait_bounded(&full[k % NSTAGE], (uint32_t)((k / NSTAGE) & 1));
    }
    __syncwarp();
}

template <int ST, int LEVELS, int NF, int NW, int NSTAGE>
constexpr size_t march2d_smem() {
    return 128 + 128 * ((NW * NSTAGE * 8 + 127) / 128) + (size_t)NW * NSTAGE * NF * (LEVELS - 1) * MarchCfg<ST>::SLOT;
}

template <int LAT, int PDE, int LEVELS, int ST, int NW, int NSTAGE>
cudaError_t launch_march2d_t(const LaunchArgs& a) {
    using T = typename Storage<ST>::T;
    constexpr int NF = pde_nf(PDE, LAT);
    constexpr size_t smem = march2d_smem<ST, LEVELS, NF, NW, NSTAGE>();
    auto kern = k_march2d<LAT, PDE, LEVELS, ST, NW, NSTAGE>;
    static int resident = 0;
    if (resident == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0, dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NW * 32, smem);
        if (e != cudaSuccess) return e;
        resident = (per_sm > 0 ? per_sm : 1) * sms;
    }
    const int strips = (a.g.nx + kWarpCols - 1) / kWarpCols;
    int H = a.H;
    if (H <= 0) {
        // rows per item: maximise (useful rows / streamed rows) x (fill of the resident warp slots)
        const long long wslots = (long long)resident * NW;
        double best = -1.0;
        for (int h = 8; h <= 256; ++h) {
            const long long items = (long long)strips * ((a.g.ny + h - 1) / h);
            const long long rounds = (items + wslots - 1) / wslots;
            const double fill = (double)items / (double)(rounds * wslots);
            const double eff = fill * (double)h / (double)(h + 2);
            if (eff > best + 1e-9) {
                best = eff;
                H = h;
            }
            if (h >= a.g.ny) break;
        }
    }
    const int nitems = strips * ((a.g.ny + H - 1) / H);
    const int blocks_needed = (nitems + NW - 1) / NW;
    const int grid = blocks_needed < resident ? blocks_needed : resident;
    kern<<<grid, NW * 32, smem, a.stream>>>(*a.maps, a.g, a.out, *static_cast<const Coef<T>*>(a.coef), a.ex, H,
                                             nitems, a.err);
    return cudaGetLastError();
}

}  // namespace mmfd
