// k_march3d.cuh -- 3D MMFD step: plane-marching CTAs fed by a TMA shared-memory ring.
//
// A CTA owns items of 128 columns x TY rows x H planes; it has TY consumer warps (one output
// row each, 4 consecutive nodes per lane) and one producer warp.  The producer's lane 0 streams
// input planes z0-1 .. z0+H: per plane, per field and input level, one cp.async.bulk.tensor.3d
// box of (128 + 2 x 16 bytes) x (TY + 2) rows x 1 plane into an NSTAGE ring, completing on the
// stage's `full` mbarrier; consumers release a stage through its `empty` mbarrier (one arrival
// per consumer warp).  A consumer reads the input nodes its row needs from the three rows
// y-1, y, y+1 of the staged plane (pull in x and y) and pushes their contributions into register
// accumulators of the output planes z-1, z, z+1 (push in z) -- the paired central form of the
// MMFD update (see mmfd_internal.h).  After plane z the accumulators of plane z-1 are complete
// and are stored (plus periodic ghost images at the domain edges).  Every wait is bounded: on
// timeout the warp records KERR_TMA_TIMEOUT, waits (bounded) for the copies still in flight
// into this CTA, and exits.
#pragma once

#include "k_direct.cuh"
#include "k_march2d.cuh"
#include "kernels.h"
#include "stencil.cuh"
#include "tma.cuh"

namespace mmfd {

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// The lean NSE variants with 4-row tiles are held to four CTAs per SM (96 registers): on nse3d_512
// FP32 that ran 136 GLUPS against 129 at three CTAs (119 registers).  With 16-row tiles a CTA of
// 17 warps fills the SM on its own.
template <int LAT, int PDE, int LEVELS, int ST, int TY, int NSTAGE, int SRC = 0, int LEAN = LEAN_NONE, int SRM = 2>
__global__ void __launch_bounds__((TY + 1) * 32, (LEAN != LEAN_NONE && TY <= 4) ? 4 : 1) k_march3d(const __grid_constant__ TmapSet maps, Geom g,
                                                           void* __restrict__ outv, Coef<typename Storage<ST>::T> cf,
                                                           StepExtra ex, int H, int nitems, int* __restrict__ err,
                                                           const __grid_constant__ SrcParam<typename Storage<ST>::T, SRC> sa) {
    using Tr = Storage<ST>;
    using S = typename Tr::S;
    using T = typename Tr::T;
    constexpr int LN = 4;
    constexpr int ES = (int)sizeof(S);
    constexpr int ALIGN = 16 / ES;
    constexpr int COLS = 32 * LN;
    constexpr int BOXW = COLS + 2 * ALIGN;
    constexpr int BOXH = TY + 2;
    constexpr int ROWB = BOXW * ES;                                // bytes per staged row
    constexpr int SLOT = ((ROWB * BOXH + 127) / 128) * 128;       // bytes per (stage, field)
    constexpr int NF = pde_nf(PDE, LAT);
    constexpr int NIN = NF * (LEVELS - 1);
    constexpr int NP = lat_npair(LAT);
    constexpr uint32_t kTx = (uint32_t)(NIN * BOXW * BOXH * ES);
    constexpr int D = 3;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + NSTAGE;
    unsigned char* ring = smem + 128 * ((2 * NSTAGE * 8 + 127) / 128);
    auto slot = [&](int s, int q) -> unsigned char* { return ring + (size_t)(s * NIN + q) * SLOT; };

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int xs = (g.nx + COLS - 1) / COLS;       // x strips
    const int ys = (g.ny + TY - 1) / TY;           // y tiles
    // This CTA's segments (tile, planes z0 .. z0 + nzs - 1), each streamed with one halo plane on
    // either side: items of H planes dealt round-robin (H > 0), or (H < 0) one balanced range of
    // the (y tile, plane) pairs, y-tile-major, per group of xs CTAs: the CTAs of a group take the
    // xs strips of the same range, so the strips of a row advance plane by plane together and
    // meet each other's halo columns in L2 (gridDim.x is a multiple of xs then).  Producer and
    // consumers walk the same sequence.
    const long long tiles = (long long)xs * ys;
    int item = blockIdx.x;
    long long w = 0, whi = 0;
    const int strip = blockIdx.x % xs;
    if (H < 0) {
        const long long total = (long long)ys * g.nz;
        const long long groups = gridDim.x / xs, grp = blockIdx.x / xs;
        w = total * grp / groups;
        whi = total * (grp + 1) / groups;
    }
    auto next_seg = [&](int& tile, int& z0, int& nzs) -> bool {
        if (H > 0) {
            if (item >= nitems) return false;
            tile = (int)(item % tiles);
            z0 = (int)(item / tiles) * H;
            nzs = min(H, g.nz - z0);
            item += gridDim.x;
            return true;
        }
        if (w >= whi) return false;
        tile = (int)(w / g.nz) * xs + strip;
        z0 = (int)(w % g.nz);
        nzs = (int)min((long long)(g.nz - z0), whi - w);
        w += nzs;
        return true;
    };

    if (threadIdx.x == 0) {
#pragma unroll
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], TY);
        }
        fence_mbar_init();
#pragma unroll
        for (int q = 0; q < NIN; ++q) tma_prefetch_desc(&maps.m[q]);
    }
    __syncthreads();

    if (warp == TY) {
        // ---------------------------------------------------------------- producer warp
        if (lane != 0) return;
        long long k = 0;
        bool failed = false;
        int tile = 0, z0 = 0, nzs = 0;
        while (!failed && next_seg(tile, z0, nzs)) {
            const int xcol = (tile % xs) * COLS;
            const int yrow = (tile / xs) * TY;      // padded row of interior y0 - 1
            const int np = nzs + 2;
            for (int i = 0; i < np; ++i, ++k) {
                const int s = (int)(k % NSTAGE);
                if (!mbar_wait_bounded(&empty[s], (uint32_t)(((k / NSTAGE) & 1) ^ 1))) {
                    failed = true;
                    break;
                }
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&full[s], kTx);
#pragma unroll
                for (int q = 0; q < NIN; ++q) tma_load_3d(slot(s, q), &maps.m[q], &full[s], xcol, yrow, z0 + i);
            }
        }
        if (failed) atomicExch(err, KERR_TMA_TIMEOUT);
        // do not leave while copies into this CTA's shared memory may still land
        const long long first = k > NSTAGE ? k - NSTAGE : 0;
        for (long long j = first; j < k; ++j) mbar_wait_bounded(&full[j % NSTAGE], (uint32_t)((j / NSTAGE) & 1));
        return;
    }

    // -------------------------------------------------------------------- consumer warps
    T accP[LN][NF], accC[LN][NF], accN[LN][NF];
    EdgeStore<3, ST> es;
    S* out = static_cast<S*>(outv);
    long long k = 0;
    bool failed = false;
    int tile = 0, z0 = 0, nzs = 0;
    while (!failed && next_seg(tile, z0, nzs)) {
        const int x0 = (tile % xs) * COLS;
        const int y0 = (tile / xs) * TY;
        const int np = nzs + 2;
        const int xb = x0 + lane * LN;
        es.init(g, xb, true);
        const int y = y0 + warp;
#pragma unroll
        for (int n = 0; n < LN; ++n)
#pragma unroll
            for (int f = 0; f < NF; ++f) accP[n][f] = accC[n][f] = accN[n][f] = acc_zero<T>();
        for (int i = 0; i < np; ++i, ++k) {
            const int s = (int)(k % NSTAGE);
            const bool ok = mbar_wait_bounded(&full[s], (uint32_t)((k / NSTAGE) & 1));
            if (__any_sync(0xffffffffu, !ok)) {
                failed = true;
                break;
            }
#pragma unroll
            for (int l = 0; l < LEVELS - 1; ++l) {
                // raw fields of nodes xb-1 .. xb+4 in rows y-1, y, y+1 of this plane
                T raw[3][LN + 2][NF];
#pragma unroll
                for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        const unsigned char* rowp = slot(s, l * NF + f) + (size_t)(warp + dy) * ROWB;
                        const S* sp = reinterpret_cast<const S*>(rowp);
                        T v4[4];
                        lds4<ST, PDE>(rowp + (size_t)(ALIGN + lane * LN) * ES, cf.ref[f], v4);
                        raw[dy][1][f] = v4[0];
                        raw[dy][2][f] = v4[1];
                        raw[dy][3][f] = v4[2];
                        raw[dy][4][f] = v4[3];
                        raw[dy][0][f] = kload<ST, PDE>(sp + ALIGN + lane * LN - 1, cf.ref[f]);
                        raw[dy][LN + 1][f] = kload<ST, PDE>(sp + ALIGN + lane * LN + LN, cf.ref[f]);
                    }
                static_for<0, 3>([&](auto dyc) {
                    constexpr int DY = decltype(dyc)::value - 1;
                    static_for<0, LN + 2>([&](auto cc) {
                        constexpr int C = decltype(cc)::value - 1;
                        const T* f = raw[DY + 1][C + 1];
                        if constexpr (PDE == PDE_LCDE) {
                            const T phi = f[0];
                            if constexpr (DY == 0 && C >= 0 && C < LN) accC[C][0] += cf.W0[l] * phi;
                            static_for<0, NP>([&](auto pcc) {
                                constexpr int P_ = decltype(pcc)::value;
                                constexpr int EX = pair_e(LAT, P_, 0), EY = pair_e(LAT, P_, 1), EZ = pair_e(LAT, P_, 2);
                                // plus: output (x, y) <- input (x + EX, y + EY); minus: <- (x - EX, y - EY)
                                constexpr int KP = C - EX, KM = C + EX;
                                if constexpr (DY == EY && KP >= 0 && KP < LN) {
                                    if constexpr (EZ == 1) accP[KP][0] += cf.Wp[l][P_] * phi;
                                    else accC[KP][0] += cf.Wp[l][P_] * phi;
                                }
                                if constexpr (DY == -EY && KM >= 0 && KM < LN) {
                                    if constexpr (EZ == 1) accN[KM][0] += cf.Wm[l][P_] * phi;
                                    else accC[KM][0] += cf.Wm[l][P_] * phi;
                                }
                            });
                        } else if constexpr (PDE == PDE_NSE && LEAN != LEAN_NONE) {
                            // lean He-Luo form (Coef::nA): a+ / a- folded into E', O'; one FMA
                            // per pair on a per-node base shared by the axis / diagonal pairs
                            constexpr auto uses = [](int p) constexpr {
                                const int ex = pair_e(LAT, p, 0), ey = pair_e(LAT, p, 1);
                                const bool plus = DY == ey && C - ex >= 0 && C - ex < LN;
                                const bool minus = DY == -ey && C + ex >= 0 && C + ex < LN;
                                return plus || minus;
                            };
                            constexpr bool CENTRE = DY == 0 && C >= 0 && C < LN;
                            constexpr bool AX = uses(0) || uses(1) || uses(2);
                            constexpr bool DG = uses(3) || uses(4) || uses(5) || uses(6) || uses(7) || uses(8);
                            if constexpr (CENTRE || AX || DG) {
                                const T rho = f[0], ux = f[1], uy = f[2], uz = f[3];
                                const T U = uz * uz + (uy * uy + ux * ux);
                                if constexpr (CENTRE) {
                                    accC[C][0] += cf.nc[l][1] * U + cf.nc[l][0] * rho;
                                    accC[C][1] += cf.ab0[l] * ux;
                                    accC[C][2] += cf.ab0[l] * uy;
                                    accC[C][3] += cf.ab0[l] * uz;
                                }
                                [[maybe_unused]] T Bk[2];
                                if constexpr (AX) Bk[0] = cf.nU[l][0] * U + cf.nA[l][0] * rho;
                                if constexpr (DG) Bk[1] = cf.nU[l][1] * U + cf.nA[l][1] * rho;
                                static_for<0, NP>([&](auto pcc) {
                                    constexpr int P_ = decltype(pcc)::value;
                                    constexpr int EX = pair_e(LAT, P_, 0), EY = pair_e(LAT, P_, 1),
                                                  EZ = pair_e(LAT, P_, 2);
                                    constexpr int KP = C - EX, KM = C + EX;
                                    constexpr bool HP = DY == EY && KP >= 0 && KP < LN;
                                    constexpr bool HM = DY == -EY && KM >= 0 && KM < LN;
                                    if constexpr (HP || HM) {
                                        const T cu = edot<LAT, P_>(ux, uy, uz);
                                        const T E = cf.nk[l][P_] * (cu * cu) + Bk[pair_class(LAT, P_)];
                                        const T O = cf.no[l][P_] * cu;
                                        [[maybe_unused]] T sE = T(0), mO = T(0);
                                        if constexpr (LEAN == LEAN_GENERAL) {
                                            sE = cf.ap[l] * E;
                                            mO = cf.abp[l] * O;
                                        }
                                        if constexpr (HP) {
                                            T* acc = EZ == 1 ? accP[KP] : accC[KP];
                                            lean_push<LAT, LEAN, P_, 1, NF>(acc, cf, l, E, O, sE, mO);
                                        }
                                        if constexpr (HM) {
                                            T* acc = EZ == 1 ? accN[KM] : accC[KM];
                                            lean_push<LAT, LEAN, P_, -1, NF>(acc, cf, l, E, O, sE, mO);
                                        }
                                    }
                                });
                            }
                        } else {
                            constexpr auto uses = [](int p) constexpr {
                                const int ex = pair_e(LAT, p, 0), ey = pair_e(LAT, p, 1);
                                const bool plus = DY == ey && C - ex >= 0 && C - ex < LN;
                                const bool minus = DY == -ey && C + ex >= 0 && C + ex < LN;
                                return plus || minus;
                            };
                            constexpr bool CENTRE = DY == 0 && C >= 0 && C < LN;
                            constexpr bool ANY = CENTRE || uses(0) || uses(1) || uses(2) || uses(3) || uses(4) ||
                                                 uses(5) || uses(6) || uses(7) || uses(8);
                            if constexpr (ANY) {
                                Basis<LAT, PDE, T> b;
                                b.init(f, cf);
                                if constexpr (CENTRE) {
                                    accC[C][0] += cf.a0[l] * b.A() + cf.ap[l] * b.rest(cf);
                                    if constexpr (PDE == PDE_NSE) {
#pragma unroll
                                        for (int a = 0; a < D; ++a) accC[C][1 + a] += cf.ab0[l] * b.mom(a);
                                    }
                                }
                                static_for<0, NP>([&](auto pcc) {
                                    constexpr int P_ = decltype(pcc)::value;
                                    constexpr int EX = pair_e(LAT, P_, 0), EY = pair_e(LAT, P_, 1),
                                                  EZ = pair_e(LAT, P_, 2);
                                    constexpr int KP = C - EX, KM = C + EX;
                                    constexpr bool HP = DY == EY && KP >= 0 && KP < LN;
                                    constexpr bool HM = DY == -EY && KM >= 0 && KM < LN;
                                    if constexpr (HP || HM) {
                                        T E, O;
                                        b.template eo<P_>(cf, E, O);
                                        const T sE = cf.ap[l] * E;
                                        [[maybe_unused]] T mO = T(0);
                                        if constexpr (PDE == PDE_NSE) mO = cf.abp[l] * O;
                                        auto push = [&](T (&acc)[LN][NF], int node, T sv, T mv) {
                                            acc[node][0] += sv;
                                            if constexpr (PDE == PDE_NSE) {
                                                if constexpr (EX != 0) acc[node][1] += (T(EX) * cf.fmom[0]) * mv;
                                                if constexpr (EY != 0) acc[node][2] += (T(EY) * cf.fmom[1]) * mv;
                                                if constexpr (EZ != 0) acc[node][3] += (T(EZ) * cf.fmom[2]) * mv;
                                            }
                                        };
                                        if constexpr (HP) {
                                            const T sv = cf.am[l] * O + sE;
                                            T mv = T(0);
                                            if constexpr (PDE == PDE_NSE) mv = cf.abm[l] * E + mO;
                                            if constexpr (EZ == 1) push(accP, KP, sv, mv);
                                            else push(accC, KP, sv, mv);
                                        }
                                        if constexpr (HM) {
                                            const T sv = sE - cf.am[l] * O;
                                            T mv = T(0);
                                            if constexpr (PDE == PDE_NSE) mv = mO - cf.abm[l] * E;
                                            if constexpr (EZ == 1) push(accN, KM, sv, mv);
                                            else push(accC, KM, sv, mv);
                                        }
                                    }
                                });
                            }
                        }
                    });
                });
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            // plane z0 - 1 + i - 1 is complete
            if (i >= 2 && y < g.ny) {
                const int zo = z0 + i - 2;
                const long long nb = ((long long)zo * g.ny + y) * g.nx;
                [[maybe_unused]] T add[4];
                if constexpr (SRC != 0) source_quad<LAT, SRC, LEVELS, T>(g, sa, y, zo, xb, add);
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    S sv[4];
#pragma unroll
                    for (int n = 0; n < 4; ++n) {
                        const unsigned rnd = sr_on<SRM>(ex) ? sr_bits(ex.seed, ex.step, nb + xb + n, f) : 0u;
                        T v = accP[n][f];
                        if constexpr (SRC != 0) {
                            if (f == 0) v += add[n];
                        }
                        sv[n] = kpack<ST, PDE>(v, cf.ref[f], rnd);
                    }
                    S* fo = out + (size_t)f * g.fs;
                    es.put(fo, g, xb, y, zo, sv);
                }
            }
#pragma unroll
            for (int n = 0; n < LN; ++n)
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    accP[n][f] = accC[n][f];
                    accC[n][f] = accN[n][f];
                    accN[n][f] = acc_zero<T>();
                }
        }
    }
    if (failed && lane == 0) atomicExch(err, KERR_TMA_TIMEOUT);
}

template <int ST, int LEVELS, int NF, int TY, int NSTAGE>
constexpr size_t march3d_smem() {
    constexpr int ES = (int)sizeof(typename Storage<ST>::S);
    constexpr int ROWB = (128 + 2 * (16 / ES)) * ES;
    constexpr int SLOT = ((ROWB * (TY + 2) + 127) / 128) * 128;
    return 128 + 128 * ((2 * NSTAGE * 8 + 127) / 128) + (size_t)NSTAGE * NF * (LEVELS - 1) * SLOT;
}

// Rows per CTA tile: 8 for the light linear stencil, 4 where registers are scarce.
constexpr int tile_rows(int pde) { return pde == PDE_LCDE ? 8 : 4; }

// Ring depth: about BUDGET bytes of stages per CTA (48 KB where several CTAs share an SM), between
// 2 and 8 planes in flight.
template <int LAT, int PDE, int LEVELS, int ST, int TY = tile_rows(PDE), size_t BUDGET = 49152>
constexpr int march3d_stages() {
    constexpr size_t per = march3d_smem<ST, LEVELS, pde_nf(PDE, LAT), TY, 1>() - 256;
    constexpr size_t n = BUDGET / per;
    return n < 2 ? 2 : (n > 8 ? 8 : (int)n);
}

// Tiles of 16 rows for the lean D3Q19 NSE kernels: one CTA of 16 row warps and the producer per
// SM, its ring given about 200 KB of shared memory.  Streaming the lean step's loads and stores
// alone (no arithmetic) through such tiles ran at 6.1 TB/s of useful bytes on 512^3, against
// 4.6 TB/s through 4-row tiles at four CTAs per SM: the y halo rows fall from 1.5x to 1.125x the
// tile and the SM holds a quarter of the concurrent plane streams.
constexpr int kLeanWideRows = 16;
constexpr size_t kLeanWideRing = 200 * 1024;

template <int LAT, int PDE, int LEVELS, int ST, int TY, int NSTAGE, int SRC = 0, int LEAN = LEAN_NONE, int SRM = 2>
cudaError_t launch_march3d_t(const LaunchArgs& a) {
    using T = typename Storage<ST>::T;
    constexpr int NF = pde_nf(PDE, LAT);
    constexpr size_t smem = march3d_smem<ST, LEVELS, NF, TY, NSTAGE>();
    constexpr int THREADS = (TY + 1) * 32;
    auto kern = k_march3d<LAT, PDE, LEVELS, ST, TY, NSTAGE, SRC, LEAN, SRM>;
    static int resident = 0;
    if (resident == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0, dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem);
        if (e != cudaSuccess) return e;
        resident = (per_sm > 0 ? per_sm : 1) * sms;
    }
    const int xs = (a.g.nx + 127) / 128;
    const int ys = (a.g.ny + TY - 1) / TY;
    int H = a.H;
    int nitems = 0, grid = 0;
    if (H <= 0 && TY == kLeanWideRows && ST == ST_BF16) {
        // 16-row BF16 tiles, one CTA per SM: each group of xs CTAs streams one balanced range of the
        // (y tile, plane) pairs, so every SM gets the same work and a tile's halo planes are read
        // once per range.  nse3d_512: 135-136 GLUPS against 128 with items of 64 planes; DRAM
        // reads 1.26x the level (384^3 capture), 1.9x when the strips of a row did not share a
        // range.  The BF16 step is bound by instruction issue; the FP32 step is not, and there
        // items of planes stay faster (135 against 132 GLUPS with the ranges): neighbouring y
        // tiles' ranges sit at unrelated planes and no longer meet each other's halo rows in L2.
        const long long total = (long long)ys * a.g.nz;     // (y tile, plane) pairs per strip
        const long long groups = resident >= xs ? resident / xs : 1;
        H = -1;
        grid = (int)(total < groups ? total : groups) * xs;
        nitems = grid;
    } else if (H <= 0) {
        double best = -1.0;
        for (int h = 4; h <= 512; ++h) {
            const long long items = (long long)xs * ys * ((a.g.nz + h - 1) / h);
            const long long rounds = (items + resident - 1) / resident;
            const double fill = (double)items / (double)(rounds * resident);
            const double eff = fill * (double)h / (double)(h + 2);
            if (eff > best + 1e-9) {
                best = eff;
                H = h;
            }
            if (h >= a.g.nz) break;
        }
    }
    if (H > 0) {
        nitems = xs * ys * ((a.g.nz + H - 1) / H);
        grid = nitems < resident ? nitems : resident;
    }
    SrcParam<T, SRC> sa{};
    if constexpr (SRC != 0) {
        sa.s[0] = static_cast<const T*>(a.src[0]);
        sa.s[1] = static_cast<const T*>(LEVELS == 3 ? a.src[1] : a.src[0]);
        sa.w = *static_cast<const SrcCoef<T>*>(a.src_coef);
    }
    kern<<<grid, THREADS, smem, a.stream>>>(*a.maps, a.g, a.out, *static_cast<const Coef<T>*>(a.coef), a.ex, H,
                                            nitems, a.err, sa);
    return cudaGetLastError();
}

// The same with the stochastic-rounding choice made per launch (see launch_march2d_sr).
template <int LAT, int PDE, int LEVELS, int ST, int TY, int NSTAGE, int SRC = 0, int LEAN = LEAN_NONE>
cudaError_t launch_march3d_sr(const LaunchArgs& a) {
    if constexpr (ST == ST_BF16) {
        if (a.ex.sr) return launch_march3d_t<LAT, PDE, LEVELS, ST, TY, NSTAGE, SRC, LEAN, 1>(a);
    }
    return launch_march3d_t<LAT, PDE, LEVELS, ST, TY, NSTAGE, SRC, LEAN, 0>(a);
}

}  // namespace mmfd
