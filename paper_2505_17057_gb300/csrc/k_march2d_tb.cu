// k_march2d_tb.cu -- temporally blocked 2D MMFD steps for two-level scalar problems (LCDE,
// NCDE): one launch advances TT time levels and reads / writes the stored level once.
//
// A warp owns items of one 128-column strip x H output rows and streams the input rows
// y0-TT .. y0+H+TT-1 of the level, two rows per stage, through its private TMA ring (as
// k_march2d does for the scalar PDEs; rows wrap periodically in y in the producer, and the
// second row of a box that starts on the last row is the ghost image of row 0).  It keeps TT sets of three register accumulator rows,
// one set per time level: an input row is pushed into level 1; the level-1 row it completes
// is pushed, as an input row, into level 2; and so on -- a wavefront of TT steps one row
// apart.  The x-neighbours of a lane's nodes at the intermediate levels come from the
// neighbouring lanes by warp shuffle.  The strip's outermost columns lose validity by one
// column per level, so strips overlap: the lanes cover columns X0 .. X0+127 (X0 = 120 s - 8)
// and only lanes 1 .. 30 (columns X0+4 .. X0+123) store.  Columns within TT of the domain's
// x-edges are read from the ghost columns, which every writer of a blocked solver keeps up to
// date to depth TT (Geom::gx).  Intermediate levels stay in the compute type (they are never
// stored), so for BF16 storage the state is rounded once per TT steps.
//
// JAC: TT Jacobi sweeps of the two-level theta-scheme (Eq. (GCN)) instead of TT steps.  A sweep
// is the LCDE stencil of the coefficient block (no centre weight) plus jw times the right-hand
// side rhs, which does not change between sweeps: when level t completes row r - 1 - t (r the
// input row), rhs of that row is added before the row moves on to level t + 1.  The TT rhs rows
// in use sit in a register window that takes one new row per input row, fetched a row early.  rhs has the
// level's ghosted layout with its x ghosts current, so the columns the wavefront needs are valid;
// lanes whose columns leave the padded row (they feed no stored node) take zero.
#include "k_march2d.cuh"

namespace mmfd {

namespace {

constexpr int kTbStride = 120;   // output columns per strip
constexpr int kTbLead = 8;       // lane 0's first column lies kTbLead columns left of the strip's output

// Push one input row (raw values of the lane's LN nodes and of the two neighbouring nodes) into
// the accumulators of rows r-1 (P), r (C) and r+1 (N): the paired central form of Eq. (2-2-1)
// for the two-level scheme (one input level).
template <int LAT, int PDE, typename T, int LN>
__device__ __forceinline__ void tb_push_row(const Coef<T>& cf, const T (&raw)[LN + 2], T (&accP)[LN], T (&accC)[LN],
                                            T (&accN)[LN]) {
    constexpr int NP = lat_npair(LAT);
    static_for<0, LN + 2>([&](auto cc) {
        constexpr int C = decltype(cc)::value - 1;
        constexpr bool OWN = C >= 0 && C < LN;
        if constexpr (PDE == PDE_LCDE) {
            const T phi = raw[C + 1];
            if constexpr (OWN) accC[C] += cf.W0[0] * phi;
            static_for<0, NP>([&](auto pcc) {
                constexpr int P_ = decltype(pcc)::value;
                constexpr int EX = pair_e(LAT, P_, 0), EY = pair_e(LAT, P_, 1);
                constexpr int TP = C - EX, TM = C + EX;
                if constexpr (TP >= 0 && TP < LN) {
                    if constexpr (EY == 1) accP[TP] += cf.Wp[0][P_] * phi;
                    else accC[TP] += cf.Wp[0][P_] * phi;
                }
                if constexpr (TM >= 0 && TM < LN) {
                    if constexpr (EY == 1) accN[TM] += cf.Wm[0][P_] * phi;
                    else accC[TM] += cf.Wm[0][P_] * phi;
                }
            });
        } else {
            constexpr int MASK = pushed_pairs<LAT, LN>(C);
            const T phi = raw[C + 1];
            const T m2 = (((cf.m2[4] * phi + cf.m2[3]) * phi + cf.m2[2]) * phi + cf.m2[1]) * phi + cf.m2[0];
            T B[2];
#pragma unroll
            for (int a = 0; a < 2; ++a)
                B[a] = ((cf.flux[a][3] * phi + cf.flux[a][2]) * phi + cf.flux[a][1]) * phi + cf.flux[a][0];
            if constexpr (OWN) {
                const T rest = cf.rM2 * m2 + cf.rPhi * phi;
                accC[C] += cf.ap[0] * rest + cf.a0[0] * phi;
            }
            T E[4], O[4];
            pair_eo<LAT, PDE, MASK>(cf, phi, B, m2, T(0), T(0), T(0), E, O);
            static_for<0, NP>([&](auto pcc) {
                constexpr int P_ = decltype(pcc)::value;
                constexpr int EX = pair_e(LAT, P_, 0), EY = pair_e(LAT, P_, 1);
                constexpr int TP = C - EX, TM = C + EX;
                constexpr bool HP = TP >= 0 && TP < LN, HM = TM >= 0 && TM < LN;
                if constexpr (HP || HM) {
                    const T sE = cf.ap[0] * E[P_];
                    if constexpr (HP) {
                        const T sv = cf.am[0] * O[P_] + sE;
                        if constexpr (EY == 1) accP[TP] += sv;
                        else accC[TP] += sv;
                    }
                    if constexpr (HM) {
                        const T sv = sE - cf.am[0] * O[P_];
                        if constexpr (EY == 1) accN[TM] += sv;
                        else accC[TM] += sv;
                    }
                }
            });
        }
    });
}

template <int LAT, int PDE, int ST, int TT, int NW, int NSTAGE, bool JAC>
__global__ void __launch_bounds__(NW * 32) k_march2d_tb(const __grid_constant__ TmapSet maps, Geom g,
                                                        void* __restrict__ outv, Coef<typename Storage<ST>::T> cf,
                                                        StepExtra ex, int H, int nitems, int* __restrict__ err,
                                                        const typename Storage<ST>::S* __restrict__ rhs,
                                                        typename Storage<ST>::T jw) {
    using Tr = Storage<ST>;
    using S = typename Tr::S;
    using T = typename Tr::T;
    constexpr int LN = 4;
    constexpr int ES = (int)sizeof(S);
    constexpr int ALIGN = 16 / ES;
    constexpr int COLS = 32 * LN;
    constexpr int BOXW = COLS + 2 * ALIGN;
    constexpr int RPS = 2;                                  // input rows per stage (box height)
    constexpr int ROWB = BOXW * ES;
    constexpr int SLOT = ((RPS * ROWB + 127) / 128) * 128;
    constexpr uint32_t kTx = (uint32_t)(RPS * ROWB);
    constexpr size_t kRingBytes = (size_t)NSTAGE * SLOT;
    static_assert(TT >= 2 && TT <= 5, "the 8-column strip overlap supports 2 .. 5 levels");
    static_assert(TT <= ALIGN, "ghost columns of 16 bytes hold at most 16 / sizeof(S) levels");
    static_assert(!JAC || (PDE == PDE_LCDE && ST != ST_BF16), "Jacobi sweeps: LCDE, FP32 / FP64 levels");

    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem) + warp * NSTAGE;
    unsigned char* ring = smem + 128 * ((NW * NSTAGE * 8 + 127) / 128) + warp * kRingBytes;

    const int strips = (g.nx + kTbLead / 2 + kTbStride - 1) / kTbStride;
    const int wstride = gridDim.x * NW;
    const int wid = blockIdx.x * NW + warp;
    if (wid >= nitems) return;

    // producer (lane 0): the item's box column (padded coordinates: X0 - ALIGN + ox = X0, a
    // multiple of 8 elements) and first input row, advanced per item
    int p_item = wid, p_row = 0, p_rows = 0, p_xcol = 0, p_y = 0;
    auto p_load_item = [&]() {
        if (p_item < nitems) {
            const int seg = p_item / strips;
            p_xcol = (p_item - seg * strips) * kTbStride - kTbLead;
            p_y = seg * H - TT;
            p_rows = (min(H, g.ny - seg * H) + 2 * TT + RPS - 1) / RPS * RPS;
        }
    };
    p_load_item();
    int ps = 0;
    long long issued = 0;
    auto issue_next = [&]() {
        if (p_item >= nitems) return;
        const int y = p_y + p_row;
        const int yw = y < 0 ? y + g.ny : (y >= g.ny ? y - g.ny : y);   // periodic in y
        mbar_arrive_expect_tx(&full[ps], kTx);
        tma_load_2d(ring + (size_t)ps * SLOT, &maps.m[0], &full[ps], p_xcol, yw + 1);
        ++issued;
        ps = ps + 1 == NSTAGE ? 0 : ps + 1;
        p_row += RPS;
        if (p_row == p_rows) {
            p_item += wstride;
            p_row = 0;
            p_load_item();
        }
    };

    if (lane == 0) {
#pragma unroll
        for (int s = 0; s < NSTAGE; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
        tma_prefetch_desc(&maps.m[0]);
        for (int k = 0; k < NSTAGE; ++k) issue_next();
    }
    __syncwarp();

    // accumulators: level t holds rows (P, C, N) = (r-1, r, r+1) of its current input row r.
    // (Unrolling the row loop three times to rotate the sets by renaming ran slower: more
    // instructions and registers, fewer resident CTAs.)
    T accP[TT][LN], accC[TT][LN], accN[TT][LN];
    S* out = static_cast<S*>(outv);
    int cs = 0;
    uint32_t cphase = 0;
    long long consumed = 0;
    bool failed = false;
    const bool store_lane = lane >= 1 && lane <= 30;

    // the lane's LN right-hand-side values of row y (periodic in y).  Columns off the padded row
    // [-ox, py - ox) take zero; a vector that straddles its ends (the ghost columns are narrower
    // than a lane's four nodes in FP64) is read node by node.
    [[maybe_unused]] auto rhs_row = [&](int y, int xb, T (&rv)[LN]) {
        if constexpr (JAC) {
        int yw = y % g.ny;
        if (yw < 0) yw += g.ny;
        const S* row = rhs + g.at(0, yw, 0);
        if (xb >= -g.ox && xb + LN <= g.py - g.ox) {
            if constexpr (sizeof(S) == 4) {
                const float4 q = __ldg(reinterpret_cast<const float4*>(row + xb));
                rv[0] = q.x; rv[1] = q.y; rv[2] = q.z; rv[3] = q.w;
            } else {
                const double2 q0 = __ldg(reinterpret_cast<const double2*>(row + xb));
                const double2 q1 = __ldg(reinterpret_cast<const double2*>(row + xb + 2));
                rv[0] = q0.x; rv[1] = q0.y; rv[2] = q1.x; rv[3] = q1.y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < LN; ++k) {
                const int x = xb + k;
                rv[k] = (x >= -g.ox && x < g.py - g.ox) ? __ldg(row + x) : T(0);
            }
        }
        }
    };

    // Jacobi right-hand side: rwin[t] holds row r - 1 - t for the current input row r (the row
    // level t completes), rnext row r, loaded one input row before it is needed
    [[maybe_unused]] T rwin[TT][LN];
    [[maybe_unused]] T rnext[LN];

    // input row i of the item at (xb, y0): push it through the TT levels and store the completed
    // level-TT row y0 - 2 TT + i if it is one of the item's output rows
    EdgeStore<2, ST> es;
    auto cascade = [&](T (&raw)[LN + 2], int i, int xb, int y0, int hrows) {
#pragma unroll
        for (int t = 0; t < TT; ++t) {
            if (t > 0) {
                raw[0] = __shfl_up_sync(0xffffffffu, raw[LN], 1);
                raw[LN + 1] = __shfl_down_sync(0xffffffffu, raw[1], 1);
            }
            tb_push_row<LAT, PDE, T, LN>(cf, raw, accP[t], accC[t], accN[t]);
#pragma unroll
            for (int k = 0; k < LN; ++k) {
                raw[1 + k] = accP[t][k];   // row r-1 of level t + 1 is complete
                accP[t][k] = accC[t][k];
                accC[t][k] = accN[t][k];
                accN[t][k] = acc_zero<T>();
            }
            if constexpr (JAC) {
#pragma unroll
                for (int k = 0; k < LN; ++k) raw[1 + k] += jw * rwin[t][k];
            }
        }
        if constexpr (JAC) {
            // advance the window to input row i + 1 and fetch the row input row i + 2 starts with
#pragma unroll
            for (int t = TT - 1; t > 0; --t)
#pragma unroll
                for (int k = 0; k < LN; ++k) rwin[t][k] = rwin[t - 1][k];
#pragma unroll
            for (int k = 0; k < LN; ++k) rwin[0][k] = rnext[k];
            rhs_row(y0 - TT + i + 1, xb, rnext);
        }
        const int yo = y0 - 2 * TT + i;
        if (i >= 2 * TT && i < hrows + 2 * TT) {   // warp-uniform; lanes 0 and 31 hold no output
            const long long nb = (long long)yo * g.nx;
            S sv[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const unsigned rnd = ex.sr ? sr_bits(ex.seed, ex.step, nb + xb + k, 0) : 0u;
                sv[k] = kpack<ST, PDE>(raw[1 + k], cf.ref[0], rnd);
            }
            es.put(out, g, xb, yo, 0, sv);
        }
    };

    auto load_row = [&](const unsigned char* base, T (&raw)[LN + 2]) {
        const S* sp = reinterpret_cast<const S*>(base);
        T v4[4];
        lds4<ST, PDE>(base + (size_t)(ALIGN + lane * LN) * ES, cf.ref[0], v4);
        raw[1] = v4[0];
        raw[2] = v4[1];
        raw[3] = v4[2];
        raw[4] = v4[3];
        raw[0] = kload<ST, PDE>(sp + ALIGN + lane * LN - 1, cf.ref[0]);
        raw[LN + 1] = kload<ST, PDE>(sp + ALIGN + lane * LN + LN, cf.ref[0]);
    };

    for (int item = wid; item < nitems && !failed; item += wstride) {
        const int seg = item / strips;
        const int x0 = (item - seg * strips) * kTbStride - kTbLead;
        const int y0 = seg * H;
        const int hrows = min(H, g.ny - y0);
        const int nrows = (hrows + 2 * TT + RPS - 1) / RPS * RPS;
        const int xb = x0 + lane * LN;
        es.init(g, xb, store_lane);
#pragma unroll
        for (int t = 0; t < TT; ++t)
#pragma unroll
            for (int k = 0; k < LN; ++k) accP[t][k] = accC[t][k] = accN[t][k] = acc_zero<T>();
        if constexpr (JAC) {
#pragma unroll
            for (int t = 0; t < TT; ++t) rhs_row(y0 - TT - 1 - t, xb, rwin[t]);
            rhs_row(y0 - TT, xb, rnext);
        }
        for (int i = 0; i < nrows; i += RPS) {
            const bool ok = mbar_wait_bounded(&full[cs], cphase);
            if (__any_sync(0xffffffffu, !ok)) {
                failed = true;
                break;
            }
            T rawA[LN + 2], rawB[LN + 2];
            load_row(ring + (size_t)cs * SLOT, rawA);
            load_row(ring + (size_t)cs * SLOT + ROWB, rawB);
            ++consumed;
            cs = cs + 1 == NSTAGE ? 0 : cs + 1;
            if (cs == 0) cphase ^= 1u;
            __syncwarp();
            if (lane == 0) {
                fence_proxy_async_smem();
                issue_next();
            }
            cascade(rawA, i, xb, y0, hrows);
            cascade(rawB, i + 1, xb, y0, hrows);
        }
    }
    if (failed && lane == 0) {
        atomicExch(err, KERR_TMA_TIMEOUT);
        for (long long k = consumed; k < issued; ++k) {
            const int s = (int)(k % NSTAGE);
            mbar_wait_bounded(&full[s], (uint32_t)((k / NSTAGE) & 1));
        }
    }
}

template <int ST, int NW, int NSTAGE>
constexpr size_t tb_smem() {
    constexpr int ES = ST == ST_F64 ? 8 : (ST == ST_F32 ? 4 : 2);
    constexpr int SLOT = ((2 * (128 + 2 * (16 / ES)) * ES + 127) / 128) * 128;
    return 128 + 128 * ((NW * NSTAGE * 8 + 127) / 128) + (size_t)NW * NSTAGE * SLOT;
}

template <int LAT, int PDE, int ST, int TT, bool JAC>
cudaError_t launch_tb(const LaunchArgs& a) {
    using T = typename Storage<ST>::T;
    using S = typename Storage<ST>::S;
    constexpr int NW = 4;
    constexpr int ES = ST == ST_F64 ? 8 : (ST == ST_F32 ? 4 : 2);
    constexpr int PER = ((2 * (128 + 2 * (16 / ES)) * ES + 127) / 128) * 128;
    constexpr int NSTAGE = 8192 / PER < 3 ? 3 : (8192 / PER > 12 ? 12 : 8192 / PER);
    constexpr size_t smem = tb_smem<ST, NW, NSTAGE>();
    auto kern = k_march2d_tb<LAT, PDE, ST, TT, NW, NSTAGE, JAC>;
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
    const int strips = (a.g.nx + kTbLead / 2 + kTbStride - 1) / kTbStride;
    int H = a.H;
    if (H <= 0) {
        // rows per item: maximise (output rows / streamed rows) x (fill of the resident warp slots)
        const long long wslots = (long long)resident * NW;
        double best = -1.0;
        for (int h = 8; h <= 512; ++h) {
            const long long items = (long long)strips * ((a.g.ny + h - 1) / h);
            const long long rounds = (items + wslots - 1) / wslots;
            const double fill = (double)items / (double)(rounds * wslots);
            const double eff = fill * (double)h / (double)(h + 2 * TT);
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
    const S* rhs = nullptr;
    T jw = T(0);
    if constexpr (JAC) {
        rhs = static_cast<const S*>(a.src[0]);
        jw = static_cast<const SrcCoef<T>*>(a.src_coef)->W0[0];
    }
    kern<<<grid, NW * 32, smem, a.stream>>>(*a.maps, a.g, a.out, *static_cast<const Coef<T>*>(a.coef), a.ex, H,
                                             nitems, a.err, rhs, jw);
    return cudaGetLastError();
}

template <int LAT, int PDE, int ST, bool JAC = false>
LaunchFn pick_depth(int depth) {
    if (depth == 2) return launch_tb<LAT, PDE, ST, 2, JAC>;
    if constexpr (ST != ST_F64) {
        if (depth == 3) return launch_tb<LAT, PDE, ST, 3, JAC>;
        if (depth == 4) return launch_tb<LAT, PDE, ST, 4, JAC>;
    }
    if constexpr (ST == ST_BF16) {
        if (depth == 5) return launch_tb<LAT, PDE, ST, 5, JAC>;
    }
    return nullptr;
}

template <int LAT>
LaunchFn pick_jac(int st, int depth) {
    if (st == ST_F64) return pick_depth<LAT, PDE_LCDE, ST_F64, true>(depth);
    if (st == ST_F32) return pick_depth<LAT, PDE_LCDE, ST_F32, true>(depth);
    return nullptr;
}

template <int LAT, int PDE>
LaunchFn pick_st(int st, int depth) {
    if (st == ST_F64) return pick_depth<LAT, PDE, ST_F64>(depth);
    if (st == ST_F32) return pick_depth<LAT, PDE, ST_F32>(depth);
    if (st == ST_BF16) return pick_depth<LAT, PDE, ST_BF16>(depth);
    return nullptr;
}

}  // namespace

int march2d_tb_max_depth(int st) { return st == ST_F64 ? 2 : (st == ST_F32 ? 4 : 5); }

LaunchFn find_march2d_tb(int lat, int pde, int levels, int st, int depth) {
    if (levels != 2 || depth < 2) return nullptr;
    if (lat == LAT_D2Q5) return pde == PDE_LCDE ? pick_st<LAT_D2Q5, PDE_LCDE>(st, depth) : nullptr;
    if (lat == LAT_D2Q9) {
        if (pde == PDE_LCDE) return pick_st<LAT_D2Q9, PDE_LCDE>(st, depth);
        if (pde == PDE_NCDE) return pick_st<LAT_D2Q9, PDE_NCDE>(st, depth);
    }
    return nullptr;
}

LaunchFn find_march2d_tb_jacobi(int lat, int st, int depth) {
    if (depth < 2) return nullptr;
    if (lat == LAT_D2Q5) return pick_jac<LAT_D2Q5>(st, depth);
    if (lat == LAT_D2Q9) return pick_jac<LAT_D2Q9>(st, depth);
    return nullptr;
}

}  // namespace mmfd
