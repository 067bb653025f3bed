// k_march2d_tb_nse.cu -- temporally blocked 2D He-Luo NSE steps: D2Q9, two levels, the lean
// streaming form (Coef::nA with streaming momentum), FP32 or BF16 storage.  One launch advances
// TT time levels and reads / writes the stored level (rho, ux, uy) once.
//
// The layout of k_march2d_tb (the scalar blocked kernel) with three fields:
// - A warp owns items of one 128-column strip x H output rows. It streams the input rows
//   y0-TT .. y0+H+TT-1 of the three fields, two rows per stage, through its private TMA ring;
//   rows wrap periodically in y in the producer.
// - It keeps TT sets of three accumulator rows of the three fields. An input row is pushed into
//   level 1 with the node update of the marching kernel (lean_push_node2d); the level-1 row it
//   completes is pushed into level 2; and so on -- a wavefront of TT steps one row apart.
// - The pushes that cross into a neighbouring lane's columns come from that lane by shuffle, at
//   every level (tb_push_row), so no lane evaluates a halo node.  Strips overlap: lanes cover
//   columns X0 .. X0+127 (X0 = 120 s - 8), lanes 1 .. 30 store.  Lanes 0 and 31 receive their
//   own values in place of the missing neighbours: at level t the first (last) t columns of
//   lane 0 (31) are wrong, which lane 1 (30) does not read for t < 4.
// - Columns within TT of the x edges are read from the ghost columns, which every writer keeps
//   current to the ghost depth.
// - Intermediate levels stay in FP32 (never stored), so BF16 storage rounds once per TT steps.
// The registers hold 3 x TT x 12 accumulators: TT is 2 or 3.
#include "k_march2d.cuh"

namespace mmfd {

namespace {

constexpr int kTbnStride = 120;   // output columns per strip
constexpr int kTbnLead = 8;       // lane 0's first column lies kTbnLead columns left of the strip's output

// The lane's LN input nodes of one row at one level, pushed into the accumulators of the output
// rows r-1 (P), r (C) and r+1 (N).  The pushes that land one column outside the lane's window are
// not recomputed by the neighbouring lane from a halo node: lane l hands the contributions of its
// node LN-1 to lane l+1's column 0 and those of its node 0 to lane l-1's column LN-1 by shuffle.
// Every accumulator still receives its contributions in the order of their input column (the left
// neighbour's first, the right neighbour's last), with the expressions of lean_push_node2d, so
// this kernel and the one-step marching kernel round alike.  Lanes 0 and 31 get their own values
// in place of the missing neighbours; they hold no output.
template <int LN, typename T>
__device__ __forceinline__ void tb_push_row(const Coef<T>& cf, const T (&raw)[LN + 2][3], T (&accP)[LN][3],
                                            T (&accC)[LN][3], T (&accN)[LN][3]) {
    constexpr int LAT = LAT_D2Q9;
    constexpr unsigned FULL = 0xffffffffu;
    {
        // node LN-1 -> column LN: pair x minus (row r), (1,1) minus (row r+1), (-1,1) plus (row r-1)
        const T* f = raw[LN];
        const T U = lean_u2(f[1], f[2]);
        T c0, E0, c2, E2, c3, E3;
        lean_e2d<LAT, 0>(cf, 0, f[1], f[2], lean_base(cf, 0, 0, U, f[0]), c0, E0);
        const T b1 = lean_base(cf, 0, 1, U, f[0]);
        lean_e2d<LAT, 2>(cf, 0, f[1], f[2], b1, c2, E2);
        lean_e2d<LAT, 3>(cf, 0, f[1], f[2], b1, c3, E3);
        const T vC = __shfl_up_sync(FULL, lean_sv2d<0, -1>(cf, 0, c0, E0), 1);
        const T vN = __shfl_up_sync(FULL, lean_sv2d<2, -1>(cf, 0, c2, E2), 1);
        const T vP = __shfl_up_sync(FULL, lean_sv2d<3, 1>(cf, 0, c3, E3), 1);
        lean_push_sv<LAT, 0, -1>(accC[0], cf, 0, vC);
        lean_push_sv<LAT, 2, -1>(accN[0], cf, 0, vN);
        lean_push_sv<LAT, 3, 1>(accP[0], cf, 0, vP);
    }
    static_for<0, LN>([&](auto cc) {
        constexpr int C = decltype(cc)::value;
        lean_push_node2d<LAT, LEAN_STREAM, LN, C>(cf, 0, raw[C + 1], accP, accC, accN);
    });
    {
        // node 0 -> column -1: pair x plus (row r), (1,1) plus (row r-1), (-1,1) minus (row r+1)
        const T* f = raw[1];
        const T U = lean_u2(f[1], f[2]);
        T c0, E0, c2, E2, c3, E3;
        lean_e2d<LAT, 0>(cf, 0, f[1], f[2], lean_base(cf, 0, 0, U, f[0]), c0, E0);
        const T b1 = lean_base(cf, 0, 1, U, f[0]);
        lean_e2d<LAT, 2>(cf, 0, f[1], f[2], b1, c2, E2);
        lean_e2d<LAT, 3>(cf, 0, f[1], f[2], b1, c3, E3);
        const T vC = __shfl_down_sync(FULL, lean_sv2d<0, 1>(cf, 0, c0, E0), 1);
        const T vP = __shfl_down_sync(FULL, lean_sv2d<2, 1>(cf, 0, c2, E2), 1);
        const T vN = __shfl_down_sync(FULL, lean_sv2d<3, -1>(cf, 0, c3, E3), 1);
        lean_push_sv<LAT, 0, 1>(accC[LN - 1], cf, 0, vC);
        lean_push_sv<LAT, 2, 1>(accP[LN - 1], cf, 0, vP);
        lean_push_sv<LAT, 3, -1>(accN[LN - 1], cf, 0, vN);
    }
}

template <int ST, int TT, int NW, int NSTAGE, int SRM>
__global__ void __launch_bounds__(NW * 32) k_march2d_tb_nse(const __grid_constant__ TmapSet maps, Geom g,
                                                            void* __restrict__ outv, Coef<typename Storage<ST>::T> cf,
                                                            StepExtra ex, int H, int nitems, int* __restrict__ err) {
    using Tr = Storage<ST>;
    using S = typename Tr::S;
    using T = typename Tr::T;
    constexpr int LAT = LAT_D2Q9;
    constexpr int PDE = PDE_NSE;
    constexpr int NF = 3;
    constexpr int LN = 4;
    constexpr int ES = (int)sizeof(S);
    constexpr int ALIGN = 16 / ES;
    constexpr int COLS = 32 * LN;
    constexpr int BOXW = COLS + 2 * ALIGN;
    constexpr int RPS = 2;                                  // input rows per stage (box height)
    constexpr int ROWB = BOXW * ES;
    constexpr int SLOT = ((RPS * ROWB + 127) / 128) * 128;  // one field of one stage
    constexpr uint32_t kTx = (uint32_t)(NF * RPS * ROWB);
    constexpr size_t kRingBytes = (size_t)NSTAGE * NF * SLOT;
    static_assert(TT >= 2 && TT <= 3, "three fields: at most three levels in registers");
    static_assert(TT < LN, "the wrong columns of the edge lanes must not reach lanes 1 and 30");
    static_assert(TT <= ALIGN, "ghost columns of 16 bytes hold at most 16 / sizeof(S) levels");
    static_assert(ST == ST_F32 || ST == ST_BF16, "the lean form runs in FP32 arithmetic");

    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem) + warp * NSTAGE;
    unsigned char* ring = smem + 128 * ((NW * NSTAGE * 8 + 127) / 128) + warp * kRingBytes;
    auto slot = [&](int s, int f) -> unsigned char* { return ring + (size_t)(s * NF + f) * SLOT; };

    const int strips = (g.nx + kTbnLead / 2 + kTbnStride - 1) / kTbnStride;
    const int wstride = gridDim.x * NW;
    const int wid = blockIdx.x * NW + warp;
    if (wid >= nitems) return;

    // producer (lane 0): the item's box column (padded coordinates) and first input row
    int p_item = wid, p_row = 0, p_rows = 0, p_xcol = 0, p_y = 0;
    auto p_load_item = [&]() {
        if (p_item < nitems) {
            const int seg = p_item / strips;
            p_xcol = (p_item - seg * strips) * kTbnStride - kTbnLead;
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
#pragma unroll
        for (int f = 0; f < NF; ++f) tma_load_2d(slot(ps, f), &maps.m[f], &full[ps], p_xcol, yw + 1);
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
#pragma unroll
        for (int f = 0; f < NF; ++f) tma_prefetch_desc(&maps.m[f]);
        for (int k = 0; k < NSTAGE; ++k) issue_next();
    }
    __syncwarp();

    // accumulators: level t holds rows (P, C, N) = (r-1, r, r+1) of its current input row r
    T accP[TT][LN][NF], accC[TT][LN][NF], accN[TT][LN][NF];
    S* out = static_cast<S*>(outv);
    int cs = 0;
    uint32_t cphase = 0;
    long long consumed = 0;
    bool failed = false;
    const bool store_lane = lane >= 1 && lane <= 30;

    // input row i of the item at (xb, y0): push it through the TT levels and store the completed
    // level-TT row y0 - 2 TT + i if it is one of the item's output rows
    EdgeStore<2, ST> es;
    auto cascade = [&](T (&raw)[LN + 2][NF], int i, int xb, int y0, int hrows) {
#pragma unroll
        for (int t = 0; t < TT; ++t) {
            tb_push_row<LN>(cf, raw, accP[t], accC[t], accN[t]);
#pragma unroll
            for (int k = 0; k < LN; ++k)
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    raw[1 + k][f] = accP[t][k][f];   // row r-1 of level t + 1 is complete
                    accP[t][k][f] = accC[t][k][f];
                    accC[t][k][f] = accN[t][k][f];
                    accN[t][k][f] = acc_zero<T>();
                }
        }
        const int yo = y0 - 2 * TT + i;
        if (i >= 2 * TT && i < hrows + 2 * TT) {   // warp-uniform; lanes 0 and 31 hold no output
            const long long nb = (long long)yo * g.nx;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                S sv[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const unsigned rnd = sr_on<SRM>(ex) ? sr_bits(ex.seed, ex.step, nb + xb + k, f) : 0u;
                    sv[k] = kpack<ST, PDE>(raw[1 + k][f], cf.ref[f], rnd);
                }
                es.put(out + (size_t)f * g.fs, g, xb, yo, 0, sv);
            }
        }
    };

    auto load_row = [&](int s, int j, T (&raw)[LN + 2][NF]) {
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const unsigned char* base = slot(s, f) + (size_t)j * ROWB;
            T v4[4];
            lds4<ST, PDE>(base + (size_t)(ALIGN + lane * LN) * ES, cf.ref[f], v4);
            raw[1][f] = v4[0];
            raw[2][f] = v4[1];
            raw[3][f] = v4[2];
            raw[4][f] = v4[3];
        }
    };

    for (int item = wid; item < nitems && !failed; item += wstride) {
        const int seg = item / strips;
        const int x0 = (item - seg * strips) * kTbnStride - kTbnLead;
        const int y0 = seg * H;
        const int hrows = min(H, g.ny - y0);
        const int nrows = (hrows + 2 * TT + RPS - 1) / RPS * RPS;
        const int xb = x0 + lane * LN;
        es.init(g, xb, store_lane);
#pragma unroll
        for (int t = 0; t < TT; ++t)
#pragma unroll
            for (int k = 0; k < LN; ++k)
#pragma unroll
                for (int f = 0; f < NF; ++f) accP[t][k][f] = accC[t][k][f] = accN[t][k][f] = acc_zero<T>();
        for (int i = 0; i < nrows; i += RPS) {
            const bool ok = mbar_wait_bounded(&full[cs], cphase);
            if (__any_sync(0xffffffffu, !ok)) {
                failed = true;
                break;
            }
            T rawA[LN + 2][NF], rawB[LN + 2][NF];
            load_row(cs, 0, rawA);
            load_row(cs, 1, rawB);
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
constexpr size_t tbn_smem() {
    constexpr int ES = ST == ST_F32 ? 4 : 2;
    constexpr int SLOT = ((2 * (128 + 2 * (16 / ES)) * ES + 127) / 128) * 128;
    return 128 + 128 * ((NW * NSTAGE * 8 + 127) / 128) + (size_t)NW * NSTAGE * 3 * SLOT;
}

template <int ST, int TT, int SRM>
cudaError_t launch_tbn_t(const LaunchArgs& a) {
    using T = typename Storage<ST>::T;
    constexpr int NW = 4;
    constexpr int NSTAGE = 3;
    constexpr size_t smem = tbn_smem<ST, NW, NSTAGE>();
    auto kern = k_march2d_tb_nse<ST, TT, NW, NSTAGE, SRM>;
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
    const int strips = (a.g.nx + kTbnLead / 2 + kTbnStride - 1) / kTbnStride;
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
    kern<<<grid, NW * 32, smem, a.stream>>>(*a.maps, a.g, a.out, *static_cast<const Coef<T>*>(a.coef), a.ex, H,
                                             nitems, a.err);
    return cudaGetLastError();
}

// stochastic rounding chosen per launch: BF16 has a kernel without and one with the rounding code
template <int ST, int TT>
cudaError_t launch_tbn(const LaunchArgs& a) {
    if constexpr (ST == ST_BF16) {
        if (a.ex.sr) return launch_tbn_t<ST, TT, 1>(a);
    }
    return launch_tbn_t<ST, TT, 0>(a);
}

}  // namespace

int march2d_tb_nse_max_depth() { return 3; }

LaunchFn find_march2d_tb_nse(int st, int depth) {
    if (st == ST_F32) return depth == 2 ? launch_tbn<ST_F32, 2> : depth == 3 ? launch_tbn<ST_F32, 3> : nullptr;
    if (st == ST_BF16) return depth == 2 ? launch_tbn<ST_BF16, 2> : depth == 3 ? launch_tbn<ST_BF16, 3> : nullptr;
    return nullptr;
}

}  // namespace mmfd
