// k_march3d_tb.cu -- temporally blocked 3D MMFD steps for the two-level linear CDE (D3Q7,
// D3Q19): one launch advances TT time levels and reads / writes the stored level once.
//
// A CTA owns items of one x strip (the 128 columns X0 .. X0+127, X0 = 120 s - 8, as in the 2D
// blocked kernel) x TYH tile rows (output rows y0 .. y0+TYH-2TT-1 plus TT halo rows on each side)
// x H output planes, and marches in z.  It has TYH row warps and one producer warp.  The
// producer's lane 0 streams the input planes z0-TT .. z0+H+TT-1 of the level, one TMA box
// (128 + 2 x 16 bytes) x 1 row x 1 plane per tile row, with rows and planes wrapped
// periodically in the coordinates it issues, into a full/empty mbarrier ring.  Every row warp
// keeps three register accumulator planes (z-1, z, z+1) per time level: it pulls the x and y
// neighbours of its four nodes per lane from the staged level-0 plane and pushes them into
// level 1; a level-k plane that is complete is written to a double-buffered shared-memory plane,
// and after a named barrier of the row warps it is pulled, with its y neighbours, into level
// k+1.  The tile loses one row per level at each side and the strip one column per level;
// warps TT .. TYH-TT-1 and lanes 1 .. 30 store the level-TT plane.  Columns within TT of the
// domain's x edges come from the ghost columns, kept current to depth TT by every writer.  Every
// wait is bounded: a warp whose wait runs out records KERR_TMA_TIMEOUT in a shared flag that all
// row warps read after the plane's first barrier, so they leave together; the producer waits
// (bounded) for the copies still in flight into the CTA before it leaves.
#include "k_march3d.cuh"

namespace mmfd {

namespace {

constexpr int kTbStride = 120;   // output columns per strip
constexpr int kTbLead = 8;       // lane 0's first column lies kTbLead columns left of the strip's output

// Four consecutive values into a level plane (16-byte aligned for FP32, 32-byte for FP64).
__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void st4(double* p, double a, double b, double c, double d) {
    reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
    reinterpret_cast<double2*>(p)[1] = make_double2(c, d);
}

__device__ __forceinline__ void ld4(const float* p, float& a, float& b, float& c, float& d) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    a = q.x; b = q.y; c = q.z; d = q.w;
}
__device__ __forceinline__ void ld4(const double* p, double& a, double& b, double& c, double& d) {
    const double2 q0 = reinterpret_cast<const double2*>(p)[0], q1 = reinterpret_cast<const double2*>(p)[1];
    a = q0.x; b = q0.y; c = q1.x; d = q1.y;
}

__device__ __forceinline__ void rows_barrier(int threads) {
    asm volatile("bar.sync 1, %0;" ::"r"(threads) : "memory");
}

// Push one plane of the level below (the six values xb-1 .. xb+4 of rows y-1, y, y+1) into the
// accumulators of planes z-1 (P), z (C), z+1 (N): the collapsed LCDE stencil of the two-level
// scheme (one input level, weights W0, Wp, Wm).
template <int LAT, typename T>
__device__ __forceinline__ void tb3_push(const Coef<T>& cf, const T (&raw)[3][6], T (&accP)[4], T (&accC)[4],
                                         T (&accN)[4]) {
    constexpr int NP = lat_npair(LAT);
#pragma unroll
    for (int k = 0; k < 4; ++k) accC[k] += cf.W0[0] * raw[1][k + 1];
    static_for<0, NP>([&](auto pc) {
        constexpr int P = decltype(pc)::value;
        constexpr int EX = pair_e(LAT, P, 0), EY = pair_e(LAT, P, 1), EZ = pair_e(LAT, P, 2);
        // output node (x, y, z) takes Wp * phi(x + e) and Wm * phi(x - e); in-plane parts go to the
        // plane of the input, the z parts to the planes below (plus) and above (minus) it
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const T vp = raw[1 + EY][k + 1 + EX];   // phi(x + e) for the node's own plane ...
            const T vm = raw[1 - EY][k + 1 - EX];   // ... and phi(x - e)
            if constexpr (EZ == 0) {
                accC[k] += cf.Wp[0][P] * vp + cf.Wm[0][P] * vm;
            } else {
                // with e_z = 1 the input plane z is x + e for plane z - 1 and x - e for plane z + 1
                accP[k] += cf.Wp[0][P] * vp;
                accN[k] += cf.Wm[0][P] * vm;
            }
        }
    });
}

template <int LAT, int ST, int TT, int TYH, int NSTAGE>
__global__ void __launch_bounds__((TYH + 1) * 32) k_march3d_tb(const __grid_constant__ TmapSet maps, Geom g,
                                                               void* __restrict__ outv,
                                                               Coef<typename Storage<ST>::T> cf, StepExtra ex,
                                                               int H, int nitems, int* __restrict__ err) {
    using Tr = Storage<ST>;
    using S = typename Tr::S;
    using T = typename Tr::T;
    constexpr int LN = 4;
    constexpr int ES = (int)sizeof(S);
    constexpr int ALIGN = 16 / ES;
    constexpr int BOXW = 128 + 2 * ALIGN;
    constexpr int ROWB = BOXW * ES;                               // bytes per staged row (16-byte multiple)
    constexpr int ROWP = ((ROWB + 127) / 128) * 128;              // row pitch in the ring: each row is its
                                                                  // own TMA box, whose destination must
                                                                  // start on a 128-byte boundary
    constexpr int SLOT = ROWP * TYH;                              // bytes per ring stage (one plane)
    constexpr uint32_t kTx = (uint32_t)(ROWB * TYH);
    constexpr int TY = TYH - 2 * TT;                              // output rows per tile
    constexpr int LROW = 136;                                     // level-plane row: columns -4 .. 131
    constexpr int LPLANE = LROW * TYH;                            // elements per level plane
    static_assert(TT >= 2 && TT <= 5 && TT <= ALIGN, "the strip overlap and ghost columns bound the depth");
    static_assert(TY >= 1, "the tile must keep output rows");

    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + NSTAGE;
    int* sflag = reinterpret_cast<int*>(empty + NSTAGE);
    unsigned char* ring = smem + 128 * ((2 * NSTAGE * 8 + 4 + 127) / 128);
    T* lev = reinterpret_cast<T*>(ring + (size_t)NSTAGE * SLOT);  // (TT - 1) levels x 2 buffers

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int strips = (g.nx + kTbLead / 2 + kTbStride - 1) / kTbStride;
    const int ytiles = (g.ny + TY - 1) / TY;
    auto wrap = [](int i, int n) { int r = i % n; return r < 0 ? r + n : r; };

    if (threadIdx.x == 0) {
#pragma unroll
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], TYH);
        }
        *sflag = 0;
        fence_mbar_init();
        tma_prefetch_desc(&maps.m[0]);
    }
    // the level planes' halo columns are read (by the strip's outer lanes, whose results are never
    // stored) but never written: start them at zero
    for (int i = threadIdx.x; i < (TT - 1) * 2 * LPLANE; i += blockDim.x) lev[i] = T(0);
    __syncthreads();

    if (warp == TYH) {
        // ---------------------------------------------------------------- producer warp
        // lane 0 waits for the free stage and sets its byte count; lanes 0 .. TYH-1 then issue one
        // row each (the copies of a plane go out in parallel)
        static_assert(TYH <= 32, "one producer lane per tile row");
        long long k = 0;
        bool failed = false;
        for (int item = blockIdx.x; item < nitems && !failed; item += gridDim.x) {
            const int s_ = item % strips;
            const int yt = (item / strips) % ytiles;
            const int zs = item / (strips * ytiles);
            const int xcol = s_ * kTbStride - kTbLead;            // padded column of the box (X0)
            const int y0 = yt * TY - TT;                           // interior row of tile row 0
            const int z0 = zs * H - TT;                            // interior plane of input plane 0
            const int np = min(H, g.nz - zs * H) + 2 * TT;
            for (int i = 0; i < np; ++i, ++k) {
                const int s = (int)(k % NSTAGE);
                bool ok = true;
                if (lane == 0) {
                    ok = mbar_wait_bounded(&empty[s], (uint32_t)(((k / NSTAGE) & 1) ^ 1));
                    if (ok) {
                        fence_proxy_async_smem();
                        mbar_arrive_expect_tx(&full[s], kTx);
                    }
                }
                if (!__shfl_sync(0xffffffffu, ok, 0)) {
                    failed = true;
                    break;
                }
                if (lane < TYH) {
                    const int zp = wrap(z0 + i, g.nz) + g.gz;
                    tma_load_3d(ring + (size_t)s * SLOT + (size_t)lane * ROWP, &maps.m[0], &full[s], xcol,
                                wrap(y0 + lane, g.ny) + 1, zp);
                }
            }
        }
        if (lane == 0) {
            if (failed) atomicExch(err, KERR_TMA_TIMEOUT);
            // do not leave while copies into this CTA's shared memory may still land
            const long long first = k > NSTAGE ? k - NSTAGE : 0;
            for (long long j = first; j < k; ++j)
                mbar_wait_bounded(&full[j % NSTAGE], (uint32_t)((j / NSTAGE) & 1));
        }
        return;
    }

    // -------------------------------------------------------------------- row warps
    T acc[TT][3][LN];   // per level: planes z-1 (0), z (1), z+1 (2) of the level's current input plane
    EdgeStore<3, ST> es;
    S* out = static_cast<S*>(outv);
    const bool store_lane = lane >= 1 && lane <= 30;
    const bool store_warp = warp >= TT && warp < TT + TY;
    const int wu = warp > 0 ? warp - 1 : 0, wd = warp < TYH - 1 ? warp + 1 : TYH - 1;  // neighbour rows (clamped)
    long long k = 0;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int s_ = item % strips;
        const int yt = (item / strips) % ytiles;
        const int zs = item / (strips * ytiles);
        const int X0 = s_ * kTbStride - kTbLead;
        const int xb = X0 + lane * LN;
        const int yo = yt * TY + warp - TT;                        // interior row of this warp
        const int zb = zs * H;
        const int hz = min(H, g.nz - zb);
        const int np = hz + 2 * TT;
        es.init(g, xb, store_lane);
#pragma unroll
        for (int t = 0; t < TT; ++t)
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int n = 0; n < LN; ++n) acc[t][p][n] = T(0);
        bool stop = false;
        for (int i = 0; i < np; ++i, ++k) {
            const int s = (int)(k % NSTAGE);
            const bool ok = mbar_wait_bounded(&full[s], (uint32_t)((k / NSTAGE) & 1));
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) atomicExch(sflag, 1);
            } else {
                // level 0 -> level 1: rows warp-1 .. warp+1 of the staged plane
                T raw[3][6];
                const int rows[3] = {wu, warp, wd};
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    const unsigned char* rowp = ring + (size_t)s * SLOT + (size_t)rows[r] * ROWP;
                    const S* sp = reinterpret_cast<const S*>(rowp);
                    T v4[4];
                    lds4<ST, PDE_LCDE>(rowp + (size_t)(ALIGN + lane * LN) * ES, cf.ref[0], v4);
                    raw[r][1] = v4[0];
                    raw[r][2] = v4[1];
                    raw[r][3] = v4[2];
                    raw[r][4] = v4[3];
                    raw[r][0] = kload<ST, PDE_LCDE>(sp + ALIGN + lane * LN - 1, cf.ref[0]);
                    raw[r][5] = kload<ST, PDE_LCDE>(sp + ALIGN + lane * LN + LN, cf.ref[0]);
                }
                tb3_push<LAT, T>(cf, raw, acc[0][0], acc[0][1], acc[0][2]);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            // levels 1 .. TT-1: the completed plane goes through shared memory to the next level
#pragma unroll
            for (int t = 0; t < TT - 1; ++t) {
                T* buf = lev + (size_t)(2 * t + (i & 1)) * LPLANE;
                st4(buf + (size_t)warp * LROW + 4 + lane * LN, acc[t][0][0], acc[t][0][1], acc[t][0][2], acc[t][0][3]);
#pragma unroll
                for (int n = 0; n < LN; ++n) {
                    acc[t][0][n] = acc[t][1][n];
                    acc[t][1][n] = acc[t][2][n];
                    acc[t][2][n] = T(0);
                }
                rows_barrier(TYH * 32);
                if (t == 0 && *reinterpret_cast<volatile int*>(sflag)) {
                    stop = true;
                    break;
                }
                T raw[3][6];
                const int rows[3] = {wu, warp, wd};
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    // the lane's four values as one aligned vector (conflict-free), the two
                    // neighbours as scalars
                    const T* rp = buf + (size_t)rows[r] * LROW + 4 + lane * LN;
                    ld4(rp, raw[r][1], raw[r][2], raw[r][3], raw[r][4]);
                    raw[r][0] = rp[-1];
                    raw[r][5] = rp[4];
                }
                tb3_push<LAT, T>(cf, raw, acc[t + 1][0], acc[t + 1][1], acc[t + 1][2]);
            }
            if (stop) break;
            // level TT: plane zb - 2 TT + i is complete
            const int zo = zb - 2 * TT + i;
            if (i >= 2 * TT && store_warp && yo < g.ny) {   // warp-uniform
                const long long nb = ((long long)zo * g.ny + yo) * g.nx;
                S sv[4];
#pragma unroll
                for (int n = 0; n < LN; ++n) {
                    const unsigned rnd = ex.sr ? sr_bits(ex.seed, ex.step, nb + xb + n, 0) : 0u;
                    sv[n] = kpack<ST, PDE_LCDE>(acc[TT - 1][0][n], cf.ref[0], rnd);
                }
                es.put(out, g, xb, yo, zo, sv);
            }
#pragma unroll
            for (int n = 0; n < LN; ++n) {
                acc[TT - 1][0][n] = acc[TT - 1][1][n];
                acc[TT - 1][1][n] = acc[TT - 1][2][n];
                acc[TT - 1][2][n] = T(0);
            }
        }
        if (stop) break;
    }
    if (lane == 0 && *reinterpret_cast<volatile int*>(sflag)) atomicExch(err, KERR_TMA_TIMEOUT);
}

template <int ST, int TT, int TYH, int NSTAGE>
constexpr size_t tb3_smem() {
    constexpr int ES = ST == ST_F64 ? 8 : (ST == ST_F32 ? 4 : 2);
    constexpr int ROWB = (128 + 2 * (16 / ES)) * ES;
    constexpr int SLOT = ((ROWB + 127) / 128) * 128 * TYH;
    constexpr int TS = ST == ST_F64 ? 8 : 4;
    return 128 + 128 * ((2 * NSTAGE * 8 + 4 + 127) / 128) + (size_t)NSTAGE * SLOT +
           (size_t)(TT - 1) * 2 * 136 * TYH * TS;
}

constexpr int kTYH = 16;   // tile rows per CTA (output rows 16 - 2 TT)

template <int LAT, int ST, int TT>
cudaError_t launch_tb3(const LaunchArgs& a) {
    using T = typename Storage<ST>::T;
    constexpr int NSTAGE = 4;
    constexpr size_t smem = tb3_smem<ST, TT, kTYH, NSTAGE>();
    constexpr int THREADS = (kTYH + 1) * 32;
    auto kern = k_march3d_tb<LAT, ST, TT, kTYH, NSTAGE>;
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
    constexpr int TY = kTYH - 2 * TT;
    const int strips = (a.g.nx + kTbLead / 2 + kTbStride - 1) / kTbStride;
    const int ytiles = (a.g.ny + TY - 1) / TY;
    int H = a.H;
    if (H <= 0) {
        // planes per item: maximise (output planes / streamed planes) x (fill of the resident CTAs)
        double best = -1.0;
        for (int h = 4; h <= 1024; ++h) {
            const long long items = (long long)strips * ytiles * ((a.g.nz + h - 1) / h);
            const long long rounds = (items + resident - 1) / resident;
            const double fill = (double)items / (double)(rounds * resident);
            const double eff = fill * (double)h / (double)(h + 2 * TT);
            if (eff > best + 1e-9) {
                best = eff;
                H = h;
            }
            if (h >= a.g.nz) break;
        }
    }
    const int nitems = strips * ytiles * ((a.g.nz + H - 1) / H);
    const int grid = nitems < resident ? nitems : resident;
    kern<<<grid, THREADS, smem, a.stream>>>(*a.maps, a.g, a.out, *static_cast<const Coef<T>*>(a.coef), a.ex, H,
                                            nitems, a.err);
    return cudaGetLastError();
}

template <int LAT, int ST>
LaunchFn pick_depth(int depth) {
    if (depth == 2) return launch_tb3<LAT, ST, 2>;
    if constexpr (ST != ST_F64) {
        if (depth == 3) return launch_tb3<LAT, ST, 3>;
        if (depth == 4) return launch_tb3<LAT, ST, 4>;
    }
    if constexpr (ST == ST_BF16) {
        if (depth == 5) return launch_tb3<LAT, ST, 5>;
    }
    return nullptr;
}

template <int LAT>
LaunchFn pick_st(int st, int depth) {
    if (st == ST_F64) return pick_depth<LAT, ST_F64>(depth);
    if (st == ST_F32) return pick_depth<LAT, ST_F32>(depth);
    if (st == ST_BF16) return pick_depth<LAT, ST_BF16>(depth);
    return nullptr;
}

}  // namespace

LaunchFn find_march3d_tb(int lat, int pde, int levels, int st, int depth) {
    if (levels != 2 || depth < 2 || pde != PDE_LCDE) return nullptr;
    if (lat == LAT_D3Q7) return pick_st<LAT_D3Q7>(st, depth);
    if (lat == LAT_D3Q19) return pick_st<LAT_D3Q19>(st, depth);
    return nullptr;
}

}  // namespace mmfd
