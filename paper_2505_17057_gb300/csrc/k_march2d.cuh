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
#include "stencil.cuh"
#include "tma.cuh"

namespace mmfd {

// Four consecutive values of storage type S from shared memory (aligned) into T (offsets, or
// values for the NCDE's BF16 levels: see kload).
template <int ST, int PDE>
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
        v[0] = __uint_as_float(q.x << 16);
        v[1] = __uint_as_float(q.x & 0xffff0000u);
        v[2] = __uint_as_float(q.y << 16);
        v[3] = __uint_as_float(q.y & 0xffff0000u);
        if constexpr (!offset_arith<PDE>()) {
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] += ref;
        }
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

// Store four consecutive nodes xb .. xb+3 (xb a multiple of 4) of row y, plane z, together with
// their periodic ghost images: the x ghosts within g.gx of either x edge, the ghost row of
// y = 0 / ny - 1 and, in 3D, the ghost plane of z = 0 / nz - 1 (with all combinations).  Nodes
// outside [0, nx) are skipped.  Straight-line predicated stores, no local arrays: the warps that
// own edge strips and rows must not fall behind the others.
// (The four values come as scalars: an array passed by address to an out-of-line function would
// have to live in local memory in the caller, on every row, for every lane.)
template <int DIM, int ST>
__device__ __noinline__ void store4_ghosted(typename Storage<ST>::S* f, const Geom g, int xb, int y, int z,
                                            typename Storage<ST>::S s0, typename Storage<ST>::S s1,
                                            typename Storage<ST>::S s2, typename Storage<ST>::S s3) {
    using S = typename Storage<ST>::S;
    const S sv[4] = {s0, s1, s2, s3};
    const bool full = xb >= 0 && xb + 3 < g.nx;
    const bool xedge = xb < g.gx || xb + 3 >= g.nx - g.gx;
    auto put_row = [&](int yy, int zz) {
        S* row = f + g.at(0, yy, zz);
        if (full) {
            stg4<ST>(row + xb, sv);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (xb + k >= 0 && xb + k < g.nx) row[xb + k] = sv[k];
        }
        if (xedge) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int x = xb + k;
                if (x >= 0 && x < g.nx) {
                    if (x < g.gx) row[x + g.nx] = sv[k];
                    if (x >= g.nx - g.gx) row[x - g.nx] = sv[k];
                }
            }
        }
    };
    const bool ylo = y == 0, yhi = y == g.ny - 1;
    auto put_plane = [&](int zz) {
        put_row(y, zz);
        if (ylo) put_row(g.ny, zz);
        if (yhi) put_row(-1, zz);
    };
    put_plane(z);
    if constexpr (DIM == 3) {
        if (z == 0) put_plane(g.nz);
        if (z == g.nz - 1) put_plane(-1);
    }
}

// The output store of the marching kernels.  A lane writes its four nodes xb .. xb+3 (xb a
// multiple of 4) and their periodic ghost images -- the ghost row of y = 0 / ny - 1 and the
// whole-vector x ghost blocks -- with predicated stores only, all 32 lanes following the same
// control flow: a lane that branched off alone onto an edge path made its whole warp run about
// three times slower on every row (measured per warp with %globaltimer), and the warps owning
// the edge strips then set the length of the launch.  What depends only on the lane's columns
// is worked out once per work item (init); the cases vectors cannot cover (z edge planes,
// ny == 1, vectors straddling x = nx, x ghosts when nx is not a multiple of 4) take
// store4_ghosted under a warp-uniform branch.
template <int DIM, int ST>
struct EdgeStore {
    using S = typename Storage<ST>::S;
    static constexpr int OX = 16 / (int)sizeof(S);   // ghost block width (elements)
    bool in = false;      // the lane's four nodes are output nodes inside [0, nx)
    bool lo = false;      // writes the x ghost block at x + nx as a vector
    bool hi = false;      // writes the x ghost block at x - nx as a vector
    bool xrare = false;   // needs the general path (partial vector, scalar x ghosts)
    bool wrare = false;   // some lane of the warp does (warp-uniform)

    // all 32 lanes, once per item
    __device__ __forceinline__ void init(const Geom& g, int xb, bool valid) {
        in = valid && xb >= 0 && xb + 3 < g.nx;
        const bool part = valid && !in && xb < g.nx && xb + 3 >= 0;
        bool xdone;
        if constexpr (OX >= 4) {
            // FP32 / BF16: the lane's nodes are one 16- or 8-byte piece of the block; the image at
            // x -+ nx is vector-aligned only when nx is a multiple of 4
            const bool al = (g.nx & 3) == 0;
            lo = in && al && xb + 3 < OX;
            hi = in && al && xb >= g.nx - OX;
            xdone = !(in && (xb < g.gx || xb + 3 >= g.nx - g.gx)) || lo || hi;
        } else {
            // FP64: the block is two doubles, the first or last half of the lane
            lo = in && xb == 0 && (g.nx & 1) == 0;
            hi = in && xb + 4 == g.nx;
            xdone = (!(in && xb < g.gx) || lo) && (!(in && xb + 3 >= g.nx - g.gx) || hi);
        }
        xrare = part || !xdone;
        wrare = __any_sync(0xffffffffu, xrare);
    }

    // all 32 lanes (warp-uniform y, z)
    __device__ __forceinline__ void put(S* f, const Geom& g, int xb, int y, int z, const S (&sv)[4]) const {
        S* p = f + g.at(xb, y, z);
        if (in) stg4<ST>(p, sv);
        const bool ydup = g.ny > 1 && (y == 0 || y == g.ny - 1);
        if (ydup || lo || hi) {
            const long long dy = y == 0 ? (long long)g.ny * g.py : -(long long)g.ny * g.py;
            if (in && ydup) stg4<ST>(p + dy, sv);
            if constexpr (OX >= 4) {
                if (lo) stg4<ST>(p + g.nx, sv);
                if (lo && ydup) stg4<ST>(p + g.nx + dy, sv);
                if (hi) stg4<ST>(p - g.nx, sv);
                if (hi && ydup) stg4<ST>(p - g.nx + dy, sv);
            } else {
                if (lo) *reinterpret_cast<double2*>(p + g.nx) = make_double2(sv[0], sv[1]);
                if (lo && ydup) *reinterpret_cast<double2*>(p + g.nx + dy) = make_double2(sv[0], sv[1]);
                if (hi) *reinterpret_cast<double2*>(p + 2 - g.nx) = make_double2(sv[2], sv[3]);
                if (hi && ydup) *reinterpret_cast<double2*>(p + 2 - g.nx + dy) = make_double2(sv[2], sv[3]);
            }
        }
        const bool plane_rare = g.ny == 1 || (DIM == 3 && (z == 0 || z == g.nz - 1));
        if (wrare || plane_rare) {
            if (xrare || (plane_rare && (in || xrare))) store4_ghosted<DIM, ST>(f, g, xb, y, z, sv[0], sv[1], sv[2], sv[3]);
        }
    }
};

// Work decomposition: an item is (128-column warp strip, H-row segment).  Every warp walks its
// own sequence of items (item = global warp id, + total warps, ...) as one stream of input
// rows; lane 0 keeps NSTAGE rows of that stream in flight through the warp's private ring, so
// the prefetch runs across item boundaries and warps never wait for one another.

// Even / odd parts E_p, O_p of the pairs a node must push (bit p of MASK set), from the node's
// basis.  On D2Q9 the two diagonal pairs (1,1) and (-1,1) share omega_p and the diagonal
// Qtilde terms by the lattice's symmetry (App. A), so their common even part is formed once:
// E_{(+-1,1)} = Ed +- q_xy uxy, O_{(+-1,1)} = +-k_x B_x + k_y B_y.
template <int LAT, int PDE, int MASK, typename T>
__device__ __forceinline__ void pair_eo(const Coef<T>& cf, T rho_or_phi, const T* B, T m2, T uxx, T uyy, T uxy,
                                        T (&E)[4], T (&O)[4]) {
    if constexpr (PDE == PDE_NSE) {
        if constexpr (MASK & 1) E[0] = cf.eC[0][1] * uyy + (cf.eC[0][0] * uxx + cf.eA[0] * rho_or_phi);
        if constexpr (MASK & 2) E[1] = cf.eC[1][1] * uyy + (cf.eC[1][0] * uxx + cf.eA[1] * rho_or_phi);
        if constexpr (LAT == LAT_D2Q9 && (MASK & 12)) {
            const T Ed = cf.eC[2][1] * uyy + (cf.eC[2][0] * uxx + cf.eA[2] * rho_or_phi);
            if constexpr (MASK & 4) E[2] = cf.eC[2][3] * uxy + Ed;
            if constexpr (MASK & 8) E[3] = Ed - cf.eC[2][3] * uxy;
        }
    } else {
        if constexpr (MASK & 1) E[0] = cf.eM2[0] * m2 + cf.ePhi[0] * rho_or_phi;
        if constexpr (MASK & 2) E[1] = cf.eM2[1] * m2 + cf.ePhi[1] * rho_or_phi;
        if constexpr (LAT == LAT_D2Q9 && (MASK & 12)) {
            const T Ed = cf.eM2[2] * m2 + cf.ePhi[2] * rho_or_phi;
            E[2] = Ed;
            E[3] = Ed;
        }
    }
    if constexpr (MASK & 1) O[0] = cf.oB[0][0] * B[0];
    if constexpr (MASK & 2) O[1] = cf.oB[1][1] * B[1];
    if constexpr (LAT == LAT_D2Q9 && (MASK & 12)) {
        const T tx = cf.oB[2][0] * B[0];
        if constexpr (MASK & 4) O[2] = cf.oB[2][1] * B[1] + tx;
        if constexpr (MASK & 8) O[3] = cf.oB[2][1] * B[1] - tx;
    }
}

// Bit mask of the pairs whose plus or minus target of input node offset C (-1 .. LN) lands
// on one of the lane's LN output nodes.
template <int LAT, int LN>
__host__ __device__ constexpr int pushed_pairs(int C) {
    int m = 0;
    for (int p = 0; p < lat_npair(LAT); ++p) {
        const int ex = pair_e(LAT, p, 0);
        const int tp = C - ex, tm = C + ex;
        if ((tp >= 0 && tp < LN) || (tm >= 0 && tm < LN)) m |= 1 << p;
    }
    return m;
}

// Pieces of the lean He-Luo node update (Coef::nA) for 2D rows, written once so that every kernel
// that evaluates them rounds alike: |u|^2, the class base B_k = nU |u|^2 + nA rho, and the even /
// odd parts of pair P, E = nk (e_p . u)^2 + B_k and O = no (e_p . u).
// Every piece is rounded as written (rmul / rfma), so a value computed once and used twice rounds
// as when computed for each use.
template <typename T>
__device__ __forceinline__ T lean_u2(T ux, T uy) {
    return rfma(uy, uy, rmul(ux, ux));
}
template <typename T>
__device__ __forceinline__ T lean_base(const Coef<T>& cf, int l, int k, T U, T rho) {
    return rfma(cf.nU[l][k], U, rmul(cf.nA[l][k], rho));
}
// e_p . u and E_p of pair P
template <int LAT, int P, typename T>
__device__ __forceinline__ void lean_e2d(const Coef<T>& cf, int l, T ux, T uy, T base, T& cu, T& E) {
    cu = edot<LAT, P>(ux, uy, T(0));
    E = rfma(cf.nk[l][P], rmul(cu, cu), base);
}
// The streaming contribution E_p +- O_p = E_p +- no (e_p . u), one fused rounding.
template <int P, int SIGN, typename T>
__device__ __forceinline__ T lean_sv2d(const Coef<T>& cf, int l, T cu, T E) {
    return rfma(SIGN > 0 ? cf.no[l][P] : -cf.no[l][P], cu, E);
}

// One input node of a 2D row (column C of the lane's window, fields f = rho, ux, uy) in the
// lean He-Luo form (Coef::nA), pushed into the accumulators of output rows r-1 (P), r (C) and
// r+1 (N): per node |u|^2 and the class bases, per pair e_p . u, E_p as one FMA on the base and
// O_p as one multiply, a+ / a- folded in for streaming momentum sets.  l: input level.  The
// marching kernel and the temporally blocked NSE kernel share it, so that they round alike.
template <int LAT, int LEAN, int LN, int C, typename T>
__device__ __forceinline__ void lean_push_node2d(const Coef<T>& cf, int l, const T* f, T (&accP)[LN][3],
                                                 T (&accC)[LN][3], T (&accN)[LN][3]) {
    constexpr int NF = 3;
    constexpr int NP = lat_npair(LAT);
    constexpr bool OWN = C >= 0 && C < LN;
    constexpr int MASK = pushed_pairs<LAT, LN>(C);
    const T rho = f[0], ux = f[1], uy = f[2];
    const T U = lean_u2(ux, uy);
    if constexpr (OWN) {
        accC[C][0] = radd(accC[C][0], rfma(cf.nc[l][1], U, rmul(cf.nc[l][0], rho)));
        accC[C][1] = rfma(cf.ab0[l], ux, accC[C][1]);
        accC[C][2] = rfma(cf.ab0[l], uy, accC[C][2]);
    }
    constexpr bool AX = (MASK & 3) != 0, DG = (MASK & 12) != 0;
    [[maybe_unused]] T Bk[2];
    if constexpr (AX) Bk[0] = lean_base(cf, l, 0, U, rho);
    if constexpr (DG) Bk[1] = lean_base(cf, l, 1, U, rho);
    static_for<0, NP>([&](auto pcc) {
        constexpr int P_ = decltype(pcc)::value;
        constexpr int EX = pair_e(LAT, P_, 0), EY = pair_e(LAT, P_, 1);
        constexpr int TP = C - EX, TM = C + EX;
        constexpr bool HP = TP >= 0 && TP < LN, HM = TM >= 0 && TM < LN;
        if constexpr (HP || HM) {
            T cu, E;
            lean_e2d<LAT, P_>(cf, l, ux, uy, Bk[pair_class(LAT, P_)], cu, E);
            if constexpr (LEAN == LEAN_STREAM) {
                if constexpr (HP) lean_push_sv<LAT, P_, 1>(EY == 1 ? accP[TP] : accC[TP], cf, l, lean_sv2d<P_, 1>(cf, l, cu, E));
                if constexpr (HM) lean_push_sv<LAT, P_, -1>(EY == 1 ? accN[TM] : accC[TM], cf, l, lean_sv2d<P_, -1>(cf, l, cu, E));
            } else {
                const T O = rmul(cf.no[l][P_], cu);
                const T sE = cf.ap[l] * E, mO = cf.abp[l] * O;
                if constexpr (HP) lean_push<LAT, LEAN, P_, 1, NF>(EY == 1 ? accP[TP] : accC[TP], cf, l, E, O, sE, mO);
                if constexpr (HM) lean_push<LAT, LEAN, P_, -1, NF>(EY == 1 ? accN[TM] : accC[TM], cf, l, E, O, sE, mO);
            }
        }
    });
}

// Six consecutive source values xb-1 .. xb+4 of one padded row (xb a multiple of 4): a vector
// load for the lane's own four (16-byte aligned in the source layout) and two scalars; columns
// beyond the right ghost column are not read (lanes past nx only feed nodes that are not stored).
template <typename T>
__device__ __forceinline__ void ld_src6(const T* __restrict__ row, int xb, int nx, T (&v)[6]) {
    if (xb + 3 < nx) {
        if constexpr (sizeof(T) == 4) {
            const float4 q = __ldg(reinterpret_cast<const float4*>(row + xb));
            v[1] = q.x; v[2] = q.y; v[3] = q.z; v[4] = q.w;
        } else {
            const double2 a = __ldg(reinterpret_cast<const double2*>(row + xb));
            const double2 b = __ldg(reinterpret_cast<const double2*>(row + xb + 2));
            v[1] = a.x; v[2] = a.y; v[3] = b.x; v[4] = b.y;
        }
        v[0] = __ldg(row + xb - 1);
        v[5] = __ldg(row + xb + 4);
    } else {
#pragma unroll
        for (int c = 0; c < 6; ++c) v[c] = xb - 1 + c <= nx ? __ldg(row + xb - 1 + c) : T(0);
    }
}

// Whether source row (y + DY, z + DZ) feeds an output node: the centre row, or the row of a
// pair's plus (+e_p) or minus (-e_p) neighbour.
template <int LAT>
__host__ __device__ constexpr bool src_row_used(int DY, int DZ) {
    if (DY == 0 && DZ == 0) return true;
    for (int p = 0; p < lat_npair(LAT); ++p) {
        const int ey = pair_e(LAT, p, 1), ez = lat_dim(LAT) == 3 ? pair_e(LAT, p, 2) : 0;
        if ((ey == DY && ez == DZ) || (-ey == DY && -ez == DZ)) return true;
    }
    return false;
}

// Source terms of the four output nodes xb .. xb+3 of row y, plane z (see SrcCoef): the folded
// stencil, taken one source row (y + DY, z + DZ) at a time so that only six values per source
// field are live.  Each source value is read by several output rows and neighbouring lanes,
// which the L1 serves; DRAM sees it about once.
template <int LAT, int SRC, int LEVELS, typename T>
__device__ __forceinline__ void source_quad(const Geom& g, const SrcArgs<T>& sa, int y, int z, int xb, T (&add)[4]) {
    constexpr int NP = lat_npair(LAT);
    constexpr int DIM = lat_dim(LAT);
    constexpr int NS = SRC == 2 ? 1 + DIM : 1;
#pragma unroll
    for (int k = 0; k < 4; ++k) add[k] = T(0);
    if (xb >= g.nx) return;
#pragma unroll
    for (int l = 0; l < LEVELS - 1; ++l) {
        static_for<0, 9>([&](auto rc) {
            constexpr int DY = decltype(rc)::value / 3 - 1, DZ = decltype(rc)::value % 3 - 1;
            if constexpr ((DIM == 3 || DZ == 0) && src_row_used<LAT>(DY, DZ)) {
                T v[NS][6];
#pragma unroll
                for (int q = 0; q < NS; ++q) ld_src6<T>(sa.s[l] + (size_t)q * g.fs + g.at(0, y + DY, z + DZ), xb, g.nx, v[q]);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    T acc = T(0);
                    if constexpr (DY == 0 && DZ == 0) acc = sa.w.W0[l] * v[0][k + 1];
                    static_for<0, NP>([&](auto pc) {
                        constexpr int P = decltype(pc)::value;
                        constexpr int EX = pair_e(LAT, P, 0), EY = pair_e(LAT, P, 1);
                        constexpr int EZ = DIM == 3 ? pair_e(LAT, P, 2) : 0;
                        if constexpr (EY == DY && EZ == DZ) {
                            acc += sa.w.Wp[l][P] * v[0][k + 1 + EX];
                            if constexpr (SRC == 2) {
#pragma unroll
                                for (int a = 0; a < DIM; ++a)
                                    if (pair_e(LAT, P, a) != 0) acc += sa.w.M[l][P][a] * v[1 + a][k + 1 + EX];
                            }
                        }
                        if constexpr (-EY == DY && -EZ == DZ) {
                            acc += sa.w.Wm[l][P] * v[0][k + 1 - EX];
                            if constexpr (SRC == 2) {
#pragma unroll
                                for (int a = 0; a < DIM; ++a)
                                    if (pair_e(LAT, P, a) != 0) acc -= sa.w.M[l][P][a] * v[1 + a][k + 1 - EX];
                            }
                        }
                    });
                    add[k] += acc;
                }
            }
        });
    }
}

template <int LAT, int PDE, int LEVELS, int ST, int NW, int NSTAGE, int LN, int RPS, int SRC = 0, int LEAN = LEAN_NONE,
          int SRM = 2>
__global__ void __launch_bounds__(NW * 32) k_march2d(const __grid_constant__ TmapSet maps, Geom g,
                                                     void* __restrict__ outv, Coef<typename Storage<ST>::T> cf,
                                                     StepExtra ex, int H, int nitems, int* __restrict__ err,
                                                     const __grid_constant__ SrcParam<typename Storage<ST>::T, SRC> sa) {
    using Tr = Storage<ST>;
    using S = typename Tr::S;
    using T = typename Tr::T;
    constexpr int ES = (int)sizeof(S);
    constexpr int ALIGN = 16 / ES;
    constexpr int COLS = 32 * LN;                         // columns per warp item
    constexpr int BOXW = COLS + 2 * ALIGN;                // TMA box width (elements)
    constexpr int ROWB = BOXW * ES;                       // bytes per staged row
    constexpr int SLOT = ((RPS * ROWB + 127) / 128) * 128; // bytes per (stage, field) slot: RPS rows
    constexpr int NF = pde_nf(PDE, LAT);
    constexpr int NIN = NF * (LEVELS - 1);
    constexpr int NP = lat_npair(LAT);
    constexpr uint32_t kTx = (uint32_t)(NIN * RPS * ROWB);
    constexpr size_t kRingBytes = (size_t)NSTAGE * NIN * SLOT;
    static_assert(BOXW <= 256, "TMA box too wide");

    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations must sit on 128-byte boundaries whatever the dynamic-smem base is
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem) + warp * NSTAGE;
    unsigned char* ring = smem + 128 * ((NW * NSTAGE * 8 + 127) / 128) + warp * kRingBytes;

    const int strips = (g.nx + COLS - 1) / COLS;
    const int wstride = gridDim.x * NW;
    const int wid = blockIdx.x * NW + warp;
    if (wid >= nitems) return;

    auto slot = [&](int s, int q) -> unsigned char* { return ring + (size_t)(s * NIN + q) * SLOT; };

    // producer (lane 0): row stream cursor with its item's box origin, ring position of the next
    // issue; the divisions happen once per item, not once per row
    int p_item = wid, p_row = 0, p_rows = 0, p_xcol = 0, p_prow0 = 0;
    auto p_load_item = [&]() {
        if (p_item < nitems) {
            const int seg = p_item / strips;
            p_xcol = (p_item - seg * strips) * COLS;     // padded column of the box
            p_prow0 = seg * H;                            // padded row of input row y0 - 1
            p_rows = (min(H, g.ny - seg * H) + 2 + RPS - 1) / RPS * RPS;
        }
    };
    p_load_item();
    int ps = 0;                 // stage of the next issue
    long long issued = 0;
    auto issue_next = [&]() {
        if (p_item >= nitems) return;
        mbar_arrive_expect_tx(&full[ps], kTx);
#pragma unroll
        for (int q = 0; q < NIN; ++q) tma_load_2d(slot(ps, q), &maps.m[q], &full[ps], p_xcol, p_prow0 + p_row);
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
        for (int q = 0; q < NIN; ++q) tma_prefetch_desc(&maps.m[q]);
        for (int k = 0; k < NSTAGE; ++k) issue_next();
    }
    __syncwarp();

    // Accumulators of the output rows around the staged input rows: with RPS = 1, acc0/1/2 are
    // rows r-1, r, r+1 of input row r; with RPS = 2 (two input rows r, r+1 per stage), acc0..3
    // are rows r-1 .. r+2.
    T acc0[LN][NF], acc1[LN][NF], acc2[LN][NF], acc3[LN][NF];
    S* out = static_cast<S*>(outv);
    int cs = 0;              // stage of the next rows to consume
    uint32_t cphase = 0;     // its mbarrier phase parity
    long long consumed = 0;
    bool failed = false;

    // Push input row j of stage s into (accP = row r-1, accC = row r, accN = row r+1).
    auto push_row = [&](int s, int j, T (&accP)[LN][NF], T (&accC)[LN][NF], T (&accN)[LN][NF]) {
#pragma unroll
        for (int l = 0; l < LEVELS - 1; ++l) {
            // raw fields of the LN + 2 nodes xb-1 .. xb+LN of this input row
            T raw[LN + 2][NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const unsigned char* base = slot(s, l * NF + f) + j * ROWB;
                const S* sp = reinterpret_cast<const S*>(base);
#pragma unroll
                for (int k4 = 0; k4 < LN; k4 += 4) {
                    T v4[4];
                    lds4<ST, PDE>(base + (size_t)(ALIGN + lane * LN + k4) * ES, cf.ref[f], v4);
                    raw[1 + k4][f] = v4[0];
                    raw[2 + k4][f] = v4[1];
                    raw[3 + k4][f] = v4[2];
                    raw[4 + k4][f] = v4[3];
                }
                raw[0][f] = kload<ST, PDE>(sp + ALIGN + lane * LN - 1, cf.ref[f]);
                raw[LN + 1][f] = kload<ST, PDE>(sp + ALIGN + lane * LN + LN, cf.ref[f]);
            }
            static_for<0, LN + 2>([&](auto cc) {
                constexpr int C = decltype(cc)::value - 1;  // node offset -1 .. LN
                constexpr bool OWN = C >= 0 && C < LN;
                if constexpr (PDE == PDE_LCDE) {
                    const T phi = raw[C + 1][0];
                    if constexpr (OWN) accC[C][0] += cf.W0[l] * phi;
                    static_for<0, NP>([&](auto pcc) {
                        constexpr int P_ = decltype(pcc)::value;
                        constexpr int EX = pair_e(LAT, P_, 0), EY = pair_e(LAT, P_, 1);
                        constexpr int TP = C - EX, TM = C + EX;
                        if constexpr (TP >= 0 && TP < LN) {
                            if constexpr (EY == 1) accP[TP][0] += cf.Wp[l][P_] * phi;
                            else accC[TP][0] += cf.Wp[l][P_] * phi;
                        }
                        if constexpr (TM >= 0 && TM < LN) {
                            if constexpr (EY == 1) accN[TM][0] += cf.Wm[l][P_] * phi;
                            else accC[TM][0] += cf.Wm[l][P_] * phi;
                        }
                    });
                } else if constexpr (PDE == PDE_NSE && LEAN != LEAN_NONE) {
                    lean_push_node2d<LAT, LEAN, LN, C>(cf, l, raw[C + 1], accP, accC, accN);
                } else {
                    constexpr int MASK = pushed_pairs<LAT, LN>(C);
                    const T* f = raw[C + 1];
                    T A, B[2], m2 = T(0), uxx = T(0), uyy = T(0), uxy = T(0);
                    if constexpr (PDE == PDE_NSE) {
                        A = f[0];
                        B[0] = f[1];
                        B[1] = f[2];
                        uxx = f[1] * f[1];
                        uyy = f[2] * f[2];
                        uxy = f[1] * f[2];
                    } else {
                        const T phi = f[0];
                        A = phi;
                        m2 = (((cf.m2[4] * phi + cf.m2[3]) * phi + cf.m2[2]) * phi + cf.m2[1]) * phi + cf.m2[0];
#pragma unroll
                        for (int a = 0; a < 2; ++a)
                            B[a] = ((cf.flux[a][3] * phi + cf.flux[a][2]) * phi + cf.flux[a][1]) * phi + cf.flux[a][0];
                    }
                    if constexpr (OWN) {
                        T rest;
                        if constexpr (PDE == PDE_NSE) rest = cf.rC[1] * uyy + (cf.rC[0] * uxx + cf.rA * A);
                        else rest = cf.rM2 * m2 + cf.rPhi * A;
                        accC[C][0] += cf.ap[l] * rest + cf.a0[l] * A;
                        if constexpr (PDE == PDE_NSE) {
                            accC[C][1] += cf.ab0[l] * B[0];
                            accC[C][2] += cf.ab0[l] * B[1];
                        }
                    }
                    T E[4], O[4];
                    pair_eo<LAT, PDE, MASK>(cf, A, B, m2, uxx, uyy, uxy, E, O);
                    static_for<0, NP>([&](auto pcc) {
                        constexpr int P_ = decltype(pcc)::value;
                        constexpr int EX = pair_e(LAT, P_, 0), EY = pair_e(LAT, P_, 1);
                        constexpr int TP = C - EX, TM = C + EX;
                        constexpr bool HP = TP >= 0 && TP < LN, HM = TM >= 0 && TM < LN;
                        if constexpr (HP || HM) {
                            // rho / phi: a+ E +- a- O; momentum: abar+ O +- abar- E (Eq. (2-4-1))
                            const T sE = cf.ap[l] * E[P_];
                            [[maybe_unused]] T mO = T(0);
                            if constexpr (PDE == PDE_NSE) mO = cf.abp[l] * O[P_];
                            auto push = [&](T (&acc)[LN][NF], int node, T sv, T mv) {
                                acc[node][0] += sv;
                                if constexpr (PDE == PDE_NSE) {
                                    if constexpr (EX != 0) acc[node][1] += (T(EX) * cf.fmom[0]) * mv;
                                    if constexpr (EY != 0) acc[node][2] += (T(EY) * cf.fmom[1]) * mv;
                                }
                            };
                            if constexpr (HP) {
                                const T sv = cf.am[l] * O[P_] + sE;
                                T mv = T(0);
                                if constexpr (PDE == PDE_NSE) mv = cf.abm[l] * E[P_] + mO;
                                if constexpr (EY == 1) push(accP, TP, sv, mv);
                                else push(accC, TP, sv, mv);
                            }
                            if constexpr (HM) {
                                const T sv = sE - cf.am[l] * O[P_];
                                T mv = T(0);
                                if constexpr (PDE == PDE_NSE) mv = mO - cf.abm[l] * E[P_];
                                if constexpr (EY == 1) push(accN, TM, sv, mv);
                                else push(accC, TM, sv, mv);
                            }
                        }
                    });
                }
            });
        }
    };

    // store the completed output row yo from acc
    EdgeStore<2, ST> es;
    // Source terms (SRC != 0) of the output row being stored, add[k] for node xb + k.
    // SRC == 1 (a source S; M_1F = 0 or S u folded): the source rows y0+i-3 .. y0+i feeding the two
    // output rows stored in iteration i sit in a rolling register window; the two new rows are
    // loaded at the top of the iteration, before the stage wait and the pushes, so that their
    // latency is hidden.  SRC == 2 (S and M_1F fields) reads its rows in the epilogue.
    [[maybe_unused]] T swin[LEVELS - 1][4][6];
    auto src_load = [&](int y0, int i, int xb) {
        if constexpr (SRC == 1) {
#pragma unroll
            for (int l = 0; l < LEVELS - 1; ++l) {
#pragma unroll
                for (int r = 0; r < 2; ++r)
#pragma unroll
                    for (int c = 0; c < 6; ++c) swin[l][r][c] = swin[l][r + 2][c];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int row = y0 + i - 1 + r;   // rows past the ghost row ny feed no stored output
                    if (xb < g.nx && row <= g.ny) {
                        ld_src6<T>(sa.s[l] + g.at(0, row, 0), xb, g.nx, swin[l][2 + r]);
                    } else {
#pragma unroll
                        for (int c = 0; c < 6; ++c) swin[l][2 + r][c] = T(0);
                    }
                }
            }
        }
    };
    // the output row whose source rows are window rows W0 .. W0 + 2 (y - 1, y, y + 1)
    auto src_window = [&](auto w0c, T (&add)[4]) {
        constexpr int W0 = decltype(w0c)::value;
        constexpr int NP = lat_npair(LAT);
#pragma unroll
        for (int k = 0; k < 4; ++k) add[k] = T(0);
        if constexpr (SRC == 1) {
#pragma unroll
        for (int l = 0; l < LEVELS - 1; ++l) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                T acc = sa.w.W0[l] * swin[l][W0 + 1][k + 1];
                static_for<0, NP>([&](auto pc) {
                    constexpr int P = decltype(pc)::value;
                    constexpr int EX = pair_e(LAT, P, 0), EY = pair_e(LAT, P, 1);
                    acc += sa.w.Wp[l][P] * swin[l][W0 + 1 + EY][k + 1 + EX] +
                           sa.w.Wm[l][P] * swin[l][W0 + 1 - EY][k + 1 - EX];
                });
                add[k] += acc;
            }
        }
        }
    };
    auto store_row = [&](int yo, int xb, const T (&acc)[LN][NF], const T (&add)[4]) {
        const long long nb = (long long)yo * g.nx;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            S* fo = out + (size_t)f * g.fs;
#pragma unroll
            for (int k4 = 0; k4 < LN; k4 += 4) {
                S sv[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const unsigned rnd = sr_on<SRM>(ex) ? sr_bits(ex.seed, ex.step, nb + xb + k4 + k, f) : 0u;
                    T v = acc[k4 + k][f];
                    if constexpr (SRC != 0) {
                        if (f == 0) v += add[k];
                    }
                    sv[k] = kpack<ST, PDE>(v, cf.ref[f], rnd);
                }
                es.put(fo, g, xb + k4, yo, 0, sv);
            }
        }
    };

    for (int item = wid; item < nitems && !failed; item += wstride) {
        const int seg = item / strips;
        const int x0 = (item - seg * strips) * COLS;
        const int y0 = seg * H;
        const int hrows = min(H, g.ny - y0);                       // output rows of the item
        const int nrows = (hrows + 2 + RPS - 1) / RPS * RPS;       // staged input rows
        const int xb = x0 + lane * LN;
        static_assert(LN == 4, "the edge store covers four nodes per lane");
        static_assert(SRC != 1 || RPS == 2, "the source window holds the rows of two output rows");
        es.init(g, xb, true);
#pragma unroll
        for (int k = 0; k < LN; ++k)
#pragma unroll
            for (int f = 0; f < NF; ++f) acc0[k][f] = acc1[k][f] = acc2[k][f] = acc3[k][f] = acc_zero<T>();
        for (int i = 0; i < nrows; i += RPS) {
            const int s = cs;
            if constexpr (SRC == 1) src_load(y0, i, xb);
            const bool ok = mbar_wait_bounded(&full[s], cphase);
            if (__any_sync(0xffffffffu, !ok)) {
                failed = true;
                break;
            }
            push_row(s, 0, acc0, acc1, acc2);
            if constexpr (RPS == 2) push_row(s, 1, acc1, acc2, acc3);
            ++consumed;
            cs = cs + 1 == NSTAGE ? 0 : cs + 1;
            if (cs == 0) cphase ^= 1u;
            __syncwarp();  // every lane is done reading stage s
            if (lane == 0) {
                fence_proxy_async_smem();
                issue_next();
            }
            // input row i (y0 - 1 + i) completes output row y0 + i - 2 (all lanes take part in
            // the store; lanes beyond nx write nothing)
            [[maybe_unused]] T add[4] = {T(0), T(0), T(0), T(0)};
            if (i >= 2) {
                if constexpr (SRC == 1) src_window(std::integral_constant<int, 0>{}, add);
                if constexpr (SRC == 2) source_quad<LAT, SRC, LEVELS, T>(g, sa, y0 + i - 2, 0, xb, add);
                store_row(y0 + i - 2, xb, acc0, add);
            }
            if constexpr (RPS == 2) {
                if (i >= 1 && i - 1 < hrows) {
                    if constexpr (SRC == 1) src_window(std::integral_constant<int, 1>{}, add);
                    if constexpr (SRC == 2) source_quad<LAT, SRC, LEVELS, T>(g, sa, y0 + i - 1, 0, xb, add);
                    store_row(y0 + i - 1, xb, acc1, add);
                }
            }
#pragma unroll
            for (int k = 0; k < LN; ++k)
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    if constexpr (RPS == 1) {
                        acc0[k][f] = acc1[k][f];
                        acc1[k][f] = acc2[k][f];
                        acc2[k][f] = acc_zero<T>();
                    } else {
                        acc0[k][f] = acc2[k][f];
                        acc1[k][f] = acc3[k][f];
                        acc2[k][f] = acc_zero<T>();
                        acc3[k][f] = acc_zero<T>();
                    }
                }
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

template <int ST, int LEVELS, int NF, int NW, int NSTAGE, int LN, int RPS>
constexpr size_t march2d_smem() {
    constexpr int ES = (int)sizeof(typename Storage<ST>::S);
    constexpr int SLOT = ((RPS * (32 * LN + 2 * (16 / ES)) * ES + 127) / 128) * 128;
    return 128 + 128 * ((NW * NSTAGE * 8 + 127) / 128) + (size_t)NW * NSTAGE * NF * (LEVELS - 1) * SLOT;
}

// Rows per stage: two input rows per TMA box halve the per-row waits, copy issues and
// accumulator rotations.  For the NSE it costs registers (128 instead of 96, four CTAs per SM
// instead of five) and still measured faster on 4096^2 (207 vs 191 GLUPS).
constexpr int rows_per_stage(int) { return 2; }

// Ring depth per warp: about 8 KB of stages, between 3 and 12 stages in flight.
template <int LAT, int PDE, int LEVELS, int ST, int LN>
constexpr int march2d_stages() {
    constexpr size_t per = (march2d_smem<ST, LEVELS, pde_nf(PDE, LAT), 1, 1, LN, rows_per_stage(PDE)>() - 256);
    constexpr size_t n = 8192 / per;
    return n < 3 ? 3 : (n > 12 ? 12 : (int)n);
}

template <int LAT, int PDE, int LEVELS, int ST, int NW, int NSTAGE, int LN, int RPS, int SRC = 0, int LEAN = LEAN_NONE,
          int SRM = 2>
cudaError_t launch_march2d_t(const LaunchArgs& a) {
    using T = typename Storage<ST>::T;
    constexpr int NF = pde_nf(PDE, LAT);
    constexpr size_t smem = march2d_smem<ST, LEVELS, NF, NW, NSTAGE, LN, RPS>();
    auto kern = k_march2d<LAT, PDE, LEVELS, ST, NW, NSTAGE, LN, RPS, SRC, LEAN, SRM>;
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
    constexpr int COLS = 32 * LN;
    const int strips = (a.g.nx + COLS - 1) / COLS;
    int H = a.H;
    if (H <= 0) {
        // rows per item: maximise (useful rows / streamed rows) x (fill of the resident warp slots);
        // small grids take short items so that every resident warp gets one
        const long long wslots = (long long)resident * NW;
        double best = -1.0;
        for (int h = 2; h <= 256; ++h) {
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
    SrcParam<T, SRC> sa{};
    if constexpr (SRC != 0) {
        sa.s[0] = static_cast<const T*>(a.src[0]);
        sa.s[1] = static_cast<const T*>(LEVELS == 3 ? a.src[1] : a.src[0]);
        sa.w = *static_cast<const SrcCoef<T>*>(a.src_coef);
    }
    kern<<<grid, NW * 32, smem, a.stream>>>(*a.maps, a.g, a.out, *static_cast<const Coef<T>*>(a.coef), a.ex, H,
                                             nitems, a.err, sa);
    return cudaGetLastError();
}

// The same with the stochastic-rounding choice made per launch (BF16 storage: an instantiation
// without and one with the rounding code; other storages never round stochastically).
template <int LAT, int PDE, int LEVELS, int ST, int NW, int NSTAGE, int LN, int RPS, int SRC = 0, int LEAN = LEAN_NONE>
cudaError_t launch_march2d_sr(const LaunchArgs& a) {
    if constexpr (ST == ST_BF16) {
        if (a.ex.sr) return launch_march2d_t<LAT, PDE, LEVELS, ST, NW, NSTAGE, LN, RPS, SRC, LEAN, 1>(a);
    }
    return launch_march2d_t<LAT, PDE, LEVELS, ST, NW, NSTAGE, LN, RPS, SRC, LEAN, 0>(a);
}

}  // namespace mmfd
