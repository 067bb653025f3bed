// mmfd_internal.h -- definitions shared by the host library and the sm_103a kernels.
//
// The MMFD update (arXiv 2505.17057, Eq. (2-2), (2-4), (3layerMMFD-1)) is linear in the
// arguments (A, B, C) of the quadratic EDF Eq. (3-3), so the kernels evaluate it in the
// paired central form of Eq. (2-2-1)/(2-4-1): for every +/- velocity pair p (representative
// direction e_p) and every neighbour y = x +/- e_p they need only
//     E_p(y) = omega_p (A + Qtilde_p : C)(y)          (even part of f_p^eq)
//     O_p(y) = omega_p (ctilde_p . B)(y)               (odd part of f_p^eq)
// and
//     phi'(x) = sum_l [ a_0 A(x) + a+ f_0^eq(x) + sum_p a+ (E_p(x+e_p) + E_p(x-e_p))
//                                              + a- (O_p(x+e_p) - O_p(x-e_p)) ]
//     m'_a(x) = sum_l [ abar_0 B_a(x) + c_a sum_p e_pa ( abar- (E_p(x+e_p) - E_p(x-e_p))
//                                                   + abar+ (O_p(x+e_p) + O_p(x-e_p)) ) ]
// with a+ = a_1 + a_{-1}, a- = a_1 - a_{-1} (Eq. (2-1-FD1-0)) per time level l.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace mmfd {

enum Pde { PDE_LCDE = 0, PDE_NCDE = 1, PDE_NSE = 2 };
enum Lat { LAT_D2Q5 = 0, LAT_D2Q9 = 1, LAT_D3Q7 = 2, LAT_D3Q19 = 3 };
enum St { ST_F64 = 0, ST_F32 = 1, ST_BF16 = 2 };

constexpr int kMaxPair = 9;

// Representative direction of velocity pair p (the other member is -e_p).
__host__ __device__ constexpr int lat_dim(int lat) { return (lat == LAT_D2Q5 || lat == LAT_D2Q9) ? 2 : 3; }
__host__ __device__ constexpr int lat_npair(int lat) {
    return lat == LAT_D2Q5 ? 2 : lat == LAT_D2Q9 ? 4 : lat == LAT_D3Q7 ? 3 : 9;
}
__host__ __device__ constexpr int pair_e(int lat, int p, int a) {
    // D2Q5 / D3Q7: the coordinate axes.  D2Q9: x, y, (1,1), (-1,1).
    // D3Q19: x, y, z, (1,1,0), (-1,1,0), (1,0,1), (-1,0,1), (0,1,1), (0,-1,1).
    return (lat == LAT_D2Q5 || lat == LAT_D3Q7) ? (p == a ? 1 : 0)
         : (lat == LAT_D2Q9)
             ? (p < 2 ? (p == a ? 1 : 0)
                : p == 2 ? (a < 2 ? 1 : 0)
                         : (a == 0 ? -1 : a == 1 ? 1 : 0))
             : (p < 3 ? (p == a ? 1 : 0)
                : p == 3 ? (a == 0 ? 1 : a == 1 ? 1 : 0)
                : p == 4 ? (a == 0 ? -1 : a == 1 ? 1 : 0)
                : p == 5 ? (a == 0 ? 1 : a == 2 ? 1 : 0)
                : p == 6 ? (a == 0 ? -1 : a == 2 ? 1 : 0)
                : p == 7 ? (a == 1 ? 1 : a == 2 ? 1 : 0)
                         : (a == 1 ? -1 : a == 2 ? 1 : 0));
}
__host__ __device__ constexpr int pde_nf(int pde, int lat) { return pde == PDE_NSE ? 1 + lat_dim(lat) : 1; }

// Padded, ghost-celled layout of one level: every field is a (nz + 2 gz) x (ny + 2) x py
// array; interior node (x, y, z) sits at column ox + x, row y + 1, plane z + gz.  Ghost
// cells hold the periodic images, so stencil loads need no wrap arithmetic.  ox is chosen
// so that interior column 0 starts on a 16-byte boundary and py * es is a multiple of 16.
struct Geom {
    int dim, nx, ny, nz;
    int ox, gz;
    int gx;                // depth of the x ghost columns kept up to date (= ox)
    long long py, pz, fs;  // row pitch, plane pitch, field stride (elements)
    int nf, es;
    __host__ __device__ long long at(int x, int y, int z) const {
        return (long long)(z + gz) * pz + (long long)(y + 1) * py + ox + x;
    }
};

// Per-launch coefficients in the compute type T (host folds the constants).
template <typename T>
struct Coef {
    // pair p: E_p = eA A + eC . (Cxx, Cyy, Czz, Cxy, Cxz, Cyz); O_p = oB . B
    T eA[kMaxPair], eC[kMaxPair][6], oB[kMaxPair][3];
    T rA, rC[3];                       // rest direction: f_0^eq = rA A + rC . diag(C)
    T a0[2], ap[2], am[2];             // scalar / rho set per level (0: t, 1: t - dt)
    T ab0[2], abp[2], abm[2];          // momentum set per level
    T fmom[3];                         // c_a / rho0 (momentum -> velocity)
    T W0[2], Wp[2][kMaxPair], Wm[2][kMaxPair];   // LCDE: collapsed linear stencil per level
    T flux[3][4], m2[5];               // NCDE polynomials
    T ePhi[kMaxPair], eM2[kMaxPair], rPhi, rM2;  // NCDE: E_p = ePhi phi + eM2 M2(phi)
    T ref[4];                          // BF16 offsets per field
    // He-Luo NSE, lean form (host-checked, see nse_lean in params.cpp): with one speed c on every
    // axis, on D2Q9 (any isotropic d_0) or on D3Q19 with d_0 = 1/3, the uu terms of Eq. (3-3)
    // reduce to |u|^2 and (e_p . u)^2.  Per level l (k: 0 axis pairs, 1 diagonal pairs):
    //   E_p = nA[l][k] rho + nU[l][k] |u|^2 + nk[l][p] (e_p . u)^2,   O_p = no[l][p] (e_p . u)
    //   a0 rho + a+ f_0^eq = nc[l][0] rho + nc[l][1] |u|^2.
    // When the momentum set is proportional to the scalar one, (abar-, abar+) = kappa (a+, a-)
    // (LBGK tau = 1 among others), a+ and a- are folded into E_p and O_p (the scalar contribution
    // is then E_p +- O_p) and the momentum one is +-kappa times it, nsm[l][a] = kappa c_a / rho0.
    // Otherwise the per-level values are E_p, O_p themselves and the general combination applies.
    T nA[2][2], nU[2][2], nk[2][kMaxPair], no[2][kMaxPair], nc[2][2], nsm[2][3];
};

// Lean NSE variants of the marching kernels (Coef::nA): 0 none, 1 streaming momentum, 2 general.
enum : int { LEAN_NONE = 0, LEAN_STREAM = 1, LEAN_GENERAL = 2 };

// Source terms of one step (Eq. (2-1) with F_j = g_j^eq(S, M_1F, 0), Eq. (SourceF)), folded on
// the host from the central form Eq. (3layerMMFD-2) per level l (0: t, 1: t - dt):
//   dt [ B_0 S(x) + sum_p omega_p ( b+ (S(x+e_p) - 2 S(x) + S(x-e_p))
//                                   + b- ctilde_p . (M_1F(x+e_p) - M_1F(x-e_p)) ) ]
// = W0 S(x) + sum_p [ Wp S(x+e_p) + Wm S(x-e_p) + M_p . (M_1F(x+e_p) - M_1F(x-e_p)) ];
// M_1F = S u (constant u) is folded into Wp / Wm.
template <typename T>
struct SrcCoef {
    T W0[2], Wp[2][kMaxPair], Wm[2][kMaxPair];
    T M[2][kMaxPair][3];
};

// Source levels (S, then the M_1F components, one field stride g.fs apart, in the level
// geometry g, compute type T) and their weights.
template <typename T>
struct SrcArgs {
    const T* s[2];
    SrcCoef<T> w;
};

// Kernel parameter of a kernel family with (SRC != 0) or without source terms.
struct NoSrc {};
template <typename T, int SRC>
using SrcParam = std::conditional_t<SRC != 0, SrcArgs<T>, NoSrc>;

struct StepExtra {
    unsigned long long seed;  // stochastic rounding
    long long step;           // global step index of the level being written
    int sr;                   // 1: stochastic rounding (BF16 storage only)
};

}  // namespace mmfd
