// params.h -- host-side resolution of a problem descriptor into scheme coefficients,
// EDF constants and kernel coefficient blocks (no GPU needed).
#pragma once

#include <string>

#include "../../include/mmfd.h"
#include "mmfd_internal.h"

namespace mmfd {

struct Resolved {
    int pde, lat, levels, dim, nf, st;
    long long n[3];
    double a[3], ahat[3], abar[3], abarhat[3];
    double A10, A20, A21, A22;
    double c[3], d0[3], cs2[3];
    double w[19];
    double Cmat[3][3];
    double m2[5];
    double ref[4];
    double max_lambda;
    Coef<double> cd;
    Coef<float> cf;
    int lean;           // LEAN_*: lean He-Luo form available to the marching kernels
    int src;            // MMFD_SRC_* (0: none)
    int nsrc;           // source fields per level (S, then M_1F components)
    double b[3], bhat[3];
    SrcCoef<double> sd;
    SrcCoef<float> sf;
    // two-level theta-scheme (Eq. (GCN)): right-hand side (I + theta L) phi^n as an LCDE stencil
    // (thr), Jacobi sweep x <- x_rhs / d + ((1 - theta) / d) (E - W0 I) x as an LCDE stencil (thj)
    // plus a centre-only source block (ths) with weight 1 / d, d = 1 + (1 - theta)(1 - W0)
    int dirichlet;      // MMFD_BC_DIRICHLET: boundary ring of nodes prescribed
    int theta_on;
    double theta;
    int sweeps;
    Coef<double> thr_d, thj_d;
    Coef<float> thr_f, thj_f;
    SrcCoef<double> ths_d;
    SrcCoef<float> ths_f;
};

// Returns MMFD_OK or an error code; *msg gets a human-readable reason on error.
int resolve(const mmfd_desc& d, Resolved& r, std::string* msg);

// Eq. (X): design targets (a_0, A_10, A_11, A_21, A_22) -> (a_{-1}, a_0, a_1), (ahat_{-1}, ahat_0, ahat_1).
int solve_three_level_targets(const double t[5], double a[3], double ah[3]);

// Frozen-coefficient stability (linstab.cpp): the largest amplification-factor modulus of the
// NCDE / NSE scheme linearised about the uniform state `state` (NCDE: phi; NSE: rho, u), over the
// grid's wave numbers (dense: every one up to 96 per axis, else up to 32, then a sample).
// Returns -1 for the linear PDEs.
double linear_amplification(const Resolved& r, const double* state, bool dense);

// Compulsory HBM bytes per lattice update: every stored level read once, one written.
double bytes_per_lu(const Resolved& r);

// Element size of a storage type.
inline int storage_bytes(int st) { return st == ST_F64 ? 8 : st == ST_F32 ? 4 : 2; }

}  // namespace mmfd
