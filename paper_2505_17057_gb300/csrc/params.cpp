// params.cpp -- problem descriptor -> scheme coefficients, EDF constants and the folded
// coefficient blocks the kernels consume.  Host only.
//
// Sources (arXiv 2505.17057): coefficient moments Eq. (4-2)/(4-2-0) (two-level, all terms on
// q = -1) and Eq. (4-2-00) (three-level, left-hand side at t + dt, Remark 1(5)); Eq. (X) for
// the three-level design; Eq. (LMMFD-2-2) for the two-level one; lattices of App. A; EDF
// Eq. (3-3)/(3-4); diffusion mapping alpha = -(A_22/A_10) dt beta c_s^2 (Eq. (M-NCDE-6)) with
// the second-order moment equation Eq. (ME-NCDE-3-2-1); stability symbol Eq. (TforMMFD-3).
#include "params.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

namespace mmfd {

namespace {

bool finite(double v) { return std::isfinite(v); }

// Weight of a lattice direction e (App. A) from d_0alpha.
double weight(int lat, const int e[3], const double d[3]) {
    const int nz = (e[0] != 0) + (e[1] != 0) + (e[2] != 0);
    switch (lat) {
    case LAT_D2Q5:
        if (nz == 0) return 1.0 - d[0] - d[1];
        return e[0] ? d[0] / 2 : d[1] / 2;
    case LAT_D3Q7:
        if (nz == 0) return 1.0 - d[0] - d[1] - d[2];
        return e[0] ? d[0] / 2 : e[1] ? d[1] / 2 : d[2] / 2;
    case LAT_D2Q9: {
        // product of one-dimensional factors w(0) = 1 - d, w(+-1) = d / 2
        double wx = e[0] ? d[0] / 2 : 1.0 - d[0];
        double wy = e[1] ? d[1] / 2 : 1.0 - d[1];
        return wx * wy;
    }
    case LAT_D3Q19:
        if (nz == 0) return 1.0 - d[0] - d[1] - d[2] + d[0] * d[1] + d[0] * d[2] + d[1] * d[2];
        if (nz == 1) {
            if (e[0]) return d[0] * (1.0 - d[1] - d[2]) / 2;
            if (e[1]) return d[1] * (1.0 - d[0] - d[2]) / 2;
            return d[2] * (1.0 - d[0] - d[1]) / 2;
        }
        if (nz == 2) {
            if (!e[2]) return d[0] * d[1] / 4;
            if (!e[1]) return d[0] * d[2] / 4;
            return d[1] * d[2] / 4;
        }
        return 0.0;
    }
    return 0.0;
}

// Directions of App. A in the paper's order (for the info block).
int lattice_dirs(int lat, int e[19][3]) {
    static const int d2q9[9][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
                                   {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
    static const int d3q19[19][3] = {{0, 0, 0},  {1, 0, 0},  {0, 1, 0},   {0, 0, 1},  {-1, 0, 0},
                                     {0, -1, 0}, {0, 0, -1}, {1, 1, 0},   {-1, 1, 0}, {-1, -1, 0},
                                     {1, -1, 0}, {1, 0, 1},  {-1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
                                     {0, 1, 1},  {0, -1, 1}, {0, -1, -1}, {0, 1, -1}};
    int b = 0;
    if (lat == LAT_D2Q5 || lat == LAT_D2Q9) {
        b = lat == LAT_D2Q5 ? 5 : 9;
        for (int j = 0; j < b; ++j) std::memcpy(e[j], d2q9[j], sizeof(e[j]));
    } else {
        b = lat == LAT_D3Q7 ? 7 : 19;
        for (int j = 0; j < b; ++j) std::memcpy(e[j], d3q19[j], sizeof(e[j]));
    }
    return b;
}

// Scheme moments A_10, A_20, A_21, A_22 from the coefficients.
void scheme_moments(int levels, const double a[3], const double ah[3], double& A10, double& A20,
                    double& A21, double& A22) {
    // a[k + 1] = a_k.
    const double s = a[0] + a[1] + a[2];
    const double k1 = a[2] - a[0];
    const double k2 = a[2] + a[0];
    if (levels == 2) {
        // every term at q = -1, left-hand side at t (Eq. (4-2-0))
        A10 = -s;
        A20 = 0.5 * s;
        A21 = -k1;
        A22 = 0.5 * k2;
    } else {
        // a_k at q = 0, ahat_k at q = -1, left-hand side at t + dt (Eq. (4-2-00a))
        const double sh = ah[0] + ah[1] + ah[2];
        A10 = -sh - 1.0;
        A20 = 0.5 * (sh - 1.0);
        A21 = -(ah[2] - ah[0]);
        A22 = 0.5 * (k2 + ah[2] + ah[0]);
    }
}

}  // namespace

int solve_three_level_targets(const double t[5], double a[3], double ah[3]) {
    const double a0 = t[0], A10 = t[1], A11 = t[2], A21 = t[3], A22 = t[4];
    for (int i = 0; i < 5; ++i)
        if (!finite(t[i])) return MMFD_ERR_ARG;
    // Eq. (X): X = A^{-1} b, b = (1 - a_0, 1 + A_10, A_11, A_21, A_22)
    a[2] = 0.5 * (-a0 + A10 + A11 + A21 + 2.0);
    a[0] = 0.5 * (-a0 + A10 - A11 - A21 + 2.0);
    a[1] = a0;
    ah[1] = 0.5 * (-2.0 * a0 - 4.0 * A22 + 2.0);
    ah[2] = 0.5 * (a0 - A10 - A21 + 2.0 * A22 - 2.0);
    ah[0] = 0.5 * (a0 - A10 + A21 + 2.0 * A22 - 2.0);
    return MMFD_OK;
}

static int coeffs_for(const mmfd_desc& d, const double* explicit_a, const double* explicit_ah,
                      const double* targets, double a[3], double ah[3]) {
    if (d.coef_mode == MMFD_COEF_EXPLICIT) {
        for (int i = 0; i < 3; ++i) {
            a[i] = explicit_a[i];
            ah[i] = d.levels == 3 ? explicit_ah[i] : 0.0;
        }
    } else if (d.coef_mode == MMFD_COEF_TARGETS) {
        if (d.levels == 2) {
            // Eq. (LMMFD-2-2), m = 1: A_00 = 1, A_10 = A_11 = -1
            const double a0 = targets[0];
            a[0] = 1.0 - 0.5 * a0;
            a[1] = a0;
            a[2] = -0.5 * a0;
            ah[0] = ah[1] = ah[2] = 0.0;
        } else if (solve_three_level_targets(targets, a, ah) != MMFD_OK) {
            return MMFD_ERR_ARG;
        }
    } else {
        return MMFD_ERR_ARG;
    }
    for (int i = 0; i < 3; ++i)
        if (!finite(a[i]) || !finite(ah[i])) return MMFD_ERR_ARG;
    return MMFD_OK;
}

// Lean He-Luo form (Coef::nA): whether the folded EDF coefficients of every pair p have the shape
//   E_p = eA_k rho + q_k |u|^2 + k_p (e_p . u)^2,   O_p = o_p (e_p . u)
// with eA_k, q_k shared by the axis pairs (k = 0) and by the diagonal pairs (k = 1), and an equal
// rest coefficient on every axis.  By Eq. (3-3)-(3-4) this holds with the same speed c on every
// axis on D2Q9 for any isotropic d_0 (a diagonal pair spans both axes, its cross term fixes k_p),
// and on D3Q19 for d_0 = 1/3 (only then does the cross term of a diagonal pair equal 2 k_p times
// the sign of e_pa e_pb, given q_k from the third axis).  Fills the per-level lean coefficients and returns LEAN_STREAM when
// every level's momentum set satisfies (abar-, abar+) = kappa (a+, a-) (a+ and a- then folded
// in), LEAN_GENERAL otherwise, LEAN_NONE when the shape does not hold.
static int nse_lean(Coef<double>& c, int lat, int dim, int levels) {
    auto close = [](double x, double y) { return x == y || std::fabs(x - y) <= 1e-13 * (std::fabs(x) + std::fabs(y)); };
    const int NP = lat_npair(lat);
    double q[kMaxPair], k[kMaxPair], o[kMaxPair];
    int cls[kMaxPair];
    for (int p = 0; p < NP; ++p) {
        int in[3], out[3], nin = 0, nout = 0;
        for (int a = 0; a < dim; ++a) {
            if (pair_e(lat, p, a) != 0) in[nin++] = a;
            else out[nout++] = a;
        }
        if (nin < 1 || nin > 2) return LEAN_NONE;
        cls[p] = nin - 1;
        double cross = 0.0;
        int sgn = 1;
        if (nin == 2) {
            const int a = in[0], b = in[1];
            cross = c.eC[p][(a == 0 && b == 1) ? 3 : (a == 0 && b == 2) ? 4 : 5];
            sgn = pair_e(lat, p, a) * pair_e(lat, p, b);
        }
        if (nout > 0) {
            q[p] = c.eC[p][out[0]];
            for (int i = 1; i < nout; ++i)
                if (!close(c.eC[p][out[i]], q[p])) return LEAN_NONE;
        } else {
            q[p] = c.eC[p][in[0]] - 0.5 * cross * sgn;   // 2D diagonal pairs: the cross term fixes k
        }
        k[p] = c.eC[p][in[0]] - q[p];
        for (int i = 1; i < nin; ++i)
            if (!close(c.eC[p][in[i]] - q[p], k[p])) return LEAN_NONE;
        if (nin == 2 && !close(cross, 2.0 * k[p] * sgn)) return LEAN_NONE;
        o[p] = c.oB[p][in[0]] * pair_e(lat, p, in[0]);
        for (int i = 1; i < nin; ++i)
            if (!close(c.oB[p][in[i]] * pair_e(lat, p, in[i]), o[p])) return LEAN_NONE;
    }
    double eAk[2] = {0.0, 0.0}, qk[2] = {0.0, 0.0};
    bool seen[2] = {false, false};
    for (int p = 0; p < NP; ++p) {
        const int kk = cls[p];
        if (!seen[kk]) {
            seen[kk] = true;
            eAk[kk] = c.eA[p];
            qk[kk] = q[p];
        } else if (!close(c.eA[p], eAk[kk]) || !close(q[p], qk[kk])) {
            return LEAN_NONE;
        }
    }
    for (int a = 1; a < dim; ++a)
        if (!close(c.rC[a], c.rC[0])) return LEAN_NONE;
    const int nl = levels == 3 ? 2 : 1;
    bool stream = true;
    double kap[2] = {0.0, 0.0};
    for (int l = 0; l < nl; ++l) {
        const double ap = c.ap[l], am = c.am[l], bp = c.abp[l], bm = c.abm[l];
        if (std::fabs(bm * am - bp * ap) > 1e-13 * (std::fabs(bm * am) + std::fabs(bp * ap))) {
            stream = false;
        } else if (ap != 0.0 || am != 0.0) {
            kap[l] = ap != 0.0 ? bm / ap : bp / am;
        } else if (bm != 0.0 || bp != 0.0) {
            stream = false;   // the level moves momentum but no scalar
        }
    }
    for (int l = 0; l < nl; ++l) {
        const double sE = stream ? c.ap[l] : 1.0, sO = stream ? c.am[l] : 1.0;
        for (int kk = 0; kk < 2; ++kk) {
            c.nA[l][kk] = sE * eAk[kk];
            c.nU[l][kk] = sE * qk[kk];
        }
        for (int p = 0; p < NP; ++p) {
            c.nk[l][p] = sE * k[p];
            c.no[l][p] = sO * o[p];
        }
        c.nc[l][0] = c.a0[l] + c.ap[l] * c.rA;
        c.nc[l][1] = c.ap[l] * c.rC[0];
        for (int a = 0; a < dim; ++a) c.nsm[l][a] = stream ? kap[l] * c.fmom[a] : 0.0;
    }
    return stream ? LEAN_STREAM : LEAN_GENERAL;
}

static int fail(std::string* msg, int code, const char* why) {
    if (msg) *msg = why;
    return code;
}

int resolve(const mmfd_desc& d_in, Resolved& r, std::string* msg) {
    std::memset(&r, 0, sizeof(r));
    if (d_in.pde < PDE_LCDE || d_in.pde > MMFD_LWE) return fail(msg, MMFD_ERR_ARG, "unknown pde");
    // the wave equation (Eq. (LWE)) is a linear-EDF scheme like the LCDE: its own mapping of K
    // onto the EDF, the LCDE's kernels
    const bool wave = d_in.pde == MMFD_LWE;
    mmfd_desc d = d_in;
    if (wave) d.pde = PDE_LCDE;
    if (d.lattice < LAT_D2Q5 || d.lattice > LAT_D3Q19) return fail(msg, MMFD_ERR_ARG, "unknown lattice");
    if (d.levels != 2 && d.levels != 3) return fail(msg, MMFD_ERR_ARG, "levels must be 2 or 3");
    if (d.storage < ST_F64 || d.storage > ST_BF16) return fail(msg, MMFD_ERR_ARG, "unknown storage");
    const int dim = lat_dim(d.lattice);
    if (d.dim != dim) return fail(msg, MMFD_ERR_ARG, "dim does not match the lattice");
    for (int a = 0; a < 3; ++a) {
        const long long n = d.n[a];
        if (a < dim && (n < 1 || n > (1ll << 20))) return fail(msg, MMFD_ERR_ARG, "grid size out of range");
        if (a >= dim && n != 1) return fail(msg, MMFD_ERR_ARG, "n[2] must be 1 in 2D");
    }
    if (!(d.dt > 0) || !finite(d.dt)) return fail(msg, MMFD_ERR_ARG, "dt must be positive");
    for (int a = 0; a < dim; ++a)
        if (!(d.dx[a] > 0) || !finite(d.dx[a])) return fail(msg, MMFD_ERR_ARG, "dx must be positive");
    if ((d.pde == PDE_NSE || d.pde == PDE_NCDE) && (d.lattice == LAT_D2Q5 || d.lattice == LAT_D3Q7))
        return fail(msg, MMFD_ERR_UNSUPPORTED,
                    "NSE and NCDE need the quadratic EDF moments of D2Q9/D3Q19 (axis lattices cannot carry C)");

    r.pde = d.pde;
    r.lat = d.lattice;
    r.levels = d.levels;
    r.dim = dim;
    r.nf = pde_nf(d.pde, d.lattice);
    r.st = d.storage;
    for (int a = 0; a < 3; ++a) r.n[a] = d.n[a];

    if (coeffs_for(d, d.a, d.ahat, d.targets, r.a, r.ahat) != MMFD_OK)
        return fail(msg, MMFD_ERR_ARG, "bad scheme coefficients");
    if (d.pde == PDE_NSE) {
        if (coeffs_for(d, d.abar, d.abarhat, d.targets_bar, r.abar, r.abarhat) != MMFD_OK)
            return fail(msg, MMFD_ERR_ARG, "bad momentum coefficients");
    }
    // A_00 = 1 (Eq. (4-2-0)); a scheme violating it does not conserve mass.
    const double A00 = r.a[0] + r.a[1] + r.a[2] + (d.levels == 3 ? r.ahat[0] + r.ahat[1] + r.ahat[2] : 0.0);
    if (std::fabs(A00 - 1.0) > 1e-12) return fail(msg, MMFD_ERR_ARG, "coefficients violate A_00 = 1");
    if (d.flags & MMFD_FLAG_TWO_SETS) {
        for (int l = 0; l < 2; ++l)
            for (int k = 0; k < 3; ++k)
                if (!finite(d.d2[l][k]) || !finite(d.d1[l][k]) || !finite(d.bar_d2[l][k]) || !finite(d.bar_d1[l][k]))
                    return fail(msg, MMFD_ERR_ARG, "non-finite coefficient in the parameter sets");
    }
    if (d.pde == PDE_NSE) {
        const double Ab00 = r.abar[0] + r.abar[1] + r.abar[2] +
                            (d.levels == 3 ? r.abarhat[0] + r.abarhat[1] + r.abarhat[2] : 0.0);
        if (std::fabs(Ab00 - 1.0) > 1e-12) return fail(msg, MMFD_ERR_ARG, "momentum coefficients violate Abar_00 = 1");
    }
    scheme_moments(d.levels, r.a, r.ahat, r.A10, r.A20, r.A21, r.A22);
    if (wave) {
        // Sec. III.B (3): A_20 = -1 and A_lm = 0 except (2, 0), (2, 2) among the moments the
        // second-order equation sees, so that d_t^2 phi = A_22 div div M_2 (Eq. (ME-NCDE-W))
        if (d.levels != 3) return fail(msg, MMFD_ERR_ARG, "the wave equation needs a three-level scheme");
        const double A11 = r.a[2] - r.a[0] + r.ahat[2] - r.ahat[0];
        if (std::fabs(r.A10) > 1e-12 || std::fabs(A11) > 1e-12 || std::fabs(r.A21) > 1e-12 ||
            std::fabs(r.A20 + 1.0) > 1e-12 || !(std::fabs(r.A22) > 0.0))
            return fail(msg, MMFD_ERR_ARG,
                        "wave equation: coefficients must give A_10 = A_11 = A_21 = 0, A_20 = -1, A_22 != 0");
        for (int a = 0; a < 3; ++a)
            if (d.u[a] != 0.0) return fail(msg, MMFD_ERR_ARG, "wave equation: u must be zero");
        if (d.source != MMFD_SRC_NONE) return fail(msg, MMFD_ERR_UNSUPPORTED, "wave equation: no source terms");
    }

    for (int a = 0; a < 3; ++a) r.c[a] = a < dim ? d.dx[a] / d.dt : 0.0;

    // ---- lattice parameters and the EDF's C per unit phi (LCDE)
    const bool axis = (d.lattice == LAT_D2Q5 || d.lattice == LAT_D3Q7);
    std::memset(r.Cmat, 0, sizeof(r.Cmat));
    if (d.pde == PDE_LCDE) {
        for (int a = 0; a < dim; ++a)
            for (int b = 0; b < dim; ++b)
                if (!finite(d.K[a][b]) || std::fabs(d.K[a][b] - d.K[b][a]) > 1e-14 * (1 + std::fabs(d.K[a][b])))
                    return fail(msg, MMFD_ERR_ARG, "K must be finite and symmetric");
        if (!wave && (r.A10 == 0.0 || r.A22 == 0.0)) return fail(msg, MMFD_ERR_ARG, "A_10 and A_22 must be nonzero for a CDE");
    }
    if (axis) {
        // Linear EDF (C = 0) with direction-dependent c_salpha^2 chosen so that the recovered
        // diffusion K_eff = -(dt/A_10)[A_22 diag(c_s^2) - (A_21 - A_20) u u] (Eq. (ME-NCDE-3-2-1))
        // has the requested diagonal.  The off-diagonal cannot be carried (no c_x c_y != 0).
        bool offdiag = false;
        for (int a = 0; a < dim; ++a)
            for (int b = 0; b < dim; ++b)
                if (a != b && d.K[a][b] != 0.0) offdiag = true;
        if (offdiag && !(d.flags & MMFD_FLAG_DROP_OFFDIAG))
            return fail(msg, MMFD_ERR_UNREPRESENTABLE,
                        "off-diagonal diffusion cannot be represented on an axis lattice (set MMFD_FLAG_DROP_OFFDIAG)");
        double sum = 0.0;
        for (int a = 0; a < dim; ++a) {
            // LCDE: Eq. (ME-NCDE-3-2-1); wave: second moment K phi / A_22 (Eq. (ME-NCDE-W-1))
            const double cs2 = wave ? d.K[a][a] / r.A22
                                    : (-r.A10 * d.K[a][a] / d.dt + (r.A21 - r.A20) * d.u[a] * d.u[a]) / r.A22;
            r.cs2[a] = cs2;
            r.d0[a] = cs2 / (r.c[a] * r.c[a]);
            if (!(r.d0[a] > 0.0) || !finite(r.d0[a])) return fail(msg, MMFD_ERR_ARG, "derived d_0 must be positive");
            sum += r.d0[a];
        }
        if (!(sum < 1.0)) return fail(msg, MMFD_ERR_UNSTABLE, "derived d_0 sum >= 1: negative rest weight (App. A)");
    } else {
        for (int a = 0; a < dim; ++a) {
            r.d0[a] = d.d0[a];
            if (!(r.d0[a] > 0.0 && r.d0[a] < 1.0)) return fail(msg, MMFD_ERR_ARG, "d_0 must lie in (0, 1)");
            r.cs2[a] = r.d0[a] * r.c[a] * r.c[a];
        }
        if (d.pde == PDE_LCDE) {
            // C = c_s^2 (beta D0 - I) + lambda_bar u u with c_s^2 beta D0 = -A_10 K / (A_22 dt)
            for (int a = 0; a < dim; ++a)
                for (int b = 0; b < dim; ++b)
                    r.Cmat[a][b] = wave ? d.K[a][b] / r.A22
                                        : -r.A10 * d.K[a][b] / (r.A22 * d.dt) + d.lambda_bar * d.u[a] * d.u[b];
            for (int a = 0; a < dim; ++a) r.Cmat[a][a] -= r.cs2[a];
        }
    }
    if (d.pde == PDE_NCDE) {
        if (r.A10 == 0.0 || r.A22 == 0.0) return fail(msg, MMFD_ERR_ARG, "A_10 and A_22 must be nonzero for a CDE");
        // alpha D = G(phi) I with G' = D(phi), G(0) = 0 (Eq. (M-NCDE-6)): second-moment target
        // beta c_s^2 D = -(A_10 / (A_22 dt)) G(phi) I.
        std::memset(r.m2, 0, sizeof(r.m2));
        for (int p = 0; p < 4; ++p) r.m2[p + 1] = -r.A10 * d.diff[p] / ((p + 1) * r.A22 * d.dt);
    }
    if (d.pde == PDE_NSE && !(d.rho0 > 0.0)) return fail(msg, MMFD_ERR_ARG, "rho0 must be positive");

    // ---- weights in App. A order
    int e[19][3];
    const int b = lattice_dirs(d.lattice, e);
    for (int j = 0; j < b; ++j) {
        r.w[j] = weight(d.lattice, e[j], r.d0);
        if (!(r.w[j] >= 0.0)) return fail(msg, MMFD_ERR_ARG, "lattice weights must be non-negative (App. A)");
    }

    // ---- storage offsets: FP32 and BF16 levels hold v - ref.  FP64 levels, and FP32 levels of the
    // NCDE (whose update is nonlinear in phi and runs on values), hold values.  The NSE velocity
    // reference must be zero: the update runs on the stored offsets, and it is affine in the
    // density only.
    for (int f = 0; f < 4; ++f) {
        double v = d.ref[f];
        if (std::isnan(v)) v = (d.pde == PDE_NSE && f == 0) ? d.rho0 : 0.0;
        if (!finite(v)) return fail(msg, MMFD_ERR_ARG, "non-finite storage reference");
        if (d.storage == ST_F64 || (d.storage == ST_F32 && d.pde == PDE_NCDE)) v = 0.0;
        if (d.pde == PDE_NSE && f >= 1 && f < r.nf && v != 0.0)
            return fail(msg, MMFD_ERR_ARG, "NSE velocity references must be zero");
        r.ref[f] = v;
    }

    // ---- folded kernel coefficients (double)
    Coef<double>& c = r.cd;
    std::memset(&c, 0, sizeof(c));
    const int NP = lat_npair(d.lattice);
    const int zero[3] = {0, 0, 0};
    const double w0 = weight(d.lattice, zero, r.d0);
    const double rho0 = d.pde == PDE_NSE ? d.rho0 : 1.0;
    for (int p = 0; p < NP; ++p) {
        int ep[3];
        double cp[3];
        for (int a = 0; a < 3; ++a) {
            ep[a] = a < dim ? pair_e(d.lattice, p, a) : 0;
            cp[a] = ep[a] * r.c[a];
        }
        const double wp = weight(d.lattice, ep, r.d0);
        c.eA[p] = wp;
        for (int a = 0; a < dim; ++a) {
            // Qtilde_paa = (c_pa^2 - cs_a^2) / (cs_a^2 (c_a^2 - cs_a^2)) (Eq. (3-4))
            c.eC[p][a] = wp * (cp[a] * cp[a] - r.cs2[a]) / (r.cs2[a] * (r.c[a] * r.c[a] - r.cs2[a]));
            c.oB[p][a] = wp * cp[a] / r.cs2[a];
        }
        // off-diagonal: both orderings of Qtilde_pab = c_pa c_pb / (2 cs_a^2 cs_b^2)
        c.eC[p][3] = wp * cp[0] * cp[1] / (r.cs2[0] * r.cs2[1]);
        if (dim == 3) {
            c.eC[p][4] = wp * cp[0] * cp[2] / (r.cs2[0] * r.cs2[2]);
            c.eC[p][5] = wp * cp[1] * cp[2] / (r.cs2[1] * r.cs2[2]);
        }
        if (axis) {
            // linear EDF: no C terms at all
            for (int k = 0; k < 6; ++k) c.eC[p][k] = 0.0;
        }
    }
    c.rA = w0;
    for (int a = 0; a < dim; ++a) c.rC[a] = axis ? 0.0 : -w0 / (r.c[a] * r.c[a] - r.cs2[a]);

    const double* sets[2] = {r.a, r.ahat};
    const double* bsets[2] = {r.abar, r.abarhat};
    const bool two = (d.flags & MMFD_FLAG_TWO_SETS) != 0;
    for (int l = 0; l < 2; ++l) {
        // pair form of one level: a0 A(x) + ap f_0^eq(x) + sum_p [ap (E_p(+) + E_p(-)) + am (O_p(+) - O_p(-))].
        // One set (Eq. (2-2-1)): ap = a_1 + a_{-1}, am = a_1 - a_{-1}, a0 = a_0.  Several sets
        // (Eq. (2-2-1b)): the zeroth-order term sum_k a_k A(x) plus the second difference of the
        // even parts with d2 and the first difference of the odd parts with d1, which expands
        // to ap = d2^+, am = d1^-, a0 = sum_k a_k - d2^+.  The momentum likewise, with bar_d2 on
        // the odd parts' second difference (abp) and bar_d1 on the even parts' first (abm).
        const double* e2 = two ? d.d2[l] : sets[l];
        const double* o1 = two ? d.d1[l] : sets[l];
        const double* be2 = two ? d.bar_d2[l] : bsets[l];
        const double* bo1 = two ? d.bar_d1[l] : bsets[l];
        c.ap[l] = e2[2] + e2[0];
        c.am[l] = o1[2] - o1[0];
        c.a0[l] = two ? sets[l][0] + sets[l][1] + sets[l][2] - c.ap[l] : sets[l][1];
        c.abp[l] = be2[2] + be2[0];
        c.abm[l] = bo1[2] - bo1[0];
        c.ab0[l] = two ? bsets[l][0] + bsets[l][1] + bsets[l][2] - c.abp[l] : bsets[l][1];
    }
    for (int a = 0; a < dim; ++a) c.fmom[a] = r.c[a] / rho0;

    if (d.pde == PDE_LCDE) {
        // f^eq = phi ubar: E_p = phi ebar_p, O_p = phi obar_p -> collapsed stencil weights
        double rbar = c.rA;
        for (int a = 0; a < dim; ++a) rbar += c.rC[a] * r.Cmat[a][a];
        for (int l = 0; l < 2; ++l) c.W0[l] = c.a0[l] + c.ap[l] * rbar;
        for (int p = 0; p < NP; ++p) {
            double eb = c.eA[p];
            for (int a = 0; a < dim; ++a) eb += c.eC[p][a] * r.Cmat[a][a];
            eb += c.eC[p][3] * r.Cmat[0][1];
            if (dim == 3) eb += c.eC[p][4] * r.Cmat[0][2] + c.eC[p][5] * r.Cmat[1][2];
            double ob = 0.0;
            for (int a = 0; a < dim; ++a) ob += c.oB[p][a] * d.u[a];
            for (int l = 0; l < 2; ++l) {
                c.Wp[l][p] = c.ap[l] * eb + c.am[l] * ob;
                c.Wm[l][p] = c.ap[l] * eb - c.am[l] * ob;
            }
        }
    } else if (d.pde == PDE_NCDE) {
        for (int a = 0; a < dim; ++a)
            for (int k = 0; k < 4; ++k) c.flux[a][k] = d.flux[a][k];
        for (int k = 0; k < 5; ++k) c.m2[k] = r.m2[k];
        for (int p = 0; p < NP; ++p) {
            double ephi = c.eA[p], em2 = 0.0;
            for (int a = 0; a < dim; ++a) {
                ephi -= c.eC[p][a] * r.cs2[a];
                em2 += c.eC[p][a];
            }
            c.ePhi[p] = ephi;
            c.eM2[p] = em2;
        }
        c.rPhi = c.rA;
        c.rM2 = 0.0;
        for (int a = 0; a < dim; ++a) {
            c.rPhi -= c.rC[a] * r.cs2[a];
            c.rM2 += c.rC[a];
        }
    } else {
        // He-Luo: fold rho0 into the u u and u terms
        for (int p = 0; p < NP; ++p) {
            for (int k = 0; k < 6; ++k) c.eC[p][k] *= rho0;
            for (int a = 0; a < 3; ++a) c.oB[p][a] *= rho0;
        }
        for (int a = 0; a < 3; ++a) c.rC[a] *= rho0;
    }
    for (int f = 0; f < 4; ++f) c.ref[f] = r.ref[f];
    r.lean = (d.pde == PDE_NSE && !axis) ? nse_lean(c, d.lattice, dim, d.levels) : LEAN_NONE;

    // float copy
    {
        const double* src = reinterpret_cast<const double*>(&r.cd);
        float* dst = reinterpret_cast<float*>(&r.cf);
        static_assert(sizeof(Coef<double>) == 2 * sizeof(Coef<float>), "Coef layout");
        for (size_t i = 0; i < sizeof(Coef<double>) / sizeof(double); ++i) dst[i] = (float)src[i];
    }

    // ---- source terms (Eq. (2-1); F_j = g_j^eq(S, M_1F, 0), Eq. (SourceF)), folded per level
    // from the central form Eq. (3layerMMFD-2): omega_p = eA[p], omega_p ctilde_p = oB[p].
    r.src = d.source;
    if (d.source < MMFD_SRC_NONE || d.source > MMFD_SRC_SM) return fail(msg, MMFD_ERR_ARG, "unknown source mode");
    if (d.source != MMFD_SRC_NONE) {
        if (d.pde == PDE_NSE) return fail(msg, MMFD_ERR_UNSUPPORTED, "source terms: LCDE and NCDE only");
        if (d.source == MMFD_SRC_SU && d.pde != PDE_LCDE)
            return fail(msg, MMFD_ERR_ARG, "MMFD_SRC_SU takes the LCDE's velocity u");
        bool zero = true;
        for (int k = 0; k < 3; ++k) {
            if (!finite(d.b[k]) || !finite(d.bhat[k])) return fail(msg, MMFD_ERR_ARG, "non-finite source coefficient");
            if (d.b[k] != 0.0 || d.bhat[k] != 0.0) zero = false;
        }
        if (d.levels == 2 && (d.bhat[0] != 0.0 || d.bhat[1] != 0.0 || d.bhat[2] != 0.0))
            return fail(msg, MMFD_ERR_ARG, "bhat must be zero for a two-level solver");
        for (int k = 0; k < 3; ++k) {
            r.b[k] = d.b[k];
            r.bhat[k] = d.bhat[k];
        }
        if (zero) {
            r.b[0] = d.levels == 3 ? 1.5 : 1.0;
            r.bhat[0] = d.levels == 3 ? -0.5 : 0.0;
        }
        r.nsrc = d.source == MMFD_SRC_SM ? 1 + dim : 1;
        SrcCoef<double>& sc = r.sd;
        std::memset(&sc, 0, sizeof(sc));
        const double* bl[2] = {r.b, r.bhat};
        double wsum = 0.0;
        for (int p = 0; p < NP; ++p) wsum += c.eA[p];
        for (int l = 0; l < d.levels - 1; ++l) {
            const double B0 = bl[l][0] + bl[l][1] + bl[l][2];
            const double bp = bl[l][2] + bl[l][0], bm = bl[l][2] - bl[l][0];
            sc.W0[l] = d.dt * (B0 - 2.0 * bp * wsum);
            for (int p = 0; p < NP; ++p) {
                double cu = 0.0;  // ctilde_p . u (M_1F = S u), per unit omega_p
                if (d.source == MMFD_SRC_SU)
                    for (int a = 0; a < dim; ++a) cu += c.oB[p][a] * d.u[a];
                sc.Wp[l][p] = d.dt * (bp * c.eA[p] + bm * cu);
                sc.Wm[l][p] = d.dt * (bp * c.eA[p] - bm * cu);
                if (d.source == MMFD_SRC_SM)
                    for (int a = 0; a < dim; ++a) sc.M[l][p][a] = d.dt * bm * c.oB[p][a];
            }
        }
        const double* ssrc = reinterpret_cast<const double*>(&r.sd);
        float* sdst = reinterpret_cast<float*>(&r.sf);
        static_assert(sizeof(SrcCoef<double>) == 2 * sizeof(SrcCoef<float>), "SrcCoef layout");
        for (size_t i = 0; i < sizeof(SrcCoef<double>) / sizeof(double); ++i) sdst[i] = (float)ssrc[i];
    }

    // ---- two-level theta-scheme (Eq. (GCN)).  With phi + L phi the explicit update above (E = I + L,
    // the collapsed stencil of level t), a step solves (I - theta_1 L) x = (I + theta L) phi^n,
    // theta_1 = 1 - theta.  The right-hand side is the stencil (1 - theta) I + theta E; the
    // system is solved by Jacobi sweeps on its diagonal d = 1 + theta_1 (1 - W0):
    //     x <- rhs / d + (theta_1 / d) (E - W0 I) x,
    // i.e. an LCDE stencil without a centre weight plus a centre-only source term rhs / d.  The
    // sweep contracts by at most rho = theta_1 sum_p (|Wp| + |Wm|) / d per step.
    // ---- boundary treatment
    if (d.boundary != MMFD_BC_PERIODIC && d.boundary != MMFD_BC_DIRICHLET)
        return fail(msg, MMFD_ERR_ARG, "unknown boundary treatment");
    r.dirichlet = d.boundary == MMFD_BC_DIRICHLET ? 1 : 0;
    if (r.dirichlet) {
        for (int a = 0; a < dim; ++a)
            if (d.n[a] < 3) return fail(msg, MMFD_ERR_ARG, "Dirichlet boundaries need at least 3 nodes along every axis");
        if (d.flags & MMFD_FLAG_THETA)
            return fail(msg, MMFD_ERR_UNSUPPORTED, "the theta-scheme is built for periodic grids");
    }

    r.theta_on = (d.flags & MMFD_FLAG_THETA) != 0 ? 1 : 0;
    r.theta = 1.0;
    r.sweeps = 0;
    double th_dg = 1.0, th_w0 = 0.0;
    if (r.theta_on) {
        if (!(d.theta >= 0.0 && d.theta <= 1.0)) return fail(msg, MMFD_ERR_ARG, "theta must lie in [0, 1]");
        if (d_in.pde != PDE_LCDE) return fail(msg, MMFD_ERR_UNSUPPORTED, "the theta-scheme is built for the LCDE");
        if (d.levels != 2) return fail(msg, MMFD_ERR_UNSUPPORTED, "the theta-scheme is a two-level scheme");
        if (d.source != MMFD_SRC_NONE) return fail(msg, MMFD_ERR_UNSUPPORTED, "theta-scheme: no source terms");
        if (d.storage == ST_BF16)
            return fail(msg, MMFD_ERR_UNSUPPORTED, "theta-scheme: FP64 or FP32 storage (the iteration stalls at BF16 rounding)");
        r.theta = d.theta;
        const double th = d.theta, th1 = 1.0 - d.theta;
        double woff = 0.0;
        for (int p = 0; p < NP; ++p) woff += std::fabs(c.Wp[0][p]) + std::fabs(c.Wm[0][p]);
        const double dg = 1.0 + th1 * (1.0 - c.W0[0]);
        if (!(dg > 0.0) || !(th1 * woff / dg < 1.0))
            return fail(msg, MMFD_ERR_UNSUPPORTED, "theta-scheme: the Jacobi iteration does not contract");
        th_dg = dg;
        th_w0 = c.W0[0];
        Coef<double>& R = r.thr_d;
        Coef<double>& J = r.thj_d;
        R = c;
        J = c;
        R.W0[0] = th1 + th * c.W0[0];
        J.W0[0] = 0.0;
        R.W0[1] = J.W0[1] = 0.0;
        for (int p = 0; p < kMaxPair; ++p) {
            R.Wp[0][p] = th * c.Wp[0][p];
            R.Wm[0][p] = th * c.Wm[0][p];
            J.Wp[0][p] = th1 * c.Wp[0][p] / dg;
            J.Wm[0][p] = th1 * c.Wm[0][p] / dg;
            R.Wp[1][p] = R.Wm[1][p] = J.Wp[1][p] = J.Wm[1][p] = 0.0;
        }
        std::memset(&r.ths_d, 0, sizeof(r.ths_d));
        r.ths_d.W0[0] = 1.0 / dg;
        const double* srcs[3] = {reinterpret_cast<const double*>(&r.thr_d), reinterpret_cast<const double*>(&r.thj_d),
                                 reinterpret_cast<const double*>(&r.ths_d)};
        float* dsts[3] = {reinterpret_cast<float*>(&r.thr_f), reinterpret_cast<float*>(&r.thj_f),
                          reinterpret_cast<float*>(&r.ths_f)};
        const size_t counts[3] = {sizeof(Coef<double>) / sizeof(double), sizeof(Coef<double>) / sizeof(double),
                                  sizeof(SrcCoef<double>) / sizeof(double)};
        for (int b = 0; b < 3; ++b)
            for (size_t i = 0; i < counts[b]; ++i) dsts[b][i] = (float)srcs[b][i];
    }

    // ---- create-time stability check (LCDE: exact symbol on the grid's wave numbers)
    r.max_lambda = -1.0;
    if (d.pde == PDE_LCDE) {
        // Wave numbers per axis over the whole band: all of them up to 96 nodes, else the 16
        // smallest of either sign (where convection-driven growth lives) and a uniform sweep of
        // 64.  The weights are real, so the symbol at -xi is the conjugate of that at xi: the
        // last axis takes only [0, pi].  The phase of pair p is a product of per-axis phasors.
        const int last = dim - 1;
        std::vector<std::complex<double>> ph[3];
        for (int a = 0; a < 3; ++a) {
            const long long n = a < dim ? d.n[a] : 1;
            std::vector<long long> ms;
            if (n <= 96) {
                for (long long m = 0; m < n; ++m) ms.push_back(m);
            } else {
                for (long long m = 0; m <= 16; ++m) {
                    ms.push_back(m);
                    if (m > 0) ms.push_back(n - m);
                }
                for (int m = 1; m < 64; ++m) ms.push_back((long long)((double)m * n / 64.0));
            }
            for (long long m : ms) {
                if (a == last && 2 * m > n) continue;
                ph[a].push_back(std::polar(1.0, 6.283185307179586 * (double)m / (double)n));
            }
        }
        int pe[kMaxPair][3];
        for (int p = 0; p < NP; ++p)
            for (int a = 0; a < 3; ++a) pe[p][a] = a < dim ? pair_e(d.lattice, p, a) : 0;
        const int nl = d.levels == 3 ? 2 : 1;
        double lmax = 0.0;
        // theta-scheme: per Fourier mode the sweeps start from phi^n, whose error is
        // ell / (1 - theta_1 ell) phi_hat^n, and multiply it by g = theta_1 (A - W0) / d each; the
        // sweep count takes every mode's error below the storage type's rounding
        const double th_eps = d.storage == ST_F64 ? 1e-15 : 6e-8;
        int th_k = 1;
        bool sampled = false;
        for (int a = 0; a < dim; ++a) sampled = sampled || d.n[a] > 96;
        for (const std::complex<double>& qz : ph[2])
            for (const std::complex<double>& qy : ph[1])
                for (const std::complex<double>& qx : ph[0]) {
                    const std::complex<double> q[3] = {qx, qy, qz};
                    std::complex<double> e[kMaxPair];
                    for (int p = 0; p < NP; ++p) {
                        std::complex<double> v(1.0, 0.0);
                        for (int a = 0; a < 3; ++a) {
                            if (pe[p][a] == 1) v *= q[a];
                            else if (pe[p][a] == -1) v *= std::conj(q[a]);
                        }
                        e[p] = v;
                    }
                    // W_p e^{i phase} + W_m e^{-i phase}
                    std::complex<double> A[2] = {0.0, 0.0};
                    for (int l = 0; l < nl; ++l) {
                        double re = c.W0[l], im = 0.0;
                        for (int p = 0; p < NP; ++p) {
                            re += (c.Wp[l][p] + c.Wm[l][p]) * e[p].real();
                            im += (c.Wp[l][p] - c.Wm[l][p]) * e[p].imag();
                        }
                        A[l] = std::complex<double>(re, im);
                    }
                    double m;
                    if (r.theta_on) {
                        // Eq. (Tcond1-1): lambda = (1 + theta ell) / (1 - theta_1 ell), ell = A - 1
                        const std::complex<double> ell = A[0] - 1.0;
                        const std::complex<double> den = 1.0 - (1.0 - r.theta) * ell;
                        m = std::abs(den) > 0.0 ? std::abs((1.0 + r.theta * ell) / den) : HUGE_VAL;
                        const double e0 = std::abs(den) > 0.0 ? std::abs(ell) / std::abs(den) : HUGE_VAL;
                        const double gm = (1.0 - r.theta) * std::abs(A[0] - th_w0) / th_dg;
                        if (e0 > th_eps && gm > 0.0) {
                            const double kk = std::ceil(std::log(th_eps / e0) / std::log(gm));
                            th_k = (int)std::min(1e6, std::max((double)th_k, kk));
                        }
                    } else if (d.levels == 2) {
                        m = std::abs(A[0]);
                    } else {
                        // roots of lambda^2 - p1 lambda - p0 (Eq. (3-level)); a vanishing
                        // discriminant is the double root p1 / 2 (the wave scheme's constant mode:
                        // the quadratic formula would put it at 1 +- O(sqrt(eps)))
                        const std::complex<double> d2 = A[0] * A[0] + 4.0 * A[1];
                        if (std::abs(d2) <= 1e-13 * std::max(1.0, std::norm(A[0]))) {
                            m = std::abs(0.5 * A[0]);
                        } else {
                            const std::complex<double> disc = std::sqrt(d2);
                            m = std::max(std::abs(0.5 * (A[0] + disc)), std::abs(0.5 * (A[0] - disc)));
                        }
                    }
                    if (m > lmax) lmax = m;
                }
        r.max_lambda = lmax;
        if (lmax > 1.0 + 1e-12 && !(d.flags & MMFD_FLAG_ALLOW_UNSTABLE))
            return fail(msg, MMFD_ERR_UNSTABLE, "max |lambda| > 1 on the grid's wave numbers");
        if (r.theta_on) {
            // theta = 1: one sweep (x = rhs).  On sampled wave numbers one sweep more as margin.
            int k = r.theta == 1.0 ? 1 : th_k + (sampled ? 1 : 0);
            if (k > 20000)
                return fail(msg, MMFD_ERR_UNSUPPORTED, "theta-scheme: the Jacobi iteration would need more than 20000 sweeps");
            r.sweeps = k;
        }
    }
    if (d.pde == PDE_NCDE || d.pde == PDE_NSE) {
        // nonlinear schemes: frozen-coefficient check about the reference state -- the NCDE at
        // phi = ref[0] (0 unless given), the NSE at rest (rho0, u = 0); see linstab.cpp
        double st[4] = {0.0, 0.0, 0.0, 0.0};
        st[0] = d.pde == PDE_NSE ? d.rho0 : (std::isnan(d.ref[0]) ? 0.0 : d.ref[0]);
        const double lmax = linear_amplification(r, st, false);
        r.max_lambda = lmax;
        if (lmax > 1.0 + 1e-9 && !(d.flags & MMFD_FLAG_ALLOW_UNSTABLE))
            return fail(msg, MMFD_ERR_UNSTABLE,
                        "max |lambda| > 1 for the scheme linearised about the reference state");
    }
    return MMFD_OK;
}

double bytes_per_lu(const Resolved& r) {
    // theta-scheme: the right-hand side reads the level and writes rhs; each Jacobi sweep reads
    // the iterate and rhs and writes the next iterate
    if (r.theta_on) return (double)storage_bytes(r.st) * (2.0 + 3.0 * r.sweeps);
    // levels read and the one written; source levels (compute type) read once per step
    const double src = r.src ? (double)(r.st == ST_F64 ? 8 : 4) * r.nsrc * (r.levels - 1) : 0.0;
    return (double)storage_bytes(r.st) * r.nf * (r.levels - 1 + 1) + src;
}

}  // namespace mmfd
