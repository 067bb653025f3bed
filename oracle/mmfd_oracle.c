/*
 * mmfd_oracle.c -- plain, slow, FP64 CPU oracle for the explicit MMFD update
 * (Shi, Du and Chai, "Equilibrium-distribution-function based mesoscopic
 * finite-difference methods for PDEs", arXiv 2505.17057).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, __graft_entry__.smoke() and the
 * cpu_baseline / --impl reference legs of bench.py may load this library.
 * It shares no code, header, table or constant with the CUDA path.
 *
 * What it computes, per step and per node x (periodic box):
 *   Sec. II, Eq. (2-1)/(2-2):  phi(x) = sum_j sum_{k,q} a_kq f_j^eq(x + k c_j dt, t + q dt)
 *   NSE, Eq. (2-4): rho with {a_kq}, (rho u) = sum_j c_j sum_{k,q} abar_kq f_j^eq(...)
 *   two-level explicit: q = -1 only (Eq. (2-2-2)); three-level explicit:
 *   Eq. (3layerMMFD-1) with a_k on level t and ahat_k on level t - dt.
 * Three algebraically identical forms are provided:
 *   form 1: MesoFD, Eq. (2-1): f_j(x) first, then the moments Eq. (2-1-1);
 *   form 2: direct MMFD, Eq. (2-2) / (2-4) / (3layerMMFD-1);
 *   form 3: central MMFD, Eq. (2-2-1) / (2-4-1) with the even/odd split Eq. (2-5)
 *           and the central differences Eq. (CentralFD).
 * Multiple-parameter-set scheme (two_sets = 1), Eq. (2-2-1b): the zeroth-order term keeps
 * {a}, the second-difference (even) term takes its own set and the first-difference (odd)
 * term another; the momentum equation likewise (its analogue of Eq. (2-4-1)).
 *   form 3 evaluates Eq. (2-2-1b) (and its momentum analogue) directly;
 *   form 4: the TRT MesoFD scheme Eq. (2-1b): f_j = sum_k (abar_k f_j^eq,+ + ahat_k f_j^eq,-)
 *           at x + k c_j, then the moments -- equal to form 3 when {a} is the even set.
 * EDFs: general quadratic form Eq. (3-3)/(3-4) with direction-dependent
 * c_s,alpha^2 = d_0alpha c_alpha^2 (App. A); linear CDE Eq. (TforMMFD-0);
 * NCDE Eq. (NCDEfeq); incompressible NSE He-Luo form of Remark 4.
 * Lattices: rD2Q5I, rD2Q9, rD3Q7, rD3Q19 of App. A.
 * Source terms (scalar PDEs): the b_kq F_j terms of Eq. (2-1) / (3layer-1) with
 * F_j = g_j^eq(S, M_1F, 0), Eq. (SourceF); forms 1-3 (form 3 per Eq. (3layerMMFD-2)).
 * Independent checks on explicit populations: SRT LB with tau = 1 and TRT LB with
 * s+ + s- = 2 (the special cases (1) and (2) of Sec. III.C), collide then stream.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no SIMD
 * intrinsics; summation order fixed: levels t then t - dt, k ascending,
 * j ascending).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_D2Q5 = 0, OR_D2Q9 = 1, OR_D3Q7 = 2, OR_D3Q19 = 3 };
enum { OR_LCDE = 0, OR_NCDE = 1, OR_NSE = 2 };
enum { OR_FORM_MESOFD = 1, OR_FORM_MMFD = 2, OR_FORM_CENTRAL = 3, OR_FORM_MESOFD_TRT = 4 };
enum { OR_OK = 0, OR_EARG = -1 };

#define OR_QMAX 19

/* Problem statement in the paper's notation. */
typedef struct {
    int lattice;        /* OR_D2Q5 ... OR_D3Q19 */
    int pde;            /* OR_LCDE, OR_NCDE, OR_NSE */
    int levels;         /* 2 or 3 */
    int n[3];           /* nx, ny, nz (nz = 1 in 2D) */
    double c[3];        /* c_alpha = dx_alpha / dt (App. A) */
    double d0[3];       /* d_0alpha = c_salpha^2 / c_alpha^2 (App. A) */
    double a[3];        /* a_k on level t (two-level: a_{k,-1}), k = -1, 0, 1 at index k + 1 */
    double ahat[3];     /* a_k on level t - dt (three-level only) */
    double abar[3];     /* NSE momentum set on level t, Eq. (2-4) */
    double abarhat[3];  /* NSE momentum set on level t - dt */
    double u[3];        /* LCDE: B = phi u, Eq. (TforMMFD-0) */
    double Cmat[9];     /* LCDE: C = phi Cmat, Cmat = c_s^2 (beta D0 - I) + lambda u u (Eq. (TforMMFD-0)) */
    double flux[12];    /* NCDE: B_alpha(phi) = sum_{p=0}^{3} flux[4 alpha + p] phi^p */
    double m2[5];       /* NCDE: isotropic second moment M2(phi) = sum_{p=0}^{4} m2[p] phi^p */
    double rho0;        /* NSE: He-Luo reference density (Remark 4) */
    /* Eq. (2-2-1b), used when two_sets = 1 (index k + 1 as above):
     *   d2[l]: set of the second-difference term on f^eq,+ of the phi / rho moment,
     *   d1[l]: set of the first-difference term on f^eq,-,
     *   bar_d2[l]: momentum, second-difference term on f^eq,-,
     *   bar_d1[l]: momentum, first-difference term on f^eq,+,
     * for level l = 0 (t) and l = 1 (t - dt). */
    int two_sets;
    double d2[2][3], d1[2][3], bar_d2[2][3], bar_d1[2][3];
    /* Source terms of Eq. (2-1): dt sum_{k,q} b_kq F_j(x + k c_j dt, t + q dt), with the source
     * distribution F_j = g_j^eq(S, M_1F, 0) of Eq. (SourceF) (scalar PDEs only).
     *   src_mode OR_SRC_S:  M_1F = 0;
     *            OR_SRC_SU: M_1F = S u with the LCDE's u (the F_j of Example 1);
     *            OR_SRC_SM: S and M_1F given as fields (1 + dim per source level).
     * b[k + 1] on level t (two-level: the only level), bhat[k + 1] on level t - dt. */
    double dt;
    int src_mode;
    double b[3], bhat[3];
} or_problem;

enum { OR_SRC_NONE = 0, OR_SRC_S = 1, OR_SRC_SU = 2, OR_SRC_SM = 3 };

/* Lattice tables of App. A, with the scalings of Eq. (3-4) folded in once. */
typedef struct {
    int dim, b;
    int e[OR_QMAX][3];      /* integer directions, c_j = (e_j1 c_1, e_j2 c_2, e_j3 c_3) */
    double w[OR_QMAX];      /* omega_j */
    double cj[OR_QMAX][3];  /* c_j components */
    int opp[OR_QMAX];       /* jbar: c_jbar = -c_j */
    double c[3], cs2[3];
} or_lat;

static void set_e(or_lat* L, int j, int x, int y, int z) {
    L->e[j][0] = x; L->e[j][1] = y; L->e[j][2] = z;
}

/* App. A: velocity sets and weights as functions of d_0alpha.
 * rD3Q19: the x-z block of Eq. (D3Q19b) prints (1,0,1),(-1,0,-1),(-1,0,-1),(1,0,1);
 * read as the four distinct diagonals (1,0,1),(-1,0,1),(-1,0,-1),(1,0,-1)
 * (the printed set repeats two velocities and misses two). */
static int lat_init(or_lat* L, int lattice, const double d0[3], const double c[3]) {
    memset(L, 0, sizeof(*L));
    double d1 = d0[0], d2 = d0[1], d3 = d0[2];
    switch (lattice) {
    case OR_D2Q5:
        L->dim = 2; L->b = 5;
        set_e(L, 0, 0, 0, 0); set_e(L, 1, 1, 0, 0); set_e(L, 2, 0, 1, 0);
        set_e(L, 3, -1, 0, 0); set_e(L, 4, 0, -1, 0);
        L->w[0] = 1.0 - d1 - d2;
        L->w[1] = L->w[3] = d1 / 2.0;
        L->w[2] = L->w[4] = d2 / 2.0;
        break;
    case OR_D2Q9:
        L->dim = 2; L->b = 9;
        set_e(L, 0, 0, 0, 0); set_e(L, 1, 1, 0, 0); set_e(L, 2, 0, 1, 0);
        set_e(L, 3, -1, 0, 0); set_e(L, 4, 0, -1, 0); set_e(L, 5, 1, 1, 0);
        set_e(L, 6, -1, 1, 0); set_e(L, 7, -1, -1, 0); set_e(L, 8, 1, -1, 0);
        L->w[0] = (1.0 - d1) * (1.0 - d2);
        L->w[1] = L->w[3] = d1 * (1.0 - d2) / 2.0;
        L->w[2] = L->w[4] = (1.0 - d1) * d2 / 2.0;
        L->w[5] = L->w[6] = L->w[7] = L->w[8] = d1 * d2 / 4.0;
        break;
    case OR_D3Q7:
        L->dim = 3; L->b = 7;
        set_e(L, 0, 0, 0, 0); set_e(L, 1, 1, 0, 0); set_e(L, 2, 0, 1, 0); set_e(L, 3, 0, 0, 1);
        set_e(L, 4, -1, 0, 0); set_e(L, 5, 0, -1, 0); set_e(L, 6, 0, 0, -1);
        L->w[0] = 1.0 - d1 - d2 - d3;
        L->w[1] = L->w[4] = d1 / 2.0;
        L->w[2] = L->w[5] = d2 / 2.0;
        L->w[3] = L->w[6] = d3 / 2.0;
        break;
    case OR_D3Q19:
        L->dim = 3; L->b = 19;
        set_e(L, 0, 0, 0, 0); set_e(L, 1, 1, 0, 0); set_e(L, 2, 0, 1, 0); set_e(L, 3, 0, 0, 1);
        set_e(L, 4, -1, 0, 0); set_e(L, 5, 0, -1, 0); set_e(L, 6, 0, 0, -1);
        set_e(L, 7, 1, 1, 0); set_e(L, 8, -1, 1, 0); set_e(L, 9, -1, -1, 0); set_e(L, 10, 1, -1, 0);
        set_e(L, 11, 1, 0, 1); set_e(L, 12, -1, 0, 1); set_e(L, 13, -1, 0, -1); set_e(L, 14, 1, 0, -1);
        set_e(L, 15, 0, 1, 1); set_e(L, 16, 0, -1, 1); set_e(L, 17, 0, -1, -1); set_e(L, 18, 0, 1, -1);
        L->w[0] = 1.0 - d1 - d2 - d3 + d1 * d2 + d1 * d3 + d2 * d3;
        L->w[1] = L->w[4] = d1 * (1.0 - d2 - d3) / 2.0;
        L->w[2] = L->w[5] = d2 * (1.0 - d1 - d3) / 2.0;
        L->w[3] = L->w[6] = d3 * (1.0 - d1 - d2) / 2.0;
        for (int j = 7; j <= 10; ++j) L->w[j] = d1 * d2 / 4.0;
        for (int j = 11; j <= 14; ++j) L->w[j] = d1 * d3 / 4.0;
        for (int j = 15; j <= 18; ++j) L->w[j] = d2 * d3 / 4.0;
        break;
    default:
        return OR_EARG;
    }
    for (int a = 0; a < 3; ++a) {
        L->c[a] = (a < L->dim) ? c[a] : 0.0;
        L->cs2[a] = (a < L->dim) ? d0[a] * c[a] * c[a] : 0.0;
    }
    for (int j = 0; j < L->b; ++j) {
        for (int a = 0; a < 3; ++a) L->cj[j][a] = L->e[j][a] * L->c[a];
        L->opp[j] = -1;
        for (int i = 0; i < L->b; ++i)
            if (L->e[i][0] == -L->e[j][0] && L->e[i][1] == -L->e[j][1] && L->e[i][2] == -L->e[j][2])
                L->opp[j] = i;
        if (L->opp[j] < 0) return OR_EARG;
    }
    return OR_OK;
}

/* Eq. (3-3)/(3-4): g_j^eq(A, B, C) = omega_j (A + ctilde_j . B + Qtilde_j : C), with
 *   ctilde_ja = c_ja / cs_a^2,
 *   Qtilde_jaa = (c_ja^2 - cs_a^2) / (cs_a^2 (c_a^2 - cs_a^2)),
 *   Qtilde_jab = c_ja c_jb / (2 cs_a^2 cs_b^2)   (a != b),
 * where Q_j = c_j c_j - Delta^(2), Delta^(2) = diag(cs_a^2) (the printed diag{c_sa}
 * is read as diag{c_sa^2}, the only reading under which Eq. (3-5) holds).
 * The double contraction Qtilde : C runs over all ordered pairs (a, b). */
static double geq_j(const or_lat* L, int j, double A, const double B[3], const double C[9]) {
    double s = A;
    for (int a = 0; a < L->dim; ++a)
        s += L->cj[j][a] * B[a] / L->cs2[a];
    for (int a = 0; a < L->dim; ++a) {
        for (int b = 0; b < L->dim; ++b) {
            double q;
            if (a == b)
                q = (L->cj[j][a] * L->cj[j][a] - L->cs2[a]) /
                    (L->cs2[a] * (L->c[a] * L->c[a] - L->cs2[a]));
            else
                q = L->cj[j][a] * L->cj[j][b] / (2.0 * L->cs2[a] * L->cs2[b]);
            s += q * C[3 * a + b];
        }
    }
    return L->w[j] * s;
}

static int nfields(const or_problem* P, const or_lat* L) {
    return (P->pde == OR_NSE) ? 1 + L->dim : 1;
}

static double poly(const double* p, int deg, double x) {
    double r = 0.0;
    for (int i = deg; i >= 0; --i) r = r * x + p[i];
    return r;
}

/* Arguments (A, B, C) of the EDF for each PDE, from the stored fields at one node. */
static void edf_args(const or_problem* P, const or_lat* L, const double* f,
                     double* A, double B[3], double C[9]) {
    memset(B, 0, 3 * sizeof(double));
    memset(C, 0, 9 * sizeof(double));
    if (P->pde == OR_LCDE) {
        /* Eq. (TforMMFD-0): f_j^eq = phi ubar_j = g_j^eq(phi, phi u, phi C). */
        double phi = f[0];
        *A = phi;
        for (int a = 0; a < L->dim; ++a) B[a] = phi * P->u[a];
        for (int k = 0; k < 9; ++k) C[k] = phi * P->Cmat[k];
    } else if (P->pde == OR_NCDE) {
        /* Eq. (NCDEfeq): f^eq = g^eq(phi, B(phi), beta cs^2 D + C - cs^2 phi I), with the
         * second-moment target beta cs^2 D + C = M2(phi) I (isotropic, no correction). */
        double phi = f[0];
        *A = phi;
        for (int a = 0; a < L->dim; ++a) B[a] = poly(&P->flux[4 * a], 3, phi);
        double m2 = poly(P->m2, 4, phi);
        for (int a = 0; a < L->dim; ++a) C[3 * a + a] = m2 - L->cs2[a] * phi;
    } else {
        /* Remark 4 (He-Luo): f^eq = g^eq(rho, rho0 u, rho0 u u); fields are (rho, u[dim]). */
        *A = f[0];
        for (int a = 0; a < L->dim; ++a) B[a] = P->rho0 * f[1 + a];
        for (int a = 0; a < L->dim; ++a)
            for (int b = 0; b < L->dim; ++b) C[3 * a + b] = P->rho0 * f[1 + a] * f[1 + b];
    }
}

/* f_j^eq at node index idx of a level (SoA fields, each N = nx ny nz values). */
static double feq_at(const or_problem* P, const or_lat* L, const double* lev, long long N,
                     long long idx, int j) {
    double f[4], A, B[3], C[9];
    int nf = nfields(P, L);
    for (int i = 0; i < nf; ++i) f[i] = lev[i * N + idx];
    edf_args(P, L, f, &A, B, C);
    return geq_j(L, j, A, B, C);
}

static long long wrap(long long i, long long n) {
    long long r = i % n;
    return r < 0 ? r + n : r;
}

/* Index of node (x + k e_j) with periodic wrap in every direction. */
static long long shifted(const or_problem* P, const or_lat* L, long long idx, int j, int k) {
    long long nx = P->n[0], ny = P->n[1], nz = P->n[2];
    long long x = idx % nx, y = (idx / nx) % ny, z = idx / (nx * ny);
    x = wrap(x + (long long)k * L->e[j][0], nx);
    y = wrap(y + (long long)k * L->e[j][1], ny);
    z = wrap(z + (long long)k * L->e[j][2], nz);
    return (z * ny + y) * nx + x;
}

/* Number of source fields per level. */
static int nsrc(const or_problem* P, const or_lat* L) {
    return P->src_mode == OR_SRC_SM ? 1 + L->dim : (P->src_mode ? 1 : 0);
}

/* F_j = g_j^eq(S, M_1F, 0) (Eq. (SourceF)) at node idx of one source level (SoA, N per field). */
static double F_at(const or_problem* P, const or_lat* L, const double* src, long long N, long long idx, int j) {
    double S = src[idx], M[3] = {0, 0, 0}, C[9] = {0};
    for (int d = 0; d < L->dim; ++d)
        M[d] = P->src_mode == OR_SRC_SU ? S * P->u[d] : (P->src_mode == OR_SRC_SM ? src[(1 + d) * N + idx] : 0.0);
    return geq_j(L, j, S, M, C);
}

static const double* bcoef(const or_problem* P, int l) { return l == 0 ? P->b : P->bhat; }

/* Coefficients of level index l (0: t, 1: t - dt) for the scalar / rho moment and for the
 * momentum moment. */
static const double* coef(const or_problem* P, int l) { return l == 0 ? P->a : P->ahat; }
static const double* coefbar(const or_problem* P, int l) { return l == 0 ? P->abar : P->abarhat; }

/* One node, form 2 (direct MMFD): Eq. (2-2) / (2-4) / (3layerMMFD-1). */
static void node_mmfd(const or_problem* P, const or_lat* L, const double* levs[2], const double* srcs[2],
                      long long N, long long idx, double* out) {
    int nf = nfields(P, L);
    double acc[4] = {0, 0, 0, 0};
    for (int l = 0; l < P->levels - 1; ++l) {
        const double* a = coef(P, l);
        const double* ab = coefbar(P, l);
        const double* bb = bcoef(P, l);
        for (int k = -1; k <= 1; ++k) {
            for (int j = 0; j < L->b; ++j) {
                long long ik = shifted(P, L, idx, j, k);
                double fe = feq_at(P, L, levs[l], N, ik, j);
                acc[0] += a[k + 1] * fe;
                if (P->pde == OR_NSE)
                    for (int d = 0; d < L->dim; ++d) acc[1 + d] += ab[k + 1] * L->cj[j][d] * fe;
                if (P->src_mode) acc[0] += P->dt * bb[k + 1] * F_at(P, L, srcs[l], N, ik, j);
            }
        }
    }
    out[0] = acc[0];
    for (int d = 1; d < nf; ++d) out[d] = acc[d] / P->rho0;
}

/* One node, form 1 (MesoFD): Eq. (2-1) gives f_j(x) per direction, then Eq. (2-1-1)
 * (and, for the NSE, the double-distribution moments Eq. (2-4)). */
static void node_mesofd(const or_problem* P, const or_lat* L, const double* levs[2], const double* srcs[2],
                        long long N, long long idx, double* out) {
    int nf = nfields(P, L);
    double fj[OR_QMAX], fbarj[OR_QMAX];
    for (int j = 0; j < L->b; ++j) {
        double s = 0.0, sb = 0.0;
        for (int l = 0; l < P->levels - 1; ++l) {
            const double* a = coef(P, l);
            const double* ab = coefbar(P, l);
            const double* bb = bcoef(P, l);
            for (int k = -1; k <= 1; ++k) {
                long long ik = shifted(P, L, idx, j, k);
                double fe = feq_at(P, L, levs[l], N, ik, j);
                s += a[k + 1] * fe;
                sb += ab[k + 1] * fe;
                if (P->src_mode) s += P->dt * bb[k + 1] * F_at(P, L, srcs[l], N, ik, j);
            }
        }
        fj[j] = s;
        fbarj[j] = sb;
    }
    double phi = 0.0, m[3] = {0, 0, 0};
    for (int j = 0; j < L->b; ++j) {
        phi += fj[j];
        for (int d = 0; d < L->dim; ++d) m[d] += L->cj[j][d] * fbarj[j];
    }
    out[0] = phi;
    for (int d = 1; d < nf; ++d) out[d] = m[d - 1] / P->rho0;
}

/* Even and odd parts, Eq. (2-5): g_j^+ = (g_j + g_jbar)/2, g_j^- = (g_j - g_jbar)/2. */
static double feq_even(const or_problem* P, const or_lat* L, const double* lev, long long N,
                       long long idx, int j) {
    return 0.5 * (feq_at(P, L, lev, N, idx, j) + feq_at(P, L, lev, N, idx, L->opp[j]));
}
static double feq_odd(const or_problem* P, const or_lat* L, const double* lev, long long N,
                      long long idx, int j) {
    return 0.5 * (feq_at(P, L, lev, N, idx, j) - feq_at(P, L, lev, N, idx, L->opp[j]));
}

/* One node, form 3 (central MMFD), Eq. (2-2-1) and Eq. (2-4-1), m_q = 1:
 *   phi = sum_q [ (sum_k a_kq) phi(x) + 1/2 sum_j ( a+_1q D2_j f^eq,+ + a-_1q D1_j f^eq,- ) ]
 *   (rho u) = sum_q [ (sum_k abar_kq) (rho u)(x)
 *                     + 1/2 sum_j c_j ( abar+_1q D2_j f^eq,- + abar-_1q D1_j f^eq,+ ) ]
 * with a+_1 = a_1 + a_{-1}, a-_1 = a_1 - a_{-1} (Eq. (2-1-FD1-0)) and the central
 * differences of Eq. (CentralFD).  phi(x) and (rho u)(x) are the zeroth and first
 * moments of f^eq at x (Eq. (3-5)). */
static void node_central(const or_problem* P, const or_lat* L, const double* levs[2], const double* srcs[2],
                         long long N, long long idx, double* out) {
    int nf = nfields(P, L);
    double acc[4] = {0, 0, 0, 0};
    for (int l = 0; l < P->levels - 1; ++l) {
        const double* lev = levs[l];
        const double* a = coef(P, l);
        const double* ab = coefbar(P, l);
        /* Eq. (2-2-1b): with two_sets the difference terms take their own sets */
        const double* e2 = P->two_sets ? P->d2[l] : a;
        const double* o1 = P->two_sets ? P->d1[l] : a;
        const double* be2 = P->two_sets ? P->bar_d2[l] : ab;
        const double* bo1 = P->two_sets ? P->bar_d1[l] : ab;
        double A0 = a[0] + a[1] + a[2];
        double Ab0 = ab[0] + ab[1] + ab[2];
        double ap = e2[2] + e2[0], am = o1[2] - o1[0];
        double abp = be2[2] + be2[0], abm = bo1[2] - bo1[0];
        double M0 = 0.0, M1[3] = {0, 0, 0};
        for (int j = 0; j < L->b; ++j) {
            double fe = feq_at(P, L, lev, N, idx, j);
            M0 += fe;
            for (int d = 0; d < L->dim; ++d) M1[d] += L->cj[j][d] * fe;
        }
        acc[0] += A0 * M0;
        for (int d = 0; d < L->dim; ++d) acc[1 + d] += Ab0 * M1[d];
        for (int j = 0; j < L->b; ++j) {
            long long ip = shifted(P, L, idx, j, 1), im = shifted(P, L, idx, j, -1);
            double ep = feq_even(P, L, lev, N, ip, j), e0 = feq_even(P, L, lev, N, idx, j),
                   em = feq_even(P, L, lev, N, im, j);
            double op = feq_odd(P, L, lev, N, ip, j), o0 = feq_odd(P, L, lev, N, idx, j),
                   om = feq_odd(P, L, lev, N, im, j);
            double d2e = ep - 2.0 * e0 + em, d1o = op - om;
            double d2o = op - 2.0 * o0 + om, d1e = ep - em;
            acc[0] += 0.5 * (ap * d2e + am * d1o);
            if (P->pde == OR_NSE)
                for (int d = 0; d < L->dim; ++d)
                    acc[1 + d] += 0.5 * L->cj[j][d] * (abp * d2o + abm * d1e);
        }
        if (P->src_mode) {
            /* Eq. (3layerMMFD-2): dt [ B_0 S(x) + 1/2 sum_j ( b+_1 D2_j F_j^+ + b-_1 D1_j F_j^- ) ],
             * B_0 = b_0 + b_1 + b_{-1}, b+-_1 = b_1 +- b_{-1}, S(x) = sum_j F_j(x) */
            const double* bb = bcoef(P, l);
            const double* src = srcs[l];
            double B0 = bb[0] + bb[1] + bb[2], bp = bb[2] + bb[0], bm = bb[2] - bb[0];
            double S0 = 0.0, t = 0.0;
            for (int j = 0; j < L->b; ++j) S0 += F_at(P, L, src, N, idx, j);
            for (int j = 0; j < L->b; ++j) {
                const int jb = L->opp[j];
                long long at[3] = {shifted(P, L, idx, j, 1), idx, shifted(P, L, idx, j, -1)};
                double Fp[3], Fm[3];   /* even / odd parts at x + c_j, x, x - c_j */
                for (int i = 0; i < 3; ++i) {
                    double fj = F_at(P, L, src, N, at[i], j), fjb = F_at(P, L, src, N, at[i], jb);
                    Fp[i] = 0.5 * (fj + fjb);
                    Fm[i] = 0.5 * (fj - fjb);
                }
                t += 0.5 * (bp * (Fp[0] - 2.0 * Fp[1] + Fp[2]) + bm * (Fm[0] - Fm[2]));
            }
            acc[0] += P->dt * (B0 * S0 + t);
        }
    }
    out[0] = acc[0];
    for (int d = 1; d < nf; ++d) out[d] = acc[d] / P->rho0;
}

/* One node, form 4: the TRT version of the MesoFD scheme, Eq. (2-1b), m_q = 1:
 *   f_j(x) = sum_q sum_k [ abar_kq f_j^eq,+ + ahat_kq f_j^eq,- ](x + k c_j, t + q dt)
 * followed by phi = sum_j f_j.  The even set is d2 and the odd set d1; for the NSE the
 * momentum distribution takes bar_d1 on the even parts and bar_d2 on the odd parts and
 * (rho u) = sum_j c_j fbar_j.  Expanding the shifts with Eq. (2-5) turns this into
 * Eq. (2-2-1b) with the zeroth-order set equal to the even set (momentum: to bar_d2). */
static void node_mesofd_trt(const or_problem* P, const or_lat* L, const double* levs[2], const double* srcs[2],
                            long long N, long long idx, double* out) {
    (void)srcs;  /* no source terms in this form */
    int nf = nfields(P, L);
    double fj[OR_QMAX], fbarj[OR_QMAX];
    for (int j = 0; j < L->b; ++j) {
        double s = 0.0, sb = 0.0;
        for (int l = 0; l < P->levels - 1; ++l) {
            for (int k = -1; k <= 1; ++k) {
                long long ik = shifted(P, L, idx, j, k);
                double fe = feq_even(P, L, levs[l], N, ik, j), fo = feq_odd(P, L, levs[l], N, ik, j);
                s += P->d2[l][k + 1] * fe + P->d1[l][k + 1] * fo;
                sb += P->bar_d1[l][k + 1] * fe + P->bar_d2[l][k + 1] * fo;
            }
        }
        fj[j] = s;
        fbarj[j] = sb;
    }
    double phi = 0.0, m[3] = {0, 0, 0};
    for (int j = 0; j < L->b; ++j) {
        phi += fj[j];
        for (int d = 0; d < L->dim; ++d) m[d] += L->cj[j][d] * fbarj[j];
    }
    out[0] = phi;
    for (int d = 1; d < nf; ++d) out[d] = m[d - 1] / P->rho0;
}

typedef void (*node_fn)(const or_problem*, const or_lat*, const double* [2], const double* [2], long long,
                        long long, double*);

static node_fn pick(int form) {
    switch (form) {
    case OR_FORM_MESOFD: return node_mesofd;
    case OR_FORM_MMFD: return node_mmfd;
    case OR_FORM_CENTRAL: return node_central;
    case OR_FORM_MESOFD_TRT: return node_mesofd_trt;
    default: return 0;
    }
}

static int check(const or_problem* P, or_lat* L) {
    if (!P) return OR_EARG;
    if (P->levels != 2 && P->levels != 3) return OR_EARG;
    if (P->pde < OR_LCDE || P->pde > OR_NSE) return OR_EARG;
    if (lat_init(L, P->lattice, P->d0, P->c) != OR_OK) return OR_EARG;
    for (int a = 0; a < 3; ++a) if (P->n[a] < 1) return OR_EARG;
    if (L->dim == 2 && P->n[2] != 1) return OR_EARG;
    if (P->pde == OR_NSE && P->rho0 == 0.0) return OR_EARG;
    if (P->src_mode < OR_SRC_NONE || P->src_mode > OR_SRC_SM) return OR_EARG;
    if (P->src_mode && (P->pde == OR_NSE || !(P->dt > 0.0))) return OR_EARG;
    if (P->src_mode == OR_SRC_SU && P->pde != OR_LCDE) return OR_EARG;
    return OR_OK;
}

/* Sources needed by a step: level t always, level t - dt for three-level problems. */
static int check_src(const or_problem* P, int form, const double* src_n, const double* src_nm1) {
    if (!P->src_mode) return OR_OK;
    if (form == OR_FORM_MESOFD_TRT || !src_n) return OR_EARG;
    if (P->levels == 3 && !src_nm1) return OR_EARG;
    return OR_OK;
}

/* ---------------------------------------------------------------- exported API */

int or_lattice(int lattice, const double d0[3], const double c[3], int* dim, int* b, int* e,
               double* w, double* cs2) {
    or_lat L;
    if (lat_init(&L, lattice, d0, c) != OR_OK) return OR_EARG;
    *dim = L.dim;
    *b = L.b;
    for (int j = 0; j < L.b; ++j) {
        for (int a = 0; a < 3; ++a) e[3 * j + a] = L.e[j][a];
        w[j] = L.w[j];
    }
    for (int a = 0; a < 3; ++a) cs2[a] = L.cs2[a];
    return OR_OK;
}

/* All b values of g^eq(A, B, C), Eq. (3-3). */
int or_geq(int lattice, const double d0[3], const double c[3], double A, const double B[3],
           const double C[9], double* g) {
    or_lat L;
    if (lat_init(&L, lattice, d0, c) != OR_OK) return OR_EARG;
    for (int j = 0; j < L.b; ++j) g[j] = geq_j(&L, j, A, B, C);
    return OR_OK;
}

/* All b values of the problem's f^eq at a single node's stored fields. */
int or_feq(const or_problem* P, const double* fields, double* feq) {
    or_lat L;
    if (check(P, &L) != OR_OK) return OR_EARG;
    double A, B[3], C[9];
    edf_args(P, &L, fields, &A, B, C);
    for (int j = 0; j < L.b; ++j) feq[j] = geq_j(&L, j, A, B, C);
    return OR_OK;
}

int or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* One step with source terms: out (nf x N, SoA) from lev_n (level t) and lev_nm1 (level t - dt;
 * ignored when levels == 2); src_n / src_nm1 the source fields (nsrc x N) at the same two
 * times (NULL when src_mode is 0; src_nm1 ignored when levels == 2). */
int or_step_src(const or_problem* P, int form, const double* lev_n, const double* lev_nm1,
                const double* src_n, const double* src_nm1, double* out) {
    or_lat L;
    if (check(P, &L) != OR_OK) return OR_EARG;
    node_fn fn = pick(form);
    if (!fn) return OR_EARG;
    if (P->levels == 3 && !lev_nm1) return OR_EARG;
    if (check_src(P, form, src_n, src_nm1) != OR_OK) return OR_EARG;
    const long long N = (long long)P->n[0] * P->n[1] * P->n[2];
    const int nf = nfields(P, &L);
    const double* levs[2] = {lev_n, lev_nm1};
    const double* srcs[2] = {src_n, src_nm1};
#pragma omp parallel for schedule(static)
    for (long long idx = 0; idx < N; ++idx) {
        double o[4];
        fn(P, &L, levs, srcs, N, idx, o);
        for (int i = 0; i < nf; ++i) out[i * N + idx] = o[i];
    }
    return OR_OK;
}

int or_step(const or_problem* P, int form, const double* lev_n, const double* lev_nm1, double* out) {
    return or_step_src(P, form, lev_n, lev_nm1, 0, 0, out);
}

/* The step's outputs at a list of node indices only (out is count x nf, node-major). */
int or_step_nodes_src(const or_problem* P, int form, const double* lev_n, const double* lev_nm1,
                      const double* src_n, const double* src_nm1, const long long* nodes, long long count,
                      double* out) {
    or_lat L;
    if (check(P, &L) != OR_OK) return OR_EARG;
    node_fn fn = pick(form);
    if (!fn) return OR_EARG;
    if (check_src(P, form, src_n, src_nm1) != OR_OK) return OR_EARG;
    const long long N = (long long)P->n[0] * P->n[1] * P->n[2];
    const int nf = nfields(P, &L);
    const double* levs[2] = {lev_n, lev_nm1};
    const double* srcs[2] = {src_n, src_nm1};
    for (long long i = 0; i < count; ++i) {
        if (nodes[i] < 0 || nodes[i] >= N) return OR_EARG;
    }
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < count; ++i) {
        double o[4];
        fn(P, &L, levs, srcs, N, nodes[i], o);
        for (int f = 0; f < nf; ++f) out[i * nf + f] = o[f];
    }
    return OR_OK;
}

int or_step_nodes(const or_problem* P, int form, const double* lev_n, const double* lev_nm1,
                  const long long* nodes, long long count, double* out) {
    return or_step_nodes_src(P, form, lev_n, lev_nm1, 0, 0, nodes, count, out);
}

/* nsteps steps in place: on return lev_n holds level t + nsteps dt and lev_nm1 (three-level)
 * the level before it. */
int or_run(const or_problem* P, int form, long long nsteps, double* lev_n, double* lev_nm1) {
    or_lat L;
    if (check(P, &L) != OR_OK) return OR_EARG;
    if (P->src_mode) return OR_EARG;  /* sources: step by step with or_step_src */
    const long long N = (long long)P->n[0] * P->n[1] * P->n[2];
    const int nf = nfields(P, &L);
    double* tmp = (double*)malloc(sizeof(double) * (size_t)(nf * N));
    if (!tmp) return OR_EARG;
    for (long long s = 0; s < nsteps; ++s) {
        int rc = or_step(P, form, lev_n, lev_nm1, tmp);
        if (rc != OR_OK) { free(tmp); return rc; }
        if (P->levels == 3) memcpy(lev_nm1, lev_n, sizeof(double) * (size_t)(nf * N));
        memcpy(lev_n, tmp, sizeof(double) * (size_t)(nf * N));
    }
    free(tmp);
    return OR_OK;
}

/* Independent lattice-Boltzmann check (Sec. III.C, special case (1)): LBGK with tau = 1,
 * written as collide-then-stream on explicit distribution arrays:
 *   f_j(x + c_j dt, t + dt) = f_j(x, t) - (f_j - f_j^eq)/tau |_{tau = 1} = f_j^eq(x, t),
 * with f^eq built from the moments of f (phi = sum f; NSE: rho = sum f, rho0 u = sum c f).
 * Two-level problems only; the a's of P are not used.  Fields in place. */
int or_lbgk_tau1_run(const or_problem* P, long long nsteps, double* fields) {
    or_lat L;
    if (check(P, &L) != OR_OK) return OR_EARG;
    if (P->src_mode) return OR_EARG;
    const long long N = (long long)P->n[0] * P->n[1] * P->n[2];
    const int nf = nfields(P, &L);
    double* f = (double*)malloc(sizeof(double) * (size_t)(L.b * N));
    double* g = (double*)malloc(sizeof(double) * (size_t)(L.b * N));
    if (!f || !g) { free(f); free(g); return OR_EARG; }
    /* initial populations at equilibrium */
    for (long long x = 0; x < N; ++x)
        for (int j = 0; j < L.b; ++j) f[j * N + x] = feq_at(P, &L, fields, N, x, j);
    for (long long s = 0; s < nsteps; ++s) {
        /* collide (tau = 1): post-collision populations are the equilibria of the moments of f */
        for (long long x = 0; x < N; ++x) {
            double m0 = 0.0, m1[3] = {0, 0, 0};
            for (int j = 0; j < L.b; ++j) {
                m0 += f[j * N + x];
                for (int d = 0; d < L.dim; ++d) m1[d] += L.cj[j][d] * f[j * N + x];
            }
            double loc[4];
            loc[0] = m0;
            for (int d = 0; d < L.dim; ++d) loc[1 + d] = m1[d] / P->rho0;
            double A, B[3], C[9];
            edf_args(P, &L, loc, &A, B, C);
            for (int j = 0; j < L.b; ++j) g[j * N + x] = geq_j(&L, j, A, B, C);
        }
        /* stream: population j moves from x to x + e_j */
        for (long long x = 0; x < N; ++x)
            for (int j = 0; j < L.b; ++j) f[j * N + shifted(P, &L, x, j, 1)] = g[j * N + x];
    }
    for (long long x = 0; x < N; ++x) {
        double m0 = 0.0, m1[3] = {0, 0, 0};
        for (int j = 0; j < L.b; ++j) {
            m0 += f[j * N + x];
            for (int d = 0; d < L.dim; ++d) m1[d] += L.cj[j][d] * f[j * N + x];
        }
        fields[x] = m0;
        for (int d = 1; d < nf; ++d) fields[d * N + x] = m1[d - 1] / P->rho0;
    }
    free(f);
    free(g);
    return OR_OK;
}

/* Independent two-relaxation-time LB code (Sec. III.C, special case (2), TRT with
 * s+ + s- = 2), collide-then-stream on explicit populations:
 *   f_j* = f_j - s+ (f_j^+ - f_j^eq,+) - s- (f_j^- - f_j^eq,-),   f_j(x + c_j, t + dt) = f_j*(x, t),
 * with the even / odd parts of Eq. (2-5) taken over j and its opposite jbar, s+ = 2 - s-, and
 * f^eq built from the moments of f.  Starts from equilibrium populations of `fields`; the a's
 * of P are not used.  Fields (moments) in place after nsteps. */
int or_trt_run(const or_problem* P, double s_minus, long long nsteps, double* fields) {
    or_lat L;
    if (check(P, &L) != OR_OK) return OR_EARG;
    if (P->src_mode) return OR_EARG;
    const double s_plus = 2.0 - s_minus;
    const long long N = (long long)P->n[0] * P->n[1] * P->n[2];
    const int nf = nfields(P, &L);
    double* f = (double*)malloc(sizeof(double) * (size_t)(L.b * N));
    double* g = (double*)malloc(sizeof(double) * (size_t)(L.b * N));
    if (!f || !g) { free(f); free(g); return OR_EARG; }
    for (long long x = 0; x < N; ++x)
        for (int j = 0; j < L.b; ++j) f[j * N + x] = feq_at(P, &L, fields, N, x, j);
    for (long long s = 0; s < nsteps; ++s) {
        for (long long x = 0; x < N; ++x) {
            double m0 = 0.0, m1[3] = {0, 0, 0};
            for (int j = 0; j < L.b; ++j) {
                m0 += f[j * N + x];
                for (int d = 0; d < L.dim; ++d) m1[d] += L.cj[j][d] * f[j * N + x];
            }
            double loc[4];
            loc[0] = m0;
            for (int d = 0; d < L.dim; ++d) loc[1 + d] = m1[d] / P->rho0;
            double A, B[3], C[9], eq[OR_QMAX];
            edf_args(P, &L, loc, &A, B, C);
            for (int j = 0; j < L.b; ++j) eq[j] = geq_j(&L, j, A, B, C);
            for (int j = 0; j < L.b; ++j) {
                const int jb = L.opp[j];
                const double fp = 0.5 * (f[j * N + x] + f[jb * N + x]), fm = 0.5 * (f[j * N + x] - f[jb * N + x]);
                const double ep = 0.5 * (eq[j] + eq[jb]), em = 0.5 * (eq[j] - eq[jb]);
                g[j * N + x] = f[j * N + x] - s_plus * (fp - ep) - s_minus * (fm - em);
            }
        }
        for (long long x = 0; x < N; ++x)
            for (int j = 0; j < L.b; ++j) f[j * N + shifted(P, &L, x, j, 1)] = g[j * N + x];
    }
    for (long long x = 0; x < N; ++x) {
        double m0 = 0.0, m1[3] = {0, 0, 0};
        for (int j = 0; j < L.b; ++j) {
            m0 += f[j * N + x];
            for (int d = 0; d < L.dim; ++d) m1[d] += L.cj[j][d] * f[j * N + x];
        }
        fields[x] = m0;
        for (int d = 1; d < nf; ++d) fields[d * N + x] = m1[d - 1] / P->rho0;
    }
    free(f);
    free(g);
    return OR_OK;
}
