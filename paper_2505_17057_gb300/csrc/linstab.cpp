// linstab.cpp -- frozen-coefficient stability of the nonlinear schemes (NCDE, He-Luo NSE).
//
// The paper's stability analysis (Sec. III.D, Theorems 1-3) covers the linear CDE, whose
// amplification symbol is Eq. (TforMMFD-3).  For the NCDE and the NSE the update is linearised
// about a uniform state: the EDF arguments (A, B, C) are replaced by their first-order variation
// (B'(phi) dphi, M2'(phi) dphi for the NCDE; rho0 (u dU + dU u) for the He-Luo C of the NSE), and
// a Fourier mode exp(i theta . x) of the perturbation is multiplied per level by a matrix M_l
// (scalar for the NCDE, (1 + dim) x (1 + dim) for the NSE) built from the same folded
// coefficients the kernels use.  Two-level: the amplification factors are the eigenvalues of
// M_0; three-level: those of the companion matrix [[M_0, M_1], [I, 0]] (Eq. (3-level) in matrix
// form).  The largest modulus over the grid's wave numbers is returned.
#include <cmath>
#include <complex>
#include <vector>

#include "params.h"

namespace mmfd {

namespace {

using cplx = std::complex<double>;
constexpr int kMaxN = 8;

// Upper Hessenberg form by Householder reflections (similarity transform).
void hessenberg(int n, cplx A[kMaxN][kMaxN]) {
    for (int k = 0; k + 2 < n; ++k) {
        double alpha = 0.0;
        for (int i = k + 1; i < n; ++i) alpha += std::norm(A[i][k]);
        alpha = std::sqrt(alpha);
        if (alpha == 0.0) continue;
        const cplx x0 = A[k + 1][k];
        const cplx ph = std::abs(x0) > 0.0 ? x0 / std::abs(x0) : cplx(1.0, 0.0);
        cplx v[kMaxN] = {};
        for (int i = k + 1; i < n; ++i) v[i] = A[i][k];
        v[k + 1] += ph * alpha;
        double vn = 0.0;
        for (int i = k + 1; i < n; ++i) vn += std::norm(v[i]);
        if (vn == 0.0) continue;
        for (int j = 0; j < n; ++j) {   // A <- H A, H = I - 2 v v^H / |v|^2
            cplx s = 0.0;
            for (int i = k + 1; i < n; ++i) s += std::conj(v[i]) * A[i][j];
            s *= 2.0 / vn;
            for (int i = k + 1; i < n; ++i) A[i][j] -= v[i] * s;
        }
        for (int i = 0; i < n; ++i) {   // A <- A H
            cplx s = 0.0;
            for (int j = k + 1; j < n; ++j) s += A[i][j] * v[j];
            s *= 2.0 / vn;
            for (int j = k + 1; j < n; ++j) A[i][j] -= s * std::conj(v[j]);
        }
    }
}

// Largest eigenvalue modulus of a small complex matrix: Hessenberg reduction, then single-shift
// QR steps with Givens rotations (Wilkinson shift, an exceptional shift every tenth step) and
// deflation of negligible subdiagonal entries.
double spectral_radius(int n, cplx A[kMaxN][kMaxN]) {
    if (n == 1) return std::abs(A[0][0]);
    double anorm = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) anorm = std::max(anorm, std::abs(A[i][j]));
    if (anorm == 0.0) return 0.0;
    hessenberg(n, A);
    double rho = 0.0;
    int hi = n - 1, iter = 0, total = 0;
    while (hi >= 0) {
        if (hi == 0) {
            rho = std::max(rho, std::abs(A[0][0]));
            break;
        }
        int l = hi;
        while (l > 0) {
            const double s = std::abs(A[l - 1][l - 1]) + std::abs(A[l][l]);
            if (std::abs(A[l][l - 1]) <= 1e-15 * s || std::abs(A[l][l - 1]) <= 1e-17 * anorm) {
                A[l][l - 1] = 0.0;
                break;
            }
            --l;
        }
        if (l == hi) {
            rho = std::max(rho, std::abs(A[hi][hi]));
            --hi;
            iter = 0;
            continue;
        }
        if (++total > 100 * n) {
            // no convergence: bound the block's eigenvalues by its Frobenius norm
            double f = 0.0;
            for (int i = l; i <= hi; ++i)
                for (int j = l; j <= hi; ++j) f += std::norm(A[i][j]);
            return std::max(rho, std::sqrt(f));
        }
        const cplx a = A[hi - 1][hi - 1], b = A[hi - 1][hi], c = A[hi][hi - 1], d = A[hi][hi];
        cplx mu;
        if (++iter % 10 == 0) {
            mu = d + 0.75 * std::abs(c);
        } else {
            const cplx tr = a + d, det = a * d - b * c;
            const cplx disc = std::sqrt(0.25 * tr * tr - det);
            const cplx m1 = 0.5 * tr + disc, m2 = 0.5 * tr - disc;
            mu = std::abs(m1 - d) < std::abs(m2 - d) ? m1 : m2;
        }
        for (int k = l; k <= hi; ++k) A[k][k] -= mu;
        double gc[kMaxN];
        cplx gs[kMaxN];
        for (int k = l; k < hi; ++k) {
            const cplx x = A[k][k], y = A[k + 1][k];
            const double r = std::sqrt(std::norm(x) + std::norm(y));
            double cc = 1.0;
            cplx ss = 0.0;
            if (r > 0.0) {
                if (std::abs(x) > 0.0) {
                    cc = std::abs(x) / r;
                    ss = (x / std::abs(x)) * std::conj(y) / r;
                } else {
                    cc = 0.0;
                    ss = std::conj(y) / std::abs(y);
                }
            }
            gc[k] = cc;
            gs[k] = ss;
            for (int j = k; j <= hi; ++j) {
                const cplx u = A[k][j], w = A[k + 1][j];
                A[k][j] = cc * u + ss * w;
                A[k + 1][j] = -std::conj(ss) * u + cc * w;
            }
        }
        for (int k = l; k < hi; ++k) {
            const int top = std::min(k + 2, hi);
            for (int i = l; i <= top; ++i) {
                const cplx u = A[i][k], w = A[i][k + 1];
                A[i][k] = gc[k] * u + std::conj(gs[k]) * w;
                A[i][k + 1] = -gs[k] * u + gc[k] * w;
            }
        }
        for (int k = l; k <= hi; ++k) A[k][k] += mu;
    }
    return rho;
}

// Phasors exp(i 2 pi m / n) of the wave numbers taken on one axis: every one up to `all` nodes,
// else the `low` smallest of either sign and a uniform sweep of `sweep`; the last axis takes
// only [0, pi] (real coefficients: the symbol at -theta is the conjugate of that at theta).
std::vector<cplx> axis_phasors(long long n, bool last, long long all, int low, int sweep) {
    std::vector<long long> ms;
    if (n <= all) {
        for (long long m = 0; m < n; ++m) ms.push_back(m);
    } else {
        for (long long m = 0; m <= low; ++m) {
            ms.push_back(m);
            if (m > 0) ms.push_back(n - m);
        }
        for (int m = 1; m < sweep; ++m) ms.push_back((long long)((double)m * n / sweep));
        ms.push_back(n / 2);
    }
    std::vector<cplx> out;
    for (long long m : ms) {
        if (last && 2 * m > n) continue;
        out.push_back(std::polar(1.0, 6.283185307179586 * (double)m / (double)n));
    }
    return out;
}

int cross_index(int a, int b) { return (a == 0 && b == 1) || (a == 1 && b == 0) ? 3 : (a + b == 2) ? 4 : 5; }

}  // namespace

double linear_amplification(const Resolved& r, const double* state, bool dense) {
    const int dim = r.dim, NP = lat_npair(r.lat), nf = r.nf;
    const int nl = r.levels == 3 ? 2 : 1;
    const Coef<double>& c = r.cd;
    // d (E_p, O_p, f_0) / d (fields) at the state, per pair p and field j
    double dE[kMaxPair][4] = {}, dO[kMaxPair][4] = {}, df0[4] = {};
    if (r.pde == PDE_NCDE) {
        const double phi = state[0];
        const double dm2 = c.m2[1] + phi * (2.0 * c.m2[2] + phi * (3.0 * c.m2[3] + phi * 4.0 * c.m2[4]));
        double dB[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < dim; ++a) dB[a] = c.flux[a][1] + phi * (2.0 * c.flux[a][2] + phi * 3.0 * c.flux[a][3]);
        for (int p = 0; p < NP; ++p) {
            dE[p][0] = c.ePhi[p] + c.eM2[p] * dm2;
            for (int a = 0; a < dim; ++a) dO[p][0] += c.oB[p][a] * dB[a];
        }
        df0[0] = c.rPhi + c.rM2 * dm2;
    } else if (r.pde == PDE_NSE) {
        const double* u = state + 1;
        for (int p = 0; p < NP; ++p) {
            dE[p][0] = c.eA[p];
            for (int a = 0; a < dim; ++a) {
                double v = 2.0 * c.eC[p][a] * u[a];
                for (int b = 0; b < dim; ++b)
                    if (b != a) v += c.eC[p][cross_index(a, b)] * u[b];
                dE[p][1 + a] = v;
                dO[p][1 + a] = c.oB[p][a];
            }
        }
        df0[0] = c.rA;
        for (int a = 0; a < dim; ++a) df0[1 + a] = 2.0 * c.rC[a] * u[a];
    } else {
        return -1.0;
    }
    const long long all = dense ? 96 : 32;
    const int low = dense ? 16 : 4, sweep = dense ? 64 : 16;
    std::vector<cplx> ph[3];
    for (int a = 0; a < 3; ++a)
        ph[a] = a < dim ? axis_phasors(r.n[a], a == dim - 1, all, low, sweep) : std::vector<cplx>{cplx(1.0, 0.0)};
    int pe[kMaxPair][3];
    for (int p = 0; p < NP; ++p)
        for (int a = 0; a < 3; ++a) pe[p][a] = a < dim ? pair_e(r.lat, p, a) : 0;
    double lmax = 0.0;
    for (const cplx& qz : ph[2])
        for (const cplx& qy : ph[1])
            for (const cplx& qx : ph[0]) {
                const cplx q[3] = {qx, qy, qz};
                double cs[kMaxPair], sn[kMaxPair];   // 2 cos(theta . e_p), 2 sin(theta . e_p)
                for (int p = 0; p < NP; ++p) {
                    cplx v(1.0, 0.0);
                    for (int a = 0; a < 3; ++a) {
                        if (pe[p][a] == 1) v *= q[a];
                        else if (pe[p][a] == -1) v *= std::conj(q[a]);
                    }
                    cs[p] = 2.0 * v.real();
                    sn[p] = 2.0 * v.imag();
                }
                cplx M[2][4][4] = {};
                for (int l = 0; l < nl; ++l) {
                    for (int j = 0; j < nf; ++j) {
                        cplx s = c.ap[l] * df0[j] + (j == 0 ? c.a0[l] : 0.0);
                        for (int p = 0; p < NP; ++p)
                            s += cplx(c.ap[l] * dE[p][j] * cs[p], c.am[l] * dO[p][j] * sn[p]);
                        M[l][0][j] = s;
                    }
                    for (int a = 0; a < nf - 1; ++a)
                        for (int j = 0; j < nf; ++j) {
                            cplx s = (j == 1 + a) ? c.ab0[l] : 0.0;
                            for (int p = 0; p < NP; ++p)
                                if (pe[p][a] != 0)
                                    s += (pe[p][a] * c.fmom[a]) *
                                         cplx(c.abp[l] * dO[p][j] * cs[p], c.abm[l] * dE[p][j] * sn[p]);
                            M[l][1 + a][j] = s;
                        }
                }
                cplx A[kMaxN][kMaxN] = {};
                const int n = nf * nl;
                for (int i = 0; i < nf; ++i)
                    for (int j = 0; j < nf; ++j) {
                        A[i][j] = M[0][i][j];
                        if (nl == 2) A[i][nf + j] = M[1][i][j];
                    }
                if (nl == 2)
                    for (int i = 0; i < nf; ++i) A[nf + i][i] = 1.0;
                lmax = std::max(lmax, spectral_radius(n, A));
            }
    return lmax;
}

}  // namespace mmfd
