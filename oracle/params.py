"""Parameter design of the MMFD schemes (Sec. III of arXiv 2505.17057) -- oracle side.

Test infrastructure only (see oracle.py).  Independent of the CUDA package's
own host-side parameter solver.

* ``coefficient_moments``: A_lm of Eq. (4-2) / (4-2-0), with the Remark 1(5)
  shift of the A_l0 when the left-hand side sits at t + dt (three-level).
* ``solve_three_level``: Eq. (X), the solution X = A^{-1} b of the linear system
  Eq. (AX_b) for (a_1, a_{-1}, ahat_0, ahat_1, ahat_{-1}) from the design targets
  (a_0, A_10, A_11, A_21, A_22).  The printed X lists ahat_{-1} twice; it is read
  as (a_1, a_{-1}, ahat_0, ahat_1, ahat_{-1}) as in Eq. (X).
* ``two_level_from_a0``: Eq. (LMMFD-2-1)/(LMMFD-2-2): A_10 = A_11 = -1 with m = 1.
* ``problem_*``: map a physical problem (diffusion tensor, velocity, nonlinear
  flux and diffusivity, He-Luo NSE) to the explicit EDF parameters using
  alpha = -(A_22 / A_10) dt beta c_s^2 (Eq. (M-NCDE-6)) and the second-order
  moment equation Eq. (ME-NCDE-3-2-1).

Exact rational arithmetic is used whenever the inputs are Fractions.
"""
from __future__ import annotations

from fractions import Fraction
from math import comb, factorial
from typing import Dict, Sequence, Tuple

import numpy as np

from oracle.oracle import Problem, LATTICE_DIM

Triple = Tuple[object, object, object]  # (a_{-1}, a_0, a_1)


def coefficient_moments(coeffs: Dict[Tuple[int, int], object], lhs_shift: bool, lmax: int = 3):
    """A_lm = (1/l!) C_l^m sum_{k,q} a_kq q^{l-m} k^m (Eq. (4-2)).

    ``coeffs`` maps (k, q) -> a_kq.  With ``lhs_shift`` (left-hand side at
    t + dt, Remark 1(5)) the pure time moments become
    A_l0 = (1/l!) [sum a_kq q^l - 1] for l >= 1.
    Returns a dict {(l, m): A_lm}.
    """
    out = {}
    for l in range(lmax + 1):
        for m in range(l + 1):
            s = 0
            for (k, q), a in coeffs.items():
                s += a * (q ** (l - m)) * (k ** m)
            if lhs_shift and m == 0 and l >= 1:
                s -= 1
            val = Fraction(comb(l, m), factorial(l)) * s if isinstance(s, Fraction) else comb(l, m) * s / factorial(l)
            out[(l, m)] = val
    return out


def three_level_coeffs(a: Triple, ahat: Triple) -> Dict[Tuple[int, int], object]:
    """(k, q) map of Eq. (3layer-1): a_k on q = 0 (level t), ahat_k on q = -1 (level t - dt)."""
    d = {}
    for k, v in zip((-1, 0, 1), a):
        d[(k, 0)] = v
    for k, v in zip((-1, 0, 1), ahat):
        d[(k, -1)] = v
    return d


def two_level_coeffs(a: Triple) -> Dict[Tuple[int, int], object]:
    """(k, q) map of the explicit two-level scheme Eq. (2-2-2): every term on q = -1."""
    return {(k, -1): v for k, v in zip((-1, 0, 1), a)}


def three_level_moments(a: Triple, ahat: Triple):
    """A_00, A_10, A_11, A_20, A_21, A_22 of Eq. (4-2-00a) (left-hand side at t + dt)."""
    A = coefficient_moments(three_level_coeffs(a, ahat), lhs_shift=True, lmax=2)
    # Eq. (4-2-00a) states A_00 = sum of all coefficients; the shift leaves l = 0 untouched.
    return A


def two_level_moments(a: Triple):
    return coefficient_moments(two_level_coeffs(a), lhs_shift=False, lmax=2)


# The coefficient matrix of Eq. (AX_b) acting on X = (a_1, a_{-1}, ahat_0, ahat_1, ahat_{-1}).
AX_MATRIX = [
    [1, 1, 1, 1, 1],
    [0, 0, -1, -1, -1],
    [1, -1, 0, 1, -1],
    [0, 0, 0, -1, 1],
    [Fraction(1, 2), Fraction(1, 2), 0, Fraction(1, 2), Fraction(1, 2)],
]
# Its printed inverse, Eq. (invA) (times 1/2).
AX_INVERSE = [[Fraction(v, 2) for v in row] for row in [
    [1, 1, 1, 1, 0],
    [1, 1, -1, -1, 0],
    [2, 0, 0, 0, -4],
    [-1, -1, 0, -1, 2],
    [-1, -1, 0, 1, 2],
]]


def solve_three_level(a0, A10, A11, A21, A22):
    """Eq. (X): returns (a, ahat) as (a_{-1}, a_0, a_1), (ahat_{-1}, ahat_0, ahat_1).

    X = A^{-1} b with b = (1 - a_0, 1 + A_10, A_11, A_21, A_22) (Eq. (AX_b)); written out:
      a_1      = (-a_0 + A_10 + A_11 + A_21 + 2) / 2
      a_{-1}   = (-a_0 + A_10 - A_11 - A_21 + 2) / 2
      ahat_0   = (-2 a_0 - 4 A_22 + 2) / 2
      ahat_1   = (a_0 - A_10 - A_21 + 2 A_22 - 2) / 2
      ahat_{-1}= (a_0 - A_10 + A_21 + 2 A_22 - 2) / 2
    """
    half = Fraction(1, 2) if all(isinstance(v, (int, Fraction)) for v in (a0, A10, A11, A21, A22)) else 0.5
    a1 = half * (-a0 + A10 + A11 + A21 + 2)
    am1 = half * (-a0 + A10 - A11 - A21 + 2)
    ah0 = half * (-2 * a0 - 4 * A22 + 2)
    ah1 = half * (a0 - A10 - A21 + 2 * A22 - 2)
    ahm1 = half * (a0 - A10 + A21 + 2 * A22 - 2)
    return (am1, a0, a1), (ahm1, ah0, ah1)


def two_level_from_a0(a0):
    """Eq. (LMMFD-2-1)/(LMMFD-2-2) with m = 1: A_00 = 1, A_10 = A_11 = -1 give
    a_{-1} = 1 - a_0/2, a_1 = -a_0/2 (and A_22 = (1 - a_0)/2)."""
    if isinstance(a0, (int, Fraction)):
        a0 = Fraction(a0)
        return (1 - a0 / 2, a0, -a0 / 2)
    return (1.0 - a0 / 2.0, float(a0), -a0 / 2.0)


# ------------------------------------------------------------------ physical -> EDF parameters

def _scheme_moments(levels: int, a: Triple, ahat: Triple):
    if levels == 2:
        A = two_level_moments(a)
    else:
        A = three_level_moments(a, ahat)
    return float(A[(1, 0)]), float(A[(2, 0)]), float(A[(2, 1)]), float(A[(2, 2)])


def lattice_c(dt: float, dx: Sequence[float], dim: int):
    return [dx[i] / dt if i < dim else 0.0 for i in range(3)]


def problem_lcde(lattice: str, levels: int, n, dt: float, dx, K, u, a: Triple,
                 ahat: Triple = (0.0, 0.0, 0.0), d0=None, lambda_bar: float = 1.0) -> Problem:
    """Linear CDE (Eq. (LCDE)) with diffusion tensor K = alpha D0 and constant u.

    Quadratic lattices (D2Q9, D3Q19): C = c_s^2 (beta D0 - I) + lambda_bar u u with
    beta D0 = K / (-(A_22/A_10) dt c_s^2) (Eq. (TforMMFD-0), alpha from Eq. (M-NCDE-6)),
    d0 as given (default 1/3).
    Axis lattices (D2Q5, D3Q7): linear EDF (C = 0, Eq. (Tcond-4) context) with direction-
    dependent c_salpha^2 chosen so that the recovered diffusion Eq. (ME-NCDE-3-2-1),
      K_eff = -(dt/A_10) [A_22 diag(c_s^2) - (A_21 - A_20) u u],
    has diagonal K_alphaalpha; the off-diagonal of K cannot be carried on these lattices.
    """
    dim = LATTICE_DIM[lattice]
    c = lattice_c(dt, dx, dim)
    A10, A20, A21, A22 = _scheme_moments(levels, a, ahat)
    K = np.asarray(K, dtype=float)
    uu = np.zeros((3, 3))
    uv = np.array(list(u) + [0.0] * (3 - len(u)))[:3]
    for i in range(dim):
        for j in range(dim):
            uu[i, j] = uv[i] * uv[j]
    Cmat = np.zeros((3, 3))
    if lattice in ("D2Q9", "D3Q19"):
        d0v = list(d0) if d0 is not None else [1.0 / 3.0] * dim
        d0v = (d0v + [0.0] * 3)[:3]
        cs2 = [d0v[i] * c[i] ** 2 for i in range(3)]
        for i in range(dim):
            for j in range(dim):
                Cmat[i, j] = -A10 * K[i, j] / (A22 * dt) + lambda_bar * uu[i, j]
            Cmat[i, i] -= cs2[i]
    else:
        d0v = [0.0, 0.0, 0.0]
        for i in range(dim):
            cs2_i = (-A10 * K[i, i] / dt + (A21 - A20) * uu[i, i]) / A22
            d0v[i] = cs2_i / c[i] ** 2
    return Problem(lattice=lattice, pde="LCDE", levels=levels, n=n, c=c, d0=d0v, a=a, ahat=ahat,
                   u=uv, Cmat=Cmat.ravel(), dt=dt)


def effective_diffusion(lattice: str, levels: int, dt: float, K, u, a: Triple,
                        ahat: Triple = (0.0, 0.0, 0.0), lambda_bar: float = 1.0):
    """The diffusion tensor the scheme recovers (second order), per Eq. (ME-NCDE-3-2-1)."""
    dim = LATTICE_DIM[lattice]
    A10, A20, A21, A22 = _scheme_moments(levels, a, ahat)
    K = np.asarray(K, dtype=float)[:dim, :dim]
    uv = np.asarray(u, dtype=float)[:dim]
    uu = np.outer(uv, uv)
    if lattice in ("D2Q9", "D3Q19"):
        return K + (-dt / A10) * (A22 * lambda_bar - (A21 - A20)) * uu
    Keff = -(dt / A10) * (-(A21 - A20) * uu)
    np.fill_diagonal(Keff, np.diag(K))
    return Keff


def wave_coefficients(gamma):
    """Sec. III.C case (4): a = (gamma, 2 (1 - gamma), gamma), ahat = (0, -1, 0)."""
    return (gamma, 2 * (1 - gamma), gamma), (0 * gamma, 0 * gamma - 1, 0 * gamma)


def problem_lwe(lattice: str, n, dt: float, dx, K, a: Triple, ahat: Triple, d0=None) -> Problem:
    """Linear wave equation d_t^2 phi = div(K grad phi) (Eq. (LWE), K = alpha D0), three-level.

    Eq. (ME-NCDE-W-1): d_t^2 phi = A_22 div div M_2 with M_2 = beta c_s^2 D0 phi, so the EDF's
    second moment is K phi / A_22: on D2Q9 / D3Q19 C = K / A_22 - c_s^2 I (u = 0 in
    Eq. (TforMMFD-0)); on D2Q5 / D3Q7 the linear EDF (C = 0) with c_salpha^2 = K_alphaalpha / A_22.
    """
    dim = LATTICE_DIM[lattice]
    c = lattice_c(dt, dx, dim)
    A = three_level_moments(a, ahat)
    A22 = float(A[(2, 2)])
    K = np.asarray(K, dtype=float)
    Cmat = np.zeros((3, 3))
    if lattice in ("D2Q9", "D3Q19"):
        d0v = list(d0) if d0 is not None else [1.0 / 3.0] * dim
        d0v = (d0v + [0.0] * 3)[:3]
        for i in range(dim):
            for j in range(dim):
                Cmat[i, j] = K[i, j] / A22
            Cmat[i, i] -= d0v[i] * c[i] ** 2
    else:
        d0v = [0.0, 0.0, 0.0]
        for i in range(dim):
            d0v[i] = K[i, i] / A22 / c[i] ** 2
    return Problem(lattice=lattice, pde="LCDE", levels=3, n=n, c=c, d0=d0v, a=a, ahat=ahat,
                   u=(0.0, 0.0, 0.0), Cmat=Cmat.ravel(), dt=dt)


def problem_ncde(lattice: str, levels: int, n, dt: float, dx, flux_poly, diff_poly, a: Triple,
                 ahat: Triple = (0.0, 0.0, 0.0), d0=None) -> Problem:
    """NCDE  d_t phi + div B(phi) = div(D(phi) grad phi), D isotropic (Eq. (NCDE0)).

    flux_poly[alpha][p]: B_alpha(phi) = sum_p flux_poly[alpha][p] phi^p.
    diff_poly[p]: D(phi) = sum_p diff_poly[p] phi^p, so div(D grad phi) = lap G(phi) with
    G' = D, G(0) = 0.  Eq. (M-NCDE-6) with alpha D = G I gives the second-moment target
    beta c_s^2 D = -(A_10/(A_22 dt)) G(phi) I, entered through Eq. (NCDEfeq) with C = 0.
    """
    dim = LATTICE_DIM[lattice]
    c = lattice_c(dt, dx, dim)
    A10, A20, A21, A22 = _scheme_moments(levels, a, ahat)
    d0v = list(d0) if d0 is not None else [1.0 / 3.0] * dim
    d0v = (d0v + [0.0] * 3)[:3]
    flux = np.zeros(12)
    for al in range(dim):
        for p, v in enumerate(flux_poly[al]):
            flux[4 * al + p] = v
    m2 = np.zeros(5)
    for p, v in enumerate(diff_poly):
        m2[p + 1] = -A10 * v / ((p + 1) * A22 * dt)
    return Problem(lattice=lattice, pde="NCDE", levels=levels, n=n, c=c, d0=d0v, a=a, ahat=ahat,
                   flux=flux, m2=m2, dt=dt)


def problem_nse(lattice: str, levels: int, n, dt: float, dx, a: Triple, abar: Triple,
                ahat: Triple = (0.0, 0.0, 0.0), abarhat: Triple = (0.0, 0.0, 0.0),
                d0=None, rho0: float = 1.0) -> Problem:
    """Incompressible NSE with the He-Luo EDF g^eq(rho, rho0 u, rho0 u u) (Remark 4);
    rho uses {a}, rho u uses {abar} (double-distribution form Eq. (2-4))."""
    dim = LATTICE_DIM[lattice]
    c = lattice_c(dt, dx, dim)
    d0v = list(d0) if d0 is not None else [1.0 / 3.0] * dim
    d0v = (d0v + [0.0] * 3)[:3]
    return Problem(lattice=lattice, pde="NSE", levels=levels, n=n, c=c, d0=d0v, a=a, ahat=ahat,
                   abar=abar, abarhat=abarhat, rho0=rho0, dt=dt)


def nse_viscosity(levels: int, abar: Triple, abarhat: Triple, dt: float, cs2: float) -> float:
    """nu = -(Abar_22 / Abar_10) dt c_s^2 (Eq. (M-NSEs-4c))."""
    A10, _, _, A22 = _scheme_moments(levels, abar, abarhat)
    return -(A22 / A10) * dt * cs2
