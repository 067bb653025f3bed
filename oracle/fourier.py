"""Fourier analysis of the linear MMFD scheme (Sec. III.D of arXiv 2505.17057) -- oracle side.

Test infrastructure only.  For the linear CDE the EDF is f_j^eq = phi ubar_j
(Eq. (TforMMFD-0)), so a Fourier mode exp(i theta . x) (theta in index units,
theta_alpha = xi_alpha dx_alpha) is multiplied on level t + q dt by

    A_q(theta) = sum_k a_kq sum_j ubar_j exp(i k theta . e_j)        (Eq. (TforMMFD-3))

* two-level explicit:  lambda = A_{-1}                             (Eq. (TforMMFD-7))
* three-level:         lambda^2 - p_1 lambda - p_0 = 0              (Eq. (3-level))
* theta-scheme:        lambda = (1 + th (A + iB)) / (1 - (1 - th)(A + iB))   (Eq. (Tcond1-1))

It also gives the exact discrete solution of the periodic LCDE
(phi_hat^n = lambda^n phi_hat^0 per mode) and the exact PDE solution.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np

from oracle import oracle as orc


def ubar(prob: orc.Problem) -> np.ndarray:
    """ubar_j = f_j^eq / phi of the LCDE problem (Eq. (TforMMFD-0))."""
    assert prob.pde == "LCDE"
    return orc.feq(prob, [1.0])


def ubar_split(prob: orc.Problem):
    """(ubar^+, ubar^-) with the even/odd split of Eq. (2-5) / (TforMMFD-2)."""
    E, _, _ = orc.lattice(prob.lattice, prob.d0, prob.c)
    ub = ubar(prob)
    opp = np.array([int(np.where((E == -E[j]).all(axis=1))[0][0]) for j in range(E.shape[0])])
    return 0.5 * (ub + ub[opp]), 0.5 * (ub - ub[opp]), E


def thetas(shape) -> list:
    """Discrete wave numbers (index units) of a periodic grid of the given numpy shape."""
    axes = [2.0 * np.pi * np.fft.fftfreq(n) for n in shape]
    return np.meshgrid(*axes, indexing="ij")


def symbol(prob: orc.Problem, coeffs: Sequence[float], shape=None) -> np.ndarray:
    """A(theta) = sum_k a_k sum_j ubar_j exp(i k theta . e_j) on the grid's wave numbers.

    shape defaults to the problem's numpy field shape; the returned array has that shape.
    Axis order follows the numpy layout: (ny, nx) in 2D, (nz, ny, nx) in 3D.
    """
    shape = prob.shape if shape is None else shape
    E, _, _ = orc.lattice(prob.lattice, prob.d0, prob.c)
    ub = ubar(prob)
    th = thetas(shape)
    dim = len(shape)
    # numpy axis i corresponds to lattice axis dim-1-i (x fastest)
    out = np.zeros(shape, dtype=complex)
    for k, a in zip((-1, 0, 1), coeffs):
        if a == 0:
            continue
        for j in range(E.shape[0]):
            phase = np.zeros(shape)
            for i in range(dim):
                phase = phase + th[i] * E[j][dim - 1 - i]
            out += a * ub[j] * np.exp(1j * k * phase)
    return out


def two_level_lambda(prob: orc.Problem, shape=None) -> np.ndarray:
    return symbol(prob, prob.a, shape)


def three_level_roots(prob: orc.Problem, shape=None):
    """Roots of lambda^2 - p_1 lambda - p_0 with p_1 = A(level t), p_0 = A(level t - dt)."""
    p1 = symbol(prob, prob.a, shape)
    p0 = symbol(prob, prob.ahat, shape)
    disc = np.sqrt(p1 * p1 + 4.0 * p0 + 0j)
    return 0.5 * (p1 + disc), 0.5 * (p1 - disc), p1, p0


def max_amplification(prob: orc.Problem, shape=None) -> float:
    if prob.levels == 2:
        return float(np.max(np.abs(two_level_lambda(prob, shape))))
    l1, l2, _, _ = three_level_roots(prob, shape)
    return float(max(np.max(np.abs(l1)), np.max(np.abs(l2))))


# ------------------------------------------------------------------ exact solutions

def discrete_exact(prob: orc.Problem, phi0: np.ndarray, nsteps: int, phim1: np.ndarray = None) -> np.ndarray:
    """Exact solution of the linear periodic scheme after nsteps (Eq. (TforMMFD-3)).

    Two-level: phi_hat^n = lambda^n phi_hat^0.  Three-level: the companion matrix
    [[p_1, p_0], [1, 0]] raised to the n-th power acts on (phi_hat^0, phi_hat^{-1}).
    """
    F0 = np.fft.fftn(phi0)
    if prob.levels == 2:
        lam = two_level_lambda(prob, phi0.shape)
        return np.real(np.fft.ifftn(F0 * lam ** nsteps))
    p1 = symbol(prob, prob.a, phi0.shape)
    p0 = symbol(prob, prob.ahat, phi0.shape)
    Fm = np.fft.fftn(phim1)
    # M^n by repeated squaring, elementwise over modes
    m00, m01, m10, m11 = p1.copy(), p0.copy(), np.ones_like(p1), np.zeros_like(p1)
    r00, r01, r10, r11 = np.ones_like(p1), np.zeros_like(p1), np.zeros_like(p1), np.ones_like(p1)
    n = int(nsteps)
    while n > 0:
        if n & 1:
            r00, r01, r10, r11 = (r00 * m00 + r01 * m10, r00 * m01 + r01 * m11,
                                  r10 * m00 + r11 * m10, r10 * m01 + r11 * m11)
        m00, m01, m10, m11 = (m00 * m00 + m01 * m10, m00 * m01 + m01 * m11,
                              m10 * m00 + m11 * m10, m10 * m01 + m11 * m11)
        n >>= 1
    return np.real(np.fft.ifftn(r00 * F0 + r01 * Fm))


def pde_exact_lcde(phi0: np.ndarray, K, u, t: float, dx: Sequence[float]) -> np.ndarray:
    """Exact solution of d_t phi + u . grad phi = div(K grad phi) (Eq. (LCDE), constant K, u)
    for the periodic trigonometric interpolant of phi0:
        phi_hat_m(t) = phi_hat_m(0) exp(-(i k . u + k^T K k) t),
    k_alpha = 2 pi m_alpha / (N_alpha dx_alpha)."""
    shape = phi0.shape
    dim = len(shape)
    ks = []
    for i in range(dim):
        lat_axis = dim - 1 - i
        n = shape[i]
        ks.append(2.0 * np.pi * np.fft.fftfreq(n, d=dx[lat_axis]))
    grids = np.meshgrid(*ks, indexing="ij")
    kv = [grids[dim - 1 - a] for a in range(dim)]  # kv[a] is the wave number along lattice axis a
    K = np.asarray(K, dtype=float)
    expo = np.zeros(shape, dtype=complex)
    for a in range(dim):
        expo += 1j * kv[a] * u[a]
        for b in range(dim):
            expo += kv[a] * K[a][b] * kv[b]
    return np.real(np.fft.ifftn(np.fft.fftn(phi0) * np.exp(-expo * t)))


# ------------------------------------------------------------------ stability predicates

def theorem1(prob: orc.Problem) -> dict:
    """Conditions (a)-(c) of Theorem 1 (Eq. (Tcond)) for the two-level explicit scheme, m = 1."""
    up, um, E = ubar_split(prob)
    am1, a0, a1 = prob.a
    ap, amn = a1 + am1, a1 - am1
    js = [j for j in range(E.shape[0]) if np.any(E[j] != 0)]
    den = np.array([ap * up[j] for j in js])
    num = np.array([(amn * um[j]) ** 2 for j in js])
    cond_a = bool(np.all(den > 0))
    cond_b = bool(den.sum() <= 1.0 + 1e-14)
    pos = den > 0
    # Remark 2: terms with a zero denominator need a zero numerator and drop out
    ok_zero = bool(np.all(num[~pos] <= 1e-30))
    cond_c = ok_zero and bool((num[pos] / den[pos]).sum() <= 1.0 + 1e-14)
    # Eq. (Tcond-3): (b) <=> a_0 + ubar_0^+ (1 - a_0) >= 0
    j0 = [j for j in range(E.shape[0]) if not np.any(E[j] != 0)][0]
    cond_b_alt = bool(a0 + up[j0] * (1.0 - a0) >= -1e-14)
    return {"a": cond_a, "b": cond_b, "c": cond_c, "b_alt": cond_b_alt}


def theorem3_holds(prob: orc.Problem, shape=None, tol: float = 1e-12) -> bool:
    """Schur-Cohn test of Theorem 3, |p_1 + conj(p_1) p_0| <= 1 - |p_0|^2, at every wave number."""
    p1 = symbol(prob, prob.a, shape)
    p0 = symbol(prob, prob.ahat, shape)
    lhs = np.abs(p1 + np.conj(p1) * p0)
    rhs = 1.0 - np.abs(p0) ** 2
    return bool(np.all(lhs <= rhs + tol))


def theta_AB(prob: orc.Problem, shape=None):
    """A and B of Eq. (Tcond1-2) (m_0 = 1) on the grid's wave numbers."""
    up, um, E = ubar_split(prob)
    shape = prob.shape if shape is None else shape
    th = thetas(shape)
    dim = len(shape)
    am1, a0, a1 = prob.a
    A = np.zeros(shape)
    B = np.zeros(shape)
    for j in range(E.shape[0]):
        xi = np.zeros(shape)
        for i in range(dim):
            xi = xi + th[i] * E[j][dim - 1 - i]
        A += (a1 + am1) * up[j] * (np.cos(xi) - 1.0)
        B += (a1 - am1) * um[j] * np.sin(xi)
    return A, B


def theta_lambda(prob: orc.Problem, theta: float, shape=None):
    """Amplification factor of the two-level theta-scheme Eq. (GCN), Eq. (Tcond1-1)."""
    A, B = theta_AB(prob, shape)
    z = A + 1j * B
    return (1.0 + theta * z) / (1.0 - (1.0 - theta) * z)
