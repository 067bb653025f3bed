"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test pins the oracle to something other than itself: values printed in
the paper, textbook special cases, closed forms, exact invariants, or an
independent brute-force computation.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import fourier as F
from oracle import oracle as orc
from oracle import params as P
from paper_2505_17057_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "coefficient_sets.json")
RNG = np.random.default_rng(20250517)


def fr(s):
    return Fraction(s)


# ----------------------------------------------------------------------------- lattices (App. A)

def test_d2q9_standard_weights():
    # Example 1 states omega_0 = 4/9, omega_1-4 = 1/9, omega_5-8 = 1/36 with c_s^2 = c^2/3.
    E, w, cs2 = orc.lattice("D2Q9", [1 / 3, 1 / 3], [1.0, 1.0])
    assert np.allclose(w, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, atol=1e-15)
    assert np.allclose(cs2[:2], [1 / 3, 1 / 3])


def test_d3q19_standard_weights():
    # Textbook D3Q19 weights 1/3, 1/18 (x6), 1/36 (x12) at d_0 = 1/3.
    E, w, cs2 = orc.lattice("D3Q19", [1 / 3] * 3, [1.0] * 3)
    assert np.allclose(w, [1 / 3] + [1 / 18] * 6 + [1 / 36] * 12, atol=1e-15)
    # 19 distinct velocities, closed under reversal
    assert len({tuple(e) for e in E}) == 19
    for e in E:
        assert any((E == -e).all(axis=1))


@pytest.mark.parametrize("lat,d0,c", [
    ("D2Q5", [0.3, 0.2], [1.0, 1.5]),
    ("D2Q9", [0.3, 0.45], [1.2, 0.8]),
    ("D3Q7", [0.2, 0.25, 0.3], [1.0, 1.1, 0.9]),
    ("D3Q19", [0.3, 0.35, 0.4], [1.0, 1.3, 0.7]),
])
def test_lattice_second_moment(lat, d0, c):
    # Delta^(2) = sum_j omega_j c_j c_j = diag(c_salpha^2) with c_salpha^2 = d_0alpha c_alpha^2 (App. A, Eq. (3-4)).
    E, w, cs2 = orc.lattice(lat, d0, c)
    dim = 2 if lat.startswith("D2") else 3
    cj = E[:, :dim] * np.array(c[:dim])
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(cj.T @ w, 0.0, atol=1e-15)
    assert np.allclose((cj.T * w) @ cj, np.diag([d0[a] * c[a] ** 2 for a in range(dim)]), atol=1e-14)


@pytest.mark.parametrize("lat,d0,c", [
    ("D2Q9", [0.3, 0.45], [1.2, 0.8]),
    ("D3Q19", [0.3, 0.35, 0.4], [1.0, 1.3, 0.7]),
])
def test_lattice_fourth_moment(lat, d0, c):
    # Eq. (3-6): Delta^(4) = <Delta^(2) Delta^(2)> + delta^(4), delta^(4)_aaaa = cs_a^2 (c_a^2 - 3 cs_a^2).
    E, w, cs2 = orc.lattice(lat, d0, c)
    dim = 2 if lat == "D2Q9" else 3
    cj = E[:, :dim] * np.array(c[:dim])
    D2 = np.diag(cs2[:dim])
    D4 = np.einsum("j,ja,jb,jc,jd->abcd", w, cj, cj, cj, cj)
    ref = (np.einsum("ab,cd->abcd", D2, D2) + np.einsum("ac,bd->abcd", D2, D2) + np.einsum("bc,ad->abcd", D2, D2))
    for a in range(dim):
        ref[a, a, a, a] += cs2[a] * (c[a] ** 2 - 3 * cs2[a])
    assert np.allclose(D4, ref, atol=1e-14)


# ----------------------------------------------------------------------------- EDF (Eq. (3-3)..(3-7))

@pytest.mark.parametrize("lat,d0,c", [
    ("D2Q9", [1 / 3, 1 / 3], [1.0, 1.0]),
    ("D2Q9", [0.3, 0.45], [1.2, 0.8]),
    ("D3Q19", [1 / 3] * 3, [1.0] * 3),
    ("D3Q19", [0.3, 0.35, 0.4], [1.0, 1.3, 0.7]),
])
def test_edf_moment_identities(lat, d0, c):
    # Eq. (3-5a,b) and Eq. (3-7) on the lattices with the Delta^(4) structure.
    dim = 2 if lat == "D2Q9" else 3
    E, w, cs2 = orc.lattice(lat, d0, c)
    cj = E[:, :dim] * np.array(c[:dim])
    for _ in range(5):
        A = RNG.normal()
        B = np.zeros(3); B[:dim] = RNG.normal(size=dim)
        Cm = np.zeros((3, 3)); S = RNG.normal(size=(dim, dim)); Cm[:dim, :dim] = S + S.T
        g = orc.geq(lat, d0, c, A, B, Cm)
        assert abs(g.sum() - A) < 1e-14
        assert np.allclose(cj.T @ g, B[:dim], atol=1e-14)
        assert np.allclose((cj.T * g) @ cj, A * np.diag(cs2[:dim]) + Cm[:dim, :dim], atol=1e-13)
        M3 = np.einsum("j,ja,jb,jc->abc", g, cj, cj, cj)
        D2 = np.diag(cs2[:dim])
        ref = (np.einsum("ab,c->abc", D2, B[:dim]) + np.einsum("ac,b->abc", D2, B[:dim])
               + np.einsum("bc,a->abc", D2, B[:dim]))
        for a in range(dim):
            ref[a, a, a] += cs2[a] * (c[a] ** 2 - 3 * cs2[a]) * B[a] / cs2[a]
        assert np.allclose(M3, ref, atol=1e-13)


@pytest.mark.parametrize("lat", ["D2Q5", "D3Q7"])
def test_linear_edf_moments_axis_lattices(lat):
    # With C = 0 the axis lattices still carry Eq. (3-5a): sum g = A, sum c g = B, sum c c g = A Delta^(2).
    dim = 2 if lat == "D2Q5" else 3
    d0 = [0.2, 0.15, 0.25][:dim]
    c = [1.0, 1.4, 0.8][:dim]
    E, w, cs2 = orc.lattice(lat, d0, c)
    cj = E[:, :dim] * np.array(c)
    A = 0.7
    B = np.array([0.1, -0.2, 0.05])
    g = orc.geq(lat, d0, c, A, B, np.zeros((3, 3)))
    assert abs(g.sum() - A) < 1e-15
    assert np.allclose(cj.T @ g, B[:dim], atol=1e-15)
    assert np.allclose((cj.T * g) @ cj, A * np.diag(cs2[:dim]), atol=1e-15)


def test_edf_matches_printed_example_form():
    # Examples 1-2 print f_j^eq = omega_j phi [1 + c_j.u/cs^2 + (uu + (beta-1) cs^2 I):(c_j c_j - cs^2 I)/(2 cs^4)]
    # on the standard D2Q9 lattice.  The oracle's LCDE EDF with C = phi (uu + (beta-1) cs^2 I) must equal it.
    c = 1.2
    cs2 = c * c / 3
    u = np.array([1.0, 1.0])
    beta = 0.5
    phi = 0.83
    prob = orc.Problem(lattice="D2Q9", pde="LCDE", levels=2, n=[1, 1], c=[c, c], d0=[1 / 3, 1 / 3],
                       a=(1, 0, 0), u=[u[0], u[1], 0],
                       Cmat=[u[0] * u[0] + (beta - 1) * cs2, u[0] * u[1], 0,
                             u[1] * u[0], u[1] * u[1] + (beta - 1) * cs2, 0, 0, 0, 0])
    g = orc.feq(prob, [phi])
    E, w, _ = orc.lattice("D2Q9", [1 / 3, 1 / 3], [c, c])
    for j in range(9):
        cj = E[j, :2] * c
        T = np.outer(u, u) + (beta - 1) * cs2 * np.eye(2)
        Q = np.outer(cj, cj) - cs2 * np.eye(2)
        ref = w[j] * phi * (1 + cj @ u / cs2 + np.sum(T * Q) / (2 * cs2 * cs2))
        assert abs(g[j] - ref) < 1e-14


# ----------------------------------------------------------------------------- scheme forms

CASES = [
    ("D2Q5", "LCDE", 2), ("D2Q9", "LCDE", 2), ("D2Q9", "LCDE", 3), ("D2Q9", "NCDE", 3),
    ("D2Q9", "NSE", 2), ("D2Q9", "NSE", 3), ("D3Q7", "LCDE", 2), ("D3Q19", "LCDE", 2),
    ("D3Q19", "NSE", 2), ("D3Q19", "NCDE", 3),
]


def _random_problem(lat, pde, levels, n):
    dim = 2 if lat.startswith("D2") else 3
    dt = 0.7
    dx = [0.9, 1.1, 1.0][:dim]
    a = (0.8, 0.3, -0.1)
    ahat = (0.15, -0.2, 0.05)
    if pde == "LCDE":
        K = np.diag([0.02, 0.015, 0.01][:dim]) + 0.002 * (1 - np.eye(dim))
        return P.problem_lcde(lat, levels, n, dt, dx, K, [0.1, -0.05, 0.03][:dim], a, ahat)
    if pde == "NCDE":
        flux = [[0, 0, 0.5, 0], [0, 0.1, 0.5, 0], [0, 0, 0.2, 0.1]][:dim]
        return P.problem_ncde(lat, levels, n, dt, dx, flux, [0.01, 0, 0.01], a, ahat)
    return P.problem_nse(lat, levels, n, dt, dx, a, (0.7, 0.4, -0.1), ahat, (0.1, -0.15, 0.05))


def _random_level(prob, scale=0.05):
    shape = prob.shape
    if prob.pde == "NSE":
        return [1 + scale * RNG.normal(size=shape)] + [scale * RNG.normal(size=shape) for _ in range(prob.dim)]
    return [1 + 0.3 * RNG.normal(size=shape)]


@pytest.mark.parametrize("lat,pde,levels", CASES)
def test_three_forms_agree(lat, pde, levels):
    # MesoFD Eq. (2-1) + moments, direct MMFD Eq. (2-2)/(2-4), central MMFD Eq. (2-2-1)/(2-4-1):
    # algebraically identical, so they agree to rounding.
    n = [5, 4] if lat.startswith("D2") else [4, 3, 5]
    prob = _random_problem(lat, pde, levels, n)
    L0 = _random_level(prob)
    L1 = _random_level(prob) if levels == 3 else None
    outs = [orc.step(prob, L0, L1, form=f) for f in ("mesofd", "mmfd", "central")]
    for i in range(prob.nf):
        scale = max(1.0, np.abs(outs[1][i]).max())
        assert np.abs(outs[0][i] - outs[1][i]).max() < 1e-13 * scale
        assert np.abs(outs[2][i] - outs[1][i]).max() < 1e-13 * scale


def test_step_nodes_matches_full_step():
    prob = _random_problem("D2Q9", "NSE", 2, [7, 6])
    L0 = _random_level(prob)
    full = orc.step(prob, L0)
    nodes = np.array([0, 5, 6, 17, 41])
    part = orc.step_nodes(prob, L0, None, nodes)
    for k, idx in enumerate(nodes):
        for i in range(prob.nf):
            assert part[k, i] == full[i].ravel()[idx]


# ----------------------------------------------------------------------------- LBGK tau = 1 special case

@pytest.mark.parametrize("lat,pde,n", [
    ("D2Q9", "LCDE", [4, 5]), ("D2Q9", "LCDE", [7, 3]), ("D2Q9", "NSE", [4, 5]), ("D2Q9", "NSE", [7, 3]),
    ("D2Q9", "NCDE", [4, 5]), ("D2Q5", "LCDE", [7, 3]), ("D3Q19", "NSE", [3, 4, 5]), ("D3Q7", "LCDE", [3, 4, 5]),
])
def test_lbgk_tau1_equivalence(lat, pde, n):
    # Sec. III.C special case (1) / Example 2 Case 1: SRT LB with tau = 1 is the MMFD scheme with
    # a_{-1} = 1, a_0 = a_1 = 0.  Compared against an independent collide-and-stream code.
    prob = _random_problem(lat, pde, 2, n)
    prob.a = (1.0, 0.0, 0.0)
    prob.abar = (1.0, 0.0, 0.0)
    L0 = _random_level(prob)
    mm, _ = orc.run(prob, L0, nsteps=6)
    lb = orc.lbgk_tau1_run(prob, L0, 6)
    for i in range(prob.nf):
        assert np.abs(mm[i] - lb[i]).max() < 1e-14 * max(1.0, np.abs(lb[i]).max())


# ----------------------------------------------------------------------------- textbook FTCS special case

def test_ftcs_special_case_d2q5():
    # Eq. (LMMFD-4a): on rD2Q5 with the linear EDF, isotropic c_s^2, d_0j = c_s^2 / c_j^2 and
    # a_0 = 1 - 2 alpha/(dt c_s^2), a_{+-1} = (2 alpha/(dt c_s^2) -+ 1)/2 (Eq. (LMMFD-2-2)),
    # the scheme is the textbook FTCS scheme
    #   phi + sum_j [alpha dt/dx_j^2 (phi_j - 2 phi + phi_jbar) - u_j dt/(2 dx_j) (phi_j - phi_jbar)].
    dt, dx, dy = 0.01, 0.1, 0.2
    cs2 = 0.6
    alpha = 0.2
    u = (0.3, -0.4)
    r = 2 * alpha / (dt * cs2)
    a = ((r + 1) / 2, 1 - r, (r - 1) / 2)
    c = [dx / dt, dy / dt]
    prob = orc.Problem(lattice="D2Q5", pde="LCDE", levels=2, n=[6, 5], c=c,
                       d0=[cs2 / c[0] ** 2, cs2 / c[1] ** 2], a=a, u=[u[0], u[1], 0])
    phi = RNG.normal(size=(5, 6))
    out = orc.step(prob, [phi])[0]
    xp, xm = np.roll(phi, -1, axis=1), np.roll(phi, 1, axis=1)
    yp, ym = np.roll(phi, -1, axis=0), np.roll(phi, 1, axis=0)
    ref = (phi + alpha * dt / dx ** 2 * (xp - 2 * phi + xm) - u[0] * dt / (2 * dx) * (xp - xm)
           + alpha * dt / dy ** 2 * (yp - 2 * phi + ym) - u[1] * dt / (2 * dy) * (yp - ym))
    assert np.abs(out - ref).max() < 1e-13


# ----------------------------------------------------------------------------- conservation

@pytest.mark.parametrize("lat,pde,levels", CASES)
def test_mass_conservation(lat, pde, levels):
    # A_00 = 1 (Eq. (4-2-0)) and the periodic shift invariance of sum_x give sum phi^{n+1} = sum phi^n
    # for the two-level scheme; the three-level scheme conserves sum (a) phi^n + sum (ahat) phi^{n-1},
    # i.e. sum phi exactly when sum ahat = 0, and the He-Luo momentum likewise.
    n = [6, 5] if lat.startswith("D2") else [4, 3, 5]
    prob = _random_problem(lat, pde, levels, n)
    if levels == 3:
        # A_10 = -1 <=> sum ahat = 0 (Eq. (4-2-00a)); then a sums to 1.
        prob.a, prob.ahat = (0.7, 0.2, 0.1), (0.1, -0.3, 0.2)
        prob.abar, prob.abarhat = (0.6, 0.3, 0.1), (0.05, -0.1, 0.05)
    L0 = _random_level(prob)
    L1 = [f * 1.0 for f in L0] if levels == 3 else None
    out, _ = orc.run(prob, L0, L1, nsteps=7)
    s0 = L0[0].sum()
    assert abs(out[0].sum() - s0) < 1e-13 * abs(s0)
    if pde == "NSE":
        for d in range(prob.dim):
            m0 = L0[1 + d].sum()
            assert abs(out[1 + d].sum() - m0) < 1e-13 * np.abs(L0[1 + d]).sum()


# ----------------------------------------------------------------------------- parameter design

def _golden():
    with open(GOLDEN) as fh:
        return json.load(fh)


def test_printed_inverse_matrix():
    # Eq. (invA) is the inverse of the matrix of Eq. (AX_b) (exact rationals).
    A, Ai = P.AX_MATRIX, P.AX_INVERSE
    for i in range(5):
        for j in range(5):
            s = sum(Fraction(A[i][k]) * Ai[k][j] for k in range(5))
            assert s == (1 if i == j else 0)


@pytest.mark.parametrize("entry", _golden()["sets"], ids=lambda e: e["name"])
def test_eq_x_reproduces_printed_sets(entry):
    t = {k: fr(v) for k, v in entry["targets"].items()}
    a, ahat = P.solve_three_level(t["a0"], t["A10"], t["A11"], t["A21"], t["A22"])
    expect = entry.get("reading", entry["printed"])
    assert list(a) == [fr(v) for v in expect["a"]]
    assert list(ahat) == [fr(v) for v in expect["ahat"]]
    # and the solved set has the targeted moments, A_00 = 1 and A_20 = -A_10/2 - 1 (Eq. (4-2-00a))
    A = P.three_level_moments(a, ahat)
    assert A[(0, 0)] == 1
    assert A[(1, 0)] == t["A10"] and A[(1, 1)] == t["A11"]
    assert A[(2, 1)] == t["A21"] and A[(2, 2)] == t["A22"]
    assert A[(2, 0)] == -t["A10"] / 2 - 1


def test_ex1_case2_printed_sign_breaks_a00():
    e = [s for s in _golden()["sets"] if s["name"] == "ex1_case2"][0]
    a = [fr(v) for v in e["printed"]["a"]]
    ah = [fr(v) for v in e["printed"]["ahat"]]
    assert sum(a) + sum(ah) == Fraction(3, 4)


@pytest.mark.parametrize("entry", _golden()["special_cases"], ids=lambda e: e["name"])
def test_special_cases_moments(entry):
    # Every special case of Sec. III.C satisfies A_00 = 1 and A_20 = -A_10/2 - 1.
    a = [fr(v) for v in entry["a"]]
    ah = [fr(v) for v in entry["ahat"]]
    A = P.three_level_moments(a, ah)
    assert A[(0, 0)] == 1
    assert A[(2, 0)] == -A[(1, 0)] / 2 - 1
    if entry["name"].startswith("wave"):
        # wave equation: A_20 = -1, A_22 = gamma (Example 3)
        assert A[(2, 0)] == -1 and A[(2, 2)] == fr(entry["gamma"])


def test_two_level_parameters():
    # Eq. (LMMFD-2-1): A_00 = 1, A_10 = A_11 = -1, A_22 = (a_1 + a_{-1})/2
    for a0 in (Fraction(0), Fraction(1, 4), Fraction(-1, 3)):
        a = P.two_level_from_a0(a0)
        A = P.two_level_moments(a)
        assert A[(0, 0)] == 1 and A[(1, 0)] == -1 and A[(1, 1)] == -1
        assert A[(2, 2)] == (1 - a0) / 2


# ----------------------------------------------------------------------------- Fourier / exact solutions

def test_config1_discrete_exact_d2q5_and_d2q9():
    # 64x64 periodic LCDE, u = (0.1, 0.05), K = [[0.02, 0.005], [0.005, 0.01]], Gaussian sigma = 6,
    # 200 steps, lattice units.  The scheme equals lambda^n per Fourier mode (Eq. (TforMMFD-7)).
    K = [[0.02, 0.005], [0.005, 0.01]]
    u = [0.1, 0.05]
    a = P.two_level_from_a0(0.0)
    phi0 = inputs.gaussian_hill_2d(64, 64, 32, 32, 6.0)
    for lat in ("D2Q5", "D2Q9"):
        prob = P.problem_lcde(lat, 2, [64, 64], 1.0, [1.0, 1.0], K, u, a)
        out = orc.run(prob, [phi0], nsteps=200)[0][0]
        ex = F.discrete_exact(prob, phi0, 200)
        assert np.abs(out - ex).max() < 1e-12
        # and approximates the PDE it recovers (second order): D2Q9 the full K, D2Q5 diag(K) + the
        # -dt (A_21 - A_20) u u cross term it cannot cancel.
        Keff = P.effective_diffusion(lat, 2, 1.0, K, u, a)
        pde = F.pde_exact_lcde(phi0, Keff, u, 200.0, [1.0, 1.0])
        gre = np.abs(out - pde).sum() / np.abs(pde).sum()
        assert gre < 0.03


def test_three_level_discrete_exact():
    # Example 2 Case 2 / Case 3 coefficient sets on a small periodic grid: three-level scheme vs the
    # companion-matrix power of Eq. (3-level).
    rows = {s["name"]: s for s in _golden()["sets"]}
    for name in ("ex2_case2", "ex2_case3"):
        s = rows[name]
        a = tuple(float(fr(v)) for v in s["printed"]["a"])
        ah = tuple(float(fr(v)) for v in s["printed"]["ahat"])
        prob = P.problem_lcde("D2Q9", 3, [12, 10], 0.05, [0.1, 0.1], [[0.02, 0], [0, 0.02]], [0.3, 0.2], a, ah)
        phi0 = RNG.normal(size=(10, 12))
        phim = RNG.normal(size=(10, 12))
        out = orc.run(prob, [phi0], [phim], nsteps=25)[0][0]
        ex = F.discrete_exact(prob, phi0, 25, phim)
        assert np.abs(out - ex).max() < 1e-11 * max(1.0, np.abs(ex).max())


def _ex2_gre(case: int, nx: int, D: float = 0.02, T: float = 1.0):
    """Example 2: d_t phi + u.grad phi = D lap phi on [0,2]^2, u = (1,1), dx = 1/nx, dt = 1/nt with
    the (nx, nt) pairs of Table 2 (nt = 12 (nx/10)^2 for D = 0.02, 6 (nx/10)^2 for D = 0.01), exact
    solution exp(-2 D pi^2 t) cos(pi (x + y) - pi (u_x + u_y) t); three-level start from the exact
    solution at t = -dt."""
    rows = {s["name"]: s for s in _golden()["sets"]}
    s = rows[f"ex2_case{case}"]
    a = tuple(float(fr(v)) for v in s["printed"]["a"])
    ah = tuple(float(fr(v)) for v in s["printed"]["ahat"])
    nt = int(round((12 if D == 0.02 else 6) * (nx / 10) ** 2))
    dt, dx = 1.0 / nt, 1.0 / nx
    N = 2 * nx
    x = np.arange(N) * dx
    X, Y = np.meshgrid(x, x, indexing="xy")

    def exact(t):
        return np.exp(-2 * D * np.pi ** 2 * t) * np.cos(np.pi * (X + Y) - 2 * np.pi * t)

    # beta from alpha = A_22 dt beta c_s^2 (Eq. (M-NCDE-6), A_10 = -1), lambda_bar = 1 (EDF of Example 2)
    prob = P.problem_lcde("D2Q9", 3, [N, N], dt, [dx, dx], [[D, 0], [0, D]], [1.0, 1.0], a, ah)
    out = orc.run(prob, [exact(0.0)], [exact(-dt)], nsteps=nt)[0][0]
    ex = exact(nt * dt)
    return np.abs(out - ex).sum() / np.abs(ex).sum()


def test_example2_second_order_convergence():
    # Table 2: all three cases converge at (at least) second order in dx with dt ~ dx^2.  The printed
    # absolute GRE values are not reproduced under any reading tried (parity unpinned for the absolute
    # values); the order is pinned.  Case 1 (SRT, tau = 1, with the u u term of the printed EDF) comes
    # out at order 4 in dx (order 2 in dt) here, above the printed order 2.
    for case in (1, 2, 3):
        g = [_ex2_gre(case, nx) for nx in (20, 40, 80)]
        orders = [np.log2(g[i] / g[i + 1]) for i in range(2)]
        assert all(o > 1.8 for o in orders), (case, g, orders)
        if case > 1:
            assert all(o < 2.4 for o in orders), (case, g, orders)


def test_table3_instability_qualitative():
    # Table 3 (Example 2 Case 1, D = 0.01): the two coarse rows (u^2/c_s^2 = 50/3, 25/6) violate the
    # bound of Theorem 1 and their amplification factor exceeds 1; the two fine rows (25/24, 25/96)
    # satisfy it.  The coarsest run is garbage (GRE > 1), the finest is accurate.
    rows = [(10, 6, True), (20, 24, True), (40, 96, False), (80, 384, False)]
    for nx, nt, unstable in rows:
        dt, dx, N = 1.0 / nt, 1.0 / nx, 2 * nx
        prob = P.problem_lcde("D2Q9", 2, [N, N], dt, [dx, dx], [[0.01, 0], [0, 0.01]], [1.0, 1.0],
                              (1.0, 0.0, 0.0))
        lam = F.max_amplification(prob)
        t1 = F.theorem1(prob)
        assert (lam > 1 + 1e-12) == unstable
        assert (t1["a"] and t1["b"] and t1["c"]) == (not unstable)
    assert _ex2_gre(1, 10, D=0.01) > 1.0
    assert _ex2_gre(1, 80, D=0.01) < 0.01


# ----------------------------------------------------------------------------- stability

def test_theorem1_sufficient_on_d2q9_config1():
    # Config-1 D2Q9 EDF has negative ubar^+ on the diagonals (violating Theorem 1(a)), yet max|lambda| = 1:
    # Theorem 1 is sufficient, not necessary, on D2Q9.
    K = [[0.02, 0.005], [0.005, 0.01]]
    prob = P.problem_lcde("D2Q9", 2, [64, 64], 1.0, [1, 1], K, [0.1, 0.05], P.two_level_from_a0(0.0))
    t1 = F.theorem1(prob)
    assert not t1["a"]
    assert F.max_amplification(prob) <= 1.0 + 1e-12


def test_theorem1_b_equivalence():
    # Eq. (Tcond-2)/(Tcond-3): condition (b) <=> a_0 + ubar_0^+ (1 - a_0) >= 0
    for a0 in np.linspace(-1.5, 0.9, 13):
        prob = P.problem_lcde("D2Q5", 2, [8, 8], 1.0, [1, 1], [[0.05, 0], [0, 0.04]], [0.05, 0.02],
                              P.two_level_from_a0(float(a0)))
        t = F.theorem1(prob)
        assert t["b"] == t["b_alt"]


def test_linear_edf_closed_form_bound():
    # Eq. (LMMFD-2-3): with the linear EDF on rD2Q5 (isotropic c_s^2), the scheme is stable iff
    # |u|^2 <= 2 alpha/dt <= c_s^2 / (1 - omega_0); checked against max |lambda| on a 256x256 grid
    # (the bound is over the continuum of wave numbers; cases keep a margin the grid resolves).
    cs2 = 0.25
    for alpha, ux in [(0.1, 0.3), (0.1, 0.5), (0.13, 0.3), (0.12, 0.45), (0.1, 0.46), (0.26, 0.3), (0.24, 0.3)]:
        r = 2 * alpha / cs2
        a = ((r + 1) / 2, 1 - r, (r - 1) / 2)
        prob = orc.Problem(lattice="D2Q5", pde="LCDE", levels=2, n=[32, 32], c=[1, 1],
                           d0=[cs2, cs2], a=a, u=[ux, 0.0, 0])
        w0 = 1 - 2 * cs2
        predicted = (ux ** 2 <= 2 * alpha + 1e-15) and (2 * alpha <= cs2 / (1 - w0) + 1e-15)
        assert predicted == (F.max_amplification(prob, (256, 256)) <= 1 + 1e-12), (alpha, ux)


def test_stability_growth_just_outside_bound():
    # Just outside the bound the oracle's growth over n steps equals |lambda_max|^n; just inside,
    # nothing grows.
    cs2 = 0.25
    for alpha, expect_growth in [(0.255, True), (0.245, False)]:
        r = 2 * alpha / cs2
        a = ((r + 1) / 2, 1 - r, (r - 1) / 2)
        prob = orc.Problem(lattice="D2Q5", pde="LCDE", levels=2, n=[16, 16], c=[1, 1],
                           d0=[cs2, cs2], a=a, u=[0.05, 0.0, 0])
        lam = F.two_level_lambda(prob, (16, 16))
        i = np.unravel_index(np.argmax(np.abs(lam)), lam.shape)
        th = F.thetas((16, 16))
        mode = np.cos(th[0][i] * np.arange(16)[:, None] + th[1][i] * np.arange(16)[None, :])
        n = 60
        out = orc.run(prob, [mode], nsteps=n)[0][0]
        growth = np.sqrt((out ** 2).sum() / (mode ** 2).sum())
        lmax = np.abs(lam).max()
        if expect_growth:
            assert lmax > 1
            assert abs(growth / lmax ** n - 1) < 1e-8
        else:
            assert lmax <= 1 + 1e-12 and growth <= 1 + 1e-12


def _three_level_case(kappa, shape=(16, 16)):
    # Eq. (X) with a_0 = 0, A_10 = A_11 = -1, A_21 = 1/4, A_22 = 1/2: the printed set
    # a = (7/8, 0, 1/8), ahat = (1/8, 0, -1/8) of Examples 1-2; isotropic diffusion kappa
    a, ah = P.solve_three_level(0.0, -1.0, -1.0, 0.25, 0.5)
    return P.problem_lcde("D2Q9", 3, list(shape[::-1]), 1.0, [1.0, 1.0], [[kappa, 0.0], [0.0, kappa]], [0.05, 0.03],
                          a, ah)


def _three_level_rmax(prob, shape=(16, 16)):
    l1, l2, _, _ = F.three_level_roots(prob, shape)
    lam = np.where(np.abs(l1) >= np.abs(l2), l1, l2)
    lam[0, 0] = 0.0          # theta = 0: conserved mass, root exactly 1
    return lam


def test_three_level_growth_just_inside_and_outside_theorem3():
    # Theorem 3 (Eq. (3-level)): on a 16^2 grid, bisect the diffusion number at which the largest
    # root of lambda^2 - p_1 lambda - p_0 reaches 1, take kappa* (1 -+ 1e-3), and run the oracle's
    # three-level scheme from an eigen-start of the fastest mode (phi^{-1} = phi^0 / lambda in that
    # mode).  Outside: Theorem 3's inequality fails and the oracle grows as |lambda_max|^n (1e-8);
    # inside: it holds and nothing grows.
    shape = (16, 16)
    lo, hi = 0.01, 1.0
    assert np.abs(_three_level_rmax(_three_level_case(lo))).max() <= 1 and \
        np.abs(_three_level_rmax(_three_level_case(hi))).max() > 1
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if np.abs(_three_level_rmax(_three_level_case(mid))).max() > 1:
            hi = mid
        else:
            lo = mid
    kstar = 0.5 * (lo + hi)
    th = F.thetas(shape)
    y, x = np.arange(shape[0])[:, None], np.arange(shape[1])[None, :]
    for kappa, outside in [(kstar * (1 + 1e-3), True), (kstar * (1 - 1e-3), False)]:
        prob = _three_level_case(kappa)
        lam = _three_level_rmax(prob)
        # a mode whose real field is a single eigenmode: +-theta distinct, or theta = -theta
        # (components 0 or pi) with a real root
        selfconj = np.isclose(np.abs(np.sin(th[0])) + np.abs(np.sin(th[1])), 0.0)
        real = np.abs(lam.imag) <= 1e-12 * np.abs(lam)
        mag = np.where(selfconj & ~real, 0.0, np.abs(lam))
        i = np.unravel_index(np.argmax(mag), mag.shape)
        li = lam[i] if not selfconj[i] else complex(lam[i].real, 0.0)
        phase = th[0][i] * y + th[1][i] * x
        phi0 = np.cos(phase)
        phim1 = np.real(np.exp(1j * phase) / li)
        n = 80
        out, _ = orc.run(prob, [phi0], [phim1], nsteps=n)
        growth = np.sqrt((out[0] ** 2).sum() / (phi0 ** 2).sum())
        if outside:
            assert not F.theorem3_holds(prob, shape)
            assert abs(li) > 1 + 1e-6
            assert abs(growth / abs(li) ** n - 1) < 1e-8, (growth, abs(li) ** n)
        else:
            mask = np.ones(shape, dtype=bool)
            mask[0, 0] = False
            p1 = F.symbol(prob, prob.a, shape)
            p0 = F.symbol(prob, prob.ahat, shape)
            sc = np.abs(p1 + np.conj(p1) * p0)[mask] <= (1.0 - np.abs(p0) ** 2)[mask] + 1e-12
            assert sc.all()
            assert abs(li) <= 1 + 1e-12 and growth <= 1 + 1e-12
            assert abs(growth / abs(li) ** n - 1) < 1e-8


def test_theorem3_matches_roots():
    # Theorem 3 (Schur-Cohn) agrees with the roots of lambda^2 - p_1 lambda - p_0 on random three-level
    # schemes away from the boundary.  The theta = 0 mode (conserved mass, root exactly 1) is excluded.
    agree = 0
    total = 0
    unstable = 0
    for _ in range(60):
        a0 = RNG.uniform(-0.5, 0.5)
        A21 = RNG.uniform(-0.6, 0.6)
        A22 = RNG.uniform(0.2, 3.0)
        a, ah = P.solve_three_level(a0, -1.0, -1.0, A21, A22)
        prob = P.problem_lcde("D2Q9", 3, [16, 16], 1.0, [1, 1], [[0.02, 0], [0, 0.02]], [0.05, 0.03], a, ah)
        l1, l2, p1, p0 = F.three_level_roots(prob, (16, 16))
        mask = np.ones(l1.shape, dtype=bool)
        mask[0, 0] = False
        rmax = max(np.abs(l1[mask]).max(), np.abs(l2[mask]).max())
        if abs(rmax - 1) < 1e-6:
            continue
        total += 1
        unstable += rmax > 1
        sc = np.all(np.abs(p1 + np.conj(p1) * p0)[mask] <= (1.0 - np.abs(p0) ** 2)[mask] + 1e-12)
        agree += (rmax <= 1) == bool(sc)
    assert total > 30 and 5 < unstable < total - 5 and agree == total


def test_theorem2_theta_scheme():
    # Eq. (Tcond1-3) holds identically, and theta <= 1/2 is unconditionally stable when (a) holds
    # (theta weights the explicit level in Eq. (GCN)).
    prob = P.problem_lcde("D2Q5", 2, [16, 16], 1.0, [1, 1], [[0.3, 0], [0, 0.25]], [0.2, 0.1],
                          P.two_level_from_a0(-2.0))
    A, B = F.theta_AB(prob, (16, 16))
    for th in (0.0, 0.25, 0.5, 0.75, 1.0):
        lam = F.theta_lambda(prob, th, (16, 16))
        lhs = np.abs(lam) ** 2 - 1
        rhs = (2 * A + (2 * th - 1) * (A * A + B * B)) / np.abs(1 - (1 - th) * (A + 1j * B)) ** 2
        assert np.allclose(lhs, rhs, atol=1e-12)
        if th <= 0.5:
            assert np.abs(lam).max() <= 1 + 1e-12
    # the explicit end (theta = 1) of this heavily diffusive scheme is unstable
    assert np.abs(F.theta_lambda(prob, 1.0, (16, 16))).max() > 1


# ----------------------------------------------------------------------------- Taylor-Green (NSE)

def test_taylor_green_decay():
    # He-Luo NSE with a_{-1} = abar_{-1} = 1 (LBGK tau = 1): nu = -(Abar_22/Abar_10) dt c_s^2 = 1/6
    # (Eq. (M-NSEs-4c)).  The velocity field follows the analytic Taylor-Green decay with a second-order
    # error under diffusive refinement (N doubled, steps x4, u0 halved: fixed Reynolds number).
    nu = P.nse_viscosity(2, (1.0, 0.0, 0.0), (0, 0, 0), 1.0, 1 / 3)
    assert abs(nu - 1 / 6) < 1e-15
    errs = []
    for N in (16, 32):
        u0 = 0.01 * 16 / N
        nsteps = int(200 * (N / 32) ** 2)
        rho, u, v = inputs.taylor_green_2d(N, N, u0, nu, 0.0)
        prob = P.problem_nse("D2Q9", 2, [N, N], 1.0, [1, 1], (1.0, 0, 0), (1.0, 0, 0))
        out, _ = orc.run(prob, [rho, u, v], nsteps=nsteps)
        _, ue, ve = inputs.taylor_green_2d(N, N, u0, nu, float(nsteps))
        errs.append(np.sqrt(((out[1] - ue) ** 2 + (out[2] - ve) ** 2).sum() / (ue ** 2 + ve ** 2).sum()))
    assert errs[1] < 0.01
    assert 1.9 < np.log2(errs[0] / errs[1]) < 2.1
