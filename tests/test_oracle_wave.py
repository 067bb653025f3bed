"""Pins of the wave-equation scheme (Sec. III.C case (4), Eq. (ME-NCDE-W-1), Example 3) in the
oracle (CPU only).  The oracle evaluates it as the three-level linear-EDF scheme of
Eq. (TforMMFD-0) with u = 0; params.problem_lwe maps the wave tensor K = alpha D0 onto the EDF.

- Example 3 Case 1 (D2Q5, beta = 1, gamma = 3/8) is the textbook five-point explicit scheme
      phi^{n+1} = 2 phi^n - phi^{n-1} + alpha (dt/dx)^2 (sum of the four neighbours - 4 phi^n).
- The scheme family has A_10 = A_11 = A_21 = 0, A_20 = -1 and A_22 = gamma (in rationals).
- Cases 1-3 of Example 3 converge at second order to an exact periodic standing wave (the
  printed Example 3 is not periodic; its boundary treatment is not stated).
- Stability: with p_0 = -1 and a real p_1 the roots of lambda^2 - p_1 lambda + 1 lie on the unit
  circle iff |p_1| <= 2; Theorem 3's inequality degenerates to 0 <= 0 here and holds for
  unstable schemes too.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import fourier as F
from oracle import oracle as orc
from oracle import params as P

CASES = {1: ("D2Q5", 1.0, 3 / 8), 2: ("D2Q9", 1.0, 3 / 8), 3: ("D2Q9", 3 / 4, 1 / 2)}


def example3_problem(case, nx, alpha=0.5, dt_over_dx=0.5):
    """Example 3's parameters on a periodic [0, 1)^2 grid of nx^2 nodes: dt = dx / 2,
    c_s^2 = c^2 / 3 (d_0 = 1/3), K = alpha I; beta fixes gamma through alpha = gamma beta c_s^2."""
    lat, beta, gamma = CASES[case]
    dx = 1.0 / nx
    dt = dt_over_dx * dx
    a, ah = P.wave_coefficients(gamma)
    return P.problem_lwe(lat, [nx, nx], dt, [dx, dx], alpha * np.eye(2), a, ah), dx, dt


def test_example3_parameters_are_consistent():
    # alpha = gamma beta c_s^2 with c_s^2 = c^2 / 3 (the printed cases): d_0 = 1/3 on D2Q5, and
    # on D2Q9 the EDF's C = c_s^2 (beta - 1) I
    for case in (1, 2, 3):
        prob, dx, dt = example3_problem(case, 10)
        lat, beta, gamma = CASES[case]
        c = dx / dt
        if lat == "D2Q5":
            assert np.allclose(prob.d0[:2], [1 / 3, 1 / 3], rtol=1e-14)
        else:
            C = np.asarray(prob.Cmat).reshape(3, 3)[:2, :2]
            assert np.allclose(C, c * c / 3 * (beta - 1) * np.eye(2), atol=1e-14)


def test_case1_is_the_textbook_leapfrog():
    prob, dx, dt = example3_problem(1, 12)
    rng = np.random.default_rng(51)
    p0, pm = rng.standard_normal((12, 12)), rng.standard_normal((12, 12))
    out = orc.step(prob, [p0], [pm])[0]
    lap = np.roll(p0, 1, 0) + np.roll(p0, -1, 0) + np.roll(p0, 1, 1) + np.roll(p0, -1, 1) - 4 * p0
    ref = 2 * p0 - pm + 0.5 * (dt / dx) ** 2 * lap
    assert np.abs(out - ref).max() < 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("gamma", [Fraction(3, 8), Fraction(1, 2), Fraction(7, 10)])
def test_wave_scheme_moments(gamma):
    a, ah = P.wave_coefficients(gamma)
    A = P.three_level_moments(a, ah)
    assert A[(0, 0)] == 1 and A[(2, 0)] == -1 and A[(2, 2)] == gamma
    assert A[(1, 0)] == 0 and A[(1, 1)] == 0 and A[(2, 1)] == 0


def standing_wave_gre(case, nx):
    # phi = cos(2 pi (x + y)) cos(omega t), omega^2 = alpha |k|^2 = 0.5 * 8 pi^2
    prob, dx, dt = example3_problem(case, nx)
    x = np.arange(nx) * dx
    X, Y = np.meshgrid(x, x, indexing="xy")
    om = 2 * np.pi
    exact = lambda t: np.cos(2 * np.pi * (X + Y)) * np.cos(om * t)
    steps = int(round(1.0 / dt))
    out, _ = orc.run(prob, [exact(0.0)], [exact(-dt)], nsteps=steps)
    ref = exact(steps * dt)
    return float(np.abs(out[0] - ref).sum() / np.abs(ref).sum())


@pytest.mark.parametrize("case", [1, 2, 3])
def test_standing_wave_second_order(case):
    gre = [standing_wave_gre(case, nx) for nx in (10, 20, 40)]
    orders = [np.log2(gre[i] / gre[i + 1]) for i in range(2)]
    assert all(o >= 1.8 for o in orders), (gre, orders)


def test_wave_stability_is_p1_within_2():
    rng = np.random.default_rng(52)
    agree = total = unstable = degenerate = 0
    shape = (16, 16)
    for _ in range(80):
        lat = ("D2Q5", "D2Q9")[rng.integers(2)]
        gamma = rng.uniform(0.2, 1.6)
        alpha = rng.uniform(0.1, 8.0)
        a, ah = P.wave_coefficients(gamma)
        try:
            prob = P.problem_lwe(lat, [16, 16], 0.5, [1.0, 1.0], alpha * np.eye(2), a, ah)
        except Exception:
            continue
        if lat == "D2Q5" and sum(prob.d0[:2]) >= 1:
            continue
        l1, l2, p1, p0 = F.three_level_roots(prob, shape)
        assert np.abs(p1.imag).max() < 1e-13 and np.abs(p0 + 1).max() < 1e-13
        # theta = 0: p_1 = 2, the double root 1 of the constant mode, on the boundary
        m = np.ones(shape, dtype=bool)
        m[0, 0] = False
        l1, l2, p1, p0 = l1[m], l2[m], p1[m], p0[m]
        rmax = max(np.abs(l1).max(), np.abs(l2).max())
        q = np.abs(p1.real).max()
        if abs(q - 2) < 1e-9:
            continue
        total += 1
        unstable += rmax > 1 + 1e-9
        agree += (rmax <= 1 + 1e-9) == (q <= 2)
        # Theorem 3's inequality: |p1 + conj(p1) p0| <= 1 - |p0|^2 reads 0 <= 0 here
        if rmax > 1 + 1e-9 and np.all(np.abs(p1 + np.conj(p1) * p0) <= 1 - np.abs(p0) ** 2 + 1e-12):
            degenerate += 1
    assert total > 40 and 5 < unstable < total - 5 and agree == total and degenerate == unstable


# ----------------------------------------------------------------------------- Table 4

def _table4():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "example3_table4.json")) as fh:
        return json.load(fh)


def test_example3_table4_case1_reproduced():
    # Example 3 as printed (Dirichlet values of exp(x + y + t), the paper's start-up, GRE over the
    # interior nodes at t = 1): Case 1 (D2Q5) gives the printed GRE of Table 4 to its three digits
    import example3_dirichlet as E3
    t4 = _table4()
    for nx, printed in zip(t4["nx"], t4["gre"]["case1"]):
        prob, _, _, _ = E3.problem(1, nx)
        got = E3.interior_gre(1, nx, lambda cur, prev: orc.step(prob, [cur], [prev])[0])
        assert float("%.2e" % got) == float(printed), (nx, got, printed)    # equal to the printed digits


def test_example3_table4_cases2_3_order():
    # Cases 2-3 (D2Q9) converge at second order as Table 4 says, but their absolute GRE comes out
    # 5-10x below the printed values under the same procedure (parity unpinned, see the readings)
    import example3_dirichlet as E3
    t4 = _table4()
    for case in (2, 3):
        gres = []
        for nx in t4["nx"]:
            prob, _, _, _ = E3.problem(case, nx)
            gres.append(E3.interior_gre(case, nx, lambda cur, prev: orc.step(prob, [cur], [prev])[0]))
        assert all(1.9 <= o <= 2.4 for o in E3.orders(gres)), (case, gres)
        printed = [float(v) for v in t4["gre"][f"case{case}"]]
        assert all(g < p / 4 for g, p in zip(gres, printed)), (case, gres, printed)
