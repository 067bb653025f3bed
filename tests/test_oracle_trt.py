"""Pins of the TRT special case of Sec. III.C (case (2), s+ + s- = 2) and of Corollary 1 (CPU only).

- The oracle's independent TRT lattice-Boltzmann code (explicit populations: collide with the
  even / odd rates s+ = 2 - s- and s-, then stream) must reduce to the pinned LBGK tau = 1 code
  at s- = 1.
- Started from equilibrium populations, its moments follow the three-level MMFD with the
  coefficients the paper lists for case (2), a = (a_{-1}, a_0, a_1) = (1, 0, 1 - s-),
  ahat = (0, -(1 - s-), 0), once the first level is one LBGK tau = 1 step.  For the NSE
  momentum the same elimination gives abar = (1, 0, -(1 - s-)), abarhat = (0, 1 - s-, 0)
  (the paper lists only the scalar set); the momentum check fails with abar = a.
- With these sets the moments of Eq. (M-NCDE-6) / (M-NSEs-4c) give the textbook TRT transport
  coefficients: the odd rate sets the scalar diffusivity c_s^2 (1/s- - 1/2) dt, the even rate
  the viscosity c_s^2 (1/s+ - 1/2) dt.
- Corollary 1: the TRT scheme is stable iff A^2 + B^2 <= 1 at every wave number, with
  A = sum_j ubar_j^+ cos(xi_j), B = sum_j ubar_j^- sin(xi_j).  Checked against the roots of
  lambda^2 - p_1 lambda - p_0, and the growth of the independent LB code against the largest root.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import fourier as F
from oracle import oracle as orc
from oracle import params as P


def trt_sets(s):
    w = 1.0 - s
    return (1.0, 0.0, w), (0.0, -w, 0.0), (1.0, 0.0, -w), (0.0, w, 0.0)


def _problem(lat, pde, n, s, momentum_like_scalar=False):
    a, ah, ab, abh = trt_sets(s)
    if momentum_like_scalar:
        ab, abh = a, ah
    dim = 2 if lat.startswith("D2") else 3
    dt, dx = 0.8, [1.0, 1.1, 0.9][:dim]
    # diffusivities in proportion to the TRT's natural one, c_s^2 (1/s- - 1/2) dt, so that the
    # EDF's second moment stays near c_s^2 phi and the runs stay stable for s- near 2
    g = min(1.0, 2.0 / s - 1.0)
    if pde == "LCDE":
        K = np.diag([0.05, 0.04, 0.06][:dim])
        if lat in ("D2Q9", "D3Q19"):
            K = K + 0.006 * (1 - np.eye(dim))
        return P.problem_lcde(lat, 3, n, dt, dx, g * K, [0.08, -0.05, 0.04][:dim], a, ah)
    if pde == "NCDE":
        flux = [[0, 0.05, 0.1, 0], [0, -0.03, 0.1, 0], [0, 0, 0.06, 0.02]][:dim]
        return P.problem_ncde(lat, 3, n, dt, dx, flux, [0.15 * g, 0, 0.05 * g], a, ah)
    return P.problem_nse(lat, 3, n, dt, dx, a, ab, ah, abh)


def _level(prob, rng):
    if prob.pde == "NSE":
        return [1.0 + 0.01 * rng.standard_normal(prob.shape)] + \
               [0.03 * rng.standard_normal(prob.shape) for _ in range(prob.dim)]
    return [0.5 + 0.2 * rng.standard_normal(prob.shape)]


def _rel(x, y):
    # relative to max(1, |field|): the populations, and their rounding, are O(rho) = O(1) even
    # where a moment (the NSE velocity) is small
    return max(float(np.abs(a - b).max() / max(1.0, np.abs(b).max())) for a, b in zip(x, y))


COMBOS = [("D2Q9", "LCDE", [7, 6]), ("D2Q5", "LCDE", [9, 5]), ("D2Q9", "NCDE", [6, 7]),
          ("D2Q9", "NSE", [7, 6]), ("D3Q7", "LCDE", [5, 4, 3]), ("D3Q19", "NCDE", [4, 5, 3]),
          ("D3Q19", "NSE", [5, 4, 3])]


@pytest.mark.parametrize("lat,pde,n", COMBOS)
def test_trt_code_at_unit_rates_is_lbgk(lat, pde, n):
    rng = np.random.default_rng(31)
    prob = _problem(lat, pde, n, 1.0)
    L0 = _level(prob, rng)
    assert _rel(orc.trt_run(prob, L0, 1.0, 5), orc.lbgk_tau1_run(prob, L0, 5)) < 1e-14


@pytest.mark.parametrize("s", [0.45, 1.3, 1.85])
@pytest.mark.parametrize("lat,pde,n", COMBOS)
def test_trt_lb_is_the_three_level_mmfd(lat, pde, n, s):
    rng = np.random.default_rng(32)
    prob = _problem(lat, pde, n, s)
    L0 = _level(prob, rng)
    steps = 8
    lb = orc.trt_run(prob, L0, s, steps)
    L1 = orc.lbgk_tau1_run(prob, L0, 1)
    assert all(np.abs(f).max() < 10 for f in lb)
    for form in ("central", "mmfd"):
        mm, _ = orc.run(prob, L1, L0, nsteps=steps - 1, form=form)
        assert _rel(mm, lb) < 1e-13, form
    if pde == "NSE":
        # the scalar set on the momentum is not the TRT scheme
        wrong = _problem(lat, pde, n, s, momentum_like_scalar=True)
        mm, _ = orc.run(wrong, L1, L0, nsteps=steps - 1)
        assert max(float(np.abs(mm[i] - lb[i]).max()) for i in range(1, prob.nf)) > 1e-6


@pytest.mark.parametrize("s", [Fraction(1, 2), Fraction(6, 5), Fraction(19, 10)])
def test_trt_transport_coefficients(s):
    w = 1 - s
    a, ah = (Fraction(1), Fraction(0), w), (Fraction(0), -w, Fraction(0))
    ab, abh = (Fraction(1), Fraction(0), -w), (Fraction(0), w, Fraction(0))
    A = P.three_level_moments(a, ah)
    assert A[(0, 0)] == 1 and A[(2, 0)] == -A[(1, 0)] / 2 - 1
    # scalar: alpha = -(A_22 / A_10) dt c_s^2 (Eq. (M-NCDE-6)) = c_s^2 (1/s- - 1/2) dt
    assert -A[(2, 2)] / A[(1, 0)] == 1 / s - Fraction(1, 2)
    Ab = P.three_level_moments(ab, abh)
    assert Ab[(0, 0)] == 1
    # momentum: nu = -(Abar_22 / Abar_10) dt c_s^2 (Eq. (M-NSEs-4c)) = c_s^2 (1/s+ - 1/2) dt
    s_plus = 2 - s
    assert -Ab[(2, 2)] / Ab[(1, 0)] == 1 / s_plus - Fraction(1, 2)
    assert P.nse_viscosity(3, tuple(map(float, ab)), tuple(map(float, abh)), 1.0, 1.0) == \
        pytest.approx(float(1 / s_plus - Fraction(1, 2)), rel=1e-15)


def _corollary1(prob, shape):
    up, um, E = F.ubar_split(prob)
    th = F.thetas(shape)
    dim = len(shape)
    A = np.zeros(shape)
    B = np.zeros(shape)
    for j in range(E.shape[0]):
        xi = sum(th[i] * E[j][dim - 1 - i] for i in range(dim))
        A += up[j] * np.cos(xi)
        B += um[j] * np.sin(xi)
    return A * A + B * B


def _linear_trt_problem(lat, s, cs2, u, n):
    a, ah, _, _ = trt_sets(s)
    return orc.Problem(lattice=lat, pde="LCDE", levels=3, n=n, c=[1, 1], d0=[cs2, cs2],
                       a=a, ahat=ah, u=[u[0], u[1], 0])


def test_corollary1_matches_roots():
    rng = np.random.default_rng(33)
    shape = (24, 24)
    agree = total = unstable = 0
    for _ in range(80):
        lat = ["D2Q5", "D2Q9"][rng.integers(2)]
        s = rng.uniform(0.15, 1.9)
        cs2 = rng.uniform(0.1, 0.45) if lat == "D2Q5" else 1.0 / 3.0
        ang = rng.uniform(0, 2 * np.pi)
        mag = rng.uniform(0.2, 1.8) * np.sqrt(cs2)
        prob = _linear_trt_problem(lat, s, cs2, (mag * np.cos(ang), mag * np.sin(ang)), [24, 24])
        l1, l2, _, _ = F.three_level_roots(prob, shape)
        # the theta = 0 mode (conserved mass: root 1, A^2 + B^2 = 1) sits on the boundary
        mask = np.ones(shape, dtype=bool)
        mask[0, 0] = False
        rmax = max(np.abs(l1[mask]).max(), np.abs(l2[mask]).max())
        q = _corollary1(prob, shape)[mask].max()
        if abs(rmax - 1) < 1e-9 or abs(q - 1) < 1e-9:
            continue
        total += 1
        unstable += rmax > 1
        agree += (rmax <= 1) == (q <= 1)
    assert total > 50 and 5 < unstable < total - 5 and agree == total


def test_corollary1_growth_of_the_lb_code():
    # an unstable TRT run grows by the largest root per step; a stable one stays bounded
    n = 16
    for s, mag, expect_growth in [(1.2, 1.4, True), (1.2, 0.6, False), (0.3, 1.3, True)]:
        cs2 = 0.25
        prob = _linear_trt_problem("D2Q5", s, cs2, (mag * np.sqrt(cs2), 0.0), [n, n])
        l1, l2, _, _ = F.three_level_roots(prob, (n, n))
        r = np.maximum(np.abs(l1), np.abs(l2))
        i = np.unravel_index(np.argmax(r), r.shape)
        th = F.thetas((n, n))
        mode = np.cos(th[0][i] * np.arange(n)[:, None] + th[1][i] * np.arange(n)[None, :])
        q = _corollary1(prob, (n, n)).max()
        out_a = orc.trt_run(prob, [mode], s, 160)[0]
        out_b = orc.trt_run(prob, [mode], s, 200)[0]
        norm = lambda x: float(np.sqrt((x ** 2).sum()))
        if expect_growth:
            assert q > 1 and r.max() > 1
            assert abs((norm(out_b) / norm(out_a)) ** (1 / 40) / r.max() - 1) < 1e-4
        else:
            assert q <= 1 + 1e-12 and r.max() <= 1 + 1e-12
            assert norm(out_b) <= 2 * norm(mode)
