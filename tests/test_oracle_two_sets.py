"""Pins of the oracle's multiple-parameter-set scheme, Eq. (2-2-1b), and of the TRT version of
the MesoFD scheme, Eq. (2-1b) (CPU only).

- The two forms are different algebra -- Eq. (2-1b) builds f_j from the even and odd parts of
  f^eq at shifted nodes and then takes moments; Eq. (2-2-1b) applies second and first central
  differences to the even and odd parts -- and must agree when the zeroth-order set of
  Eq. (2-2-1b) is the even set (momentum: the odd set).
- Equal sets reduce Eq. (2-2-1b) to the one-set scheme Eq. (2-2-1), bit for bit.
- For the linear CDE the update is a Fourier multiplier.  Written out independently here:
      lambda(theta) = sum_k a_k + sum_j [ d2^+ ubar_j^+ (cos(theta.e_j) - 1) + i d1^- ubar_j^- sin(theta.e_j) ]
  (d2^+ = d2_1 + d2_{-1}, d1^- = d1_1 - d1_{-1}, ubar^+- the even/odd parts of f^eq / phi),
  so the oracle's steps must equal the exact discrete solution; swapping the even and odd
  sets must not.
- Periodic differences sum to zero, so sum(phi) scales by sum_k a_k whatever d2, d1 are.
"""
import numpy as np
import pytest

from oracle import fourier as F
from oracle import oracle as orc
from oracle import params as P

TWO = (0.95, 0.1, -0.05)
THREE_A, THREE_AH = (7 / 8, 0.0, 1 / 8), (1 / 8, 0.0, -1 / 8)


def _base(lat, pde, levels, n):
    dim = 2 if lat.startswith("D2") else 3
    dt, dx = 0.8, [1.0, 1.1, 0.9][:dim]
    a = TWO if levels == 2 else THREE_A
    ah = (0.0, 0.0, 0.0) if levels == 2 else THREE_AH
    if pde == "LCDE":
        K = np.diag([0.05, 0.04, 0.06][:dim])
        if lat in ("D2Q9", "D3Q19"):
            K = K + 0.006 * (1 - np.eye(dim))
        return P.problem_lcde(lat, levels, n, dt, dx, K, [0.08, -0.05, 0.04][:dim], a, ah)
    if pde == "NCDE":
        flux = [[0, 0.05, 0.1, 0], [0, -0.03, 0.1, 0], [0, 0, 0.06, 0.02]][:dim]
        return P.problem_ncde(lat, levels, n, dt, dx, flux, [0.15, 0, 0.05], a, ah)
    ab = (0.9, 0.2, -0.1) if levels == 2 else (0.8, 0.0, 0.2)
    abh = (0.0, 0.0, 0.0) if levels == 2 else (0.1, 0.0, -0.1)
    return P.problem_nse(lat, levels, n, dt, dx, a, ab, ah, abh)


def _level(prob, rng):
    if prob.pde == "NSE":
        return [1.0 + 0.01 * rng.standard_normal(prob.shape)] + \
               [0.03 * rng.standard_normal(prob.shape) for _ in range(prob.dim)]
    return [0.5 + 0.2 * rng.standard_normal(prob.shape)]


def _sets(rng):
    pert = lambda: tuple(0.05 * rng.standard_normal(3))
    add = lambda t, d: tuple(x + y for x, y in zip(t, d))
    return {"d2": (add(TWO, pert()), add(THREE_AH, pert())), "d1": (add(TWO, pert()), add(THREE_AH, pert())),
            "bar_d2": (add(TWO, pert()), add(THREE_AH, pert())), "bar_d1": (add(TWO, pert()), add(THREE_AH, pert()))}


COMBOS = [("D2Q5", "LCDE", 2), ("D2Q9", "LCDE", 3), ("D2Q9", "NCDE", 2), ("D2Q9", "NCDE", 3),
          ("D2Q9", "NSE", 2), ("D2Q9", "NSE", 3), ("D3Q7", "LCDE", 2), ("D3Q19", "NSE", 2),
          ("D3Q19", "NCDE", 3)]


def _rel(x, y):
    return max(float(np.abs(a - b).max() / np.abs(b).max()) for a, b in zip(x, y))


@pytest.mark.parametrize("lat,pde,levels", COMBOS)
def test_trt_mesofd_equals_multi_set_central(lat, pde, levels):
    rng = np.random.default_rng(11)
    n = [7, 6] if lat.startswith("D2") else [5, 4, 3]
    prob = _base(lat, pde, levels, n)
    sets = _sets(rng)
    prob.sets = sets
    # Eq. (2-1b) has no separate zeroth-order set: it is the even set (momentum: the odd set)
    prob.a, prob.ahat = sets["d2"][0], (sets["d2"][1] if levels == 3 else (0.0, 0.0, 0.0))
    prob.abar, prob.abarhat = sets["bar_d2"][0], (sets["bar_d2"][1] if levels == 3 else (0.0, 0.0, 0.0))
    L0 = _level(prob, rng)
    L1 = _level(prob, rng) if levels == 3 else None
    meso = orc.step(prob, L0, L1, form="mesofd_trt")
    cent = orc.step(prob, L0, L1, form="central")
    assert _rel(meso, cent) < 1e-13


@pytest.mark.parametrize("lat,pde,levels", COMBOS)
def test_equal_sets_reduce_to_one_set(lat, pde, levels):
    rng = np.random.default_rng(12)
    n = [7, 6] if lat.startswith("D2") else [5, 4, 3]
    prob = _base(lat, pde, levels, n)
    L0 = _level(prob, rng)
    L1 = _level(prob, rng) if levels == 3 else None
    one = orc.step(prob, L0, L1, form="central")
    direct = orc.step(prob, L0, L1, form="mmfd")
    prob.sets = {"d2": (prob.a, prob.ahat), "d1": (prob.a, prob.ahat),
                 "bar_d2": (prob.abar, prob.abarhat), "bar_d1": (prob.abar, prob.abarhat)}
    two = orc.step(prob, L0, L1, form="central")
    assert all(np.array_equal(x, y) for x, y in zip(two, one))
    assert _rel(two, direct) < 1e-13


def _symbol_two_sets(prob, a, d2, d1, shape):
    up, um, E = F.ubar_split(prob)
    th = F.thetas(shape)
    dim = len(shape)
    lam = np.full(shape, complex(sum(a)))
    dp, dm = d2[2] + d2[0], d1[2] - d1[0]
    for j in range(E.shape[0]):
        ph = sum(th[i] * E[j][dim - 1 - i] for i in range(dim))
        lam = lam + dp * up[j] * (np.cos(ph) - 1.0) + 1j * dm * um[j] * np.sin(ph)
    return lam


@pytest.mark.parametrize("lat", ["D2Q9", "D2Q5", "D3Q7"])
def test_two_set_lcde_is_its_fourier_multiplier(lat):
    rng = np.random.default_rng(13)
    n = [16, 12] if lat.startswith("D2") else [8, 6, 5]
    prob = _base(lat, "LCDE", 2, n)
    d2, d1 = (0.97, 0.05, -0.02), (0.9, 0.05, 0.05)
    prob.sets = {"d2": (d2, (0, 0, 0)), "d1": (d1, (0, 0, 0))}
    phi0 = 1.0 + 0.3 * rng.standard_normal(prob.shape)
    steps = 15
    out, _ = orc.run(prob, [phi0], None, nsteps=steps, form="central")
    lam = _symbol_two_sets(prob, prob.a, d2, d1, prob.shape)
    exact = np.real(np.fft.ifftn(np.fft.fftn(phi0) * lam ** steps))
    assert float(np.abs(out[0] - exact).max()) < 1e-12
    # the even and odd sets act on different parts: swapping them changes the answer
    prob.sets = {"d2": (d1, (0, 0, 0)), "d1": (d2, (0, 0, 0))}
    swapped, _ = orc.run(prob, [phi0], None, nsteps=steps, form="central")
    assert float(np.abs(swapped[0] - exact).max()) > 1e-6


@pytest.mark.parametrize("lat,pde,levels", [("D2Q9", "LCDE", 2), ("D2Q9", "NCDE", 3), ("D2Q9", "NSE", 2)])
def test_sum_scales_with_zeroth_order_set_only(lat, pde, levels):
    rng = np.random.default_rng(14)
    prob = _base(lat, pde, levels, [9, 8])
    prob.sets = _sets(rng)
    L0 = _level(prob, rng)
    L1 = _level(prob, rng) if levels == 3 else None
    out = orc.step(prob, L0, L1, form="central")
    expect = sum(prob.a) * L0[0].sum() + (sum(prob.ahat) * L1[0].sum() if levels == 3 else 0.0)
    assert abs(out[0].sum() - expect) < 1e-12 * np.abs(L0[0]).sum()
