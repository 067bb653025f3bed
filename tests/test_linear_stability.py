"""Frozen-coefficient stability of the nonlinear schemes (NCDE, He-Luo NSE) -- host side, no GPU.

mmfd_linear_stability linearises the library's update about a uniform state and returns the
largest amplification-factor modulus over the grid's wave numbers (eigenvalues of the per-mode
symbol matrix; three-level: its companion matrix, Eq. (3-level)).  It is pinned against the
oracle: the Jacobian of one oracle step (central differences, exact up to rounding for the
quadratic He-Luo EDF and to O(eps^2) for the NCDE polynomials) about the same uniform state on a
tiny periodic grid, whose eigenvalues are exactly the union of the per-mode symbols' (the
linearised operator is translation invariant).  mmfd_create / mmfd_describe run the check about
the reference state and refuse unstable descriptors."""
import numpy as np
import pytest

import gpu_cases as G
from oracle import oracle as orc
from oracle import params as P
from paper_2505_17057_gb300 import mmfd


def oracle_max_amplification(prob, state):
    nf, levels, shape = prob.nf, prob.levels, prob.shape
    base = [np.full(shape, float(s)) for s in state[:nf]]
    N = int(np.prod(shape))
    eps = 1e-6

    def step(L0, L1):
        out, _ = orc.run(prob, L0, L1, nsteps=1)
        return np.concatenate([o.reshape(-1) for o in out])

    cols = {0: [], 1: []}
    for which in ([0, 1] if levels == 3 else [0]):
        for f in range(nf):
            for i in range(N):
                Lp = [[b.copy() for b in base], [b.copy() for b in base]]
                Lm = [[b.copy() for b in base], [b.copy() for b in base]]
                Lp[which][f].reshape(-1)[i] += eps
                Lm[which][f].reshape(-1)[i] -= eps
                l1p = Lp[1] if levels == 3 else None
                l1m = Lm[1] if levels == 3 else None
                cols[which].append((step(Lp[0], l1p) - step(Lm[0], l1m)) / (2 * eps))
    J0 = np.array(cols[0]).T
    if levels == 3:
        J1 = np.array(cols[1]).T
        n = J0.shape[0]
        J0 = np.block([[J0, J1], [np.eye(n), np.zeros((n, n))]])
    return float(np.abs(np.linalg.eigvals(J0)).max())


def case(lat, pde, levels, n, dt_scale=1.0):
    kw, prob = G.case(lat, pde, levels, n, "fp64")
    if dt_scale != 1.0:
        kw["dt"] *= dt_scale
        prob = P.problem_ncde(lat, levels, prob.n, kw["dt"], kw["dx"], kw["flux"], kw["diff"][:3], kw["a"], kw["ahat"])
    return kw, prob


CASES = [
    # unstable linearisations (the largest modulus is a distinctive number): diffusion-number x 6
    # for the NCDE, a fast uniform flow for the NSE
    ("D2Q9", "NCDE", 2, [6, 5], [0.7], 6.0),
    ("D2Q9", "NCDE", 3, [6, 5], [0.7], 6.0),
    ("D3Q19", "NCDE", 3, [4, 3, 3], [0.7], 6.0),
    ("D2Q9", "NSE", 2, [6, 5], [1.02, 0.45, -0.35], 1.0),
    ("D3Q19", "NSE", 2, [4, 3, 3], [1.02, 0.4, -0.3, 0.35], 1.0),
    # stable ones (the conserved modes at theta = 0 set the maximum, 1)
    ("D2Q9", "NCDE", 2, [6, 5], [0.7], 1.0),
    ("D2Q9", "NSE", 3, [5, 4], [1.02, 0.05, -0.03], 1.0),
    ("D3Q19", "NSE", 3, [4, 3, 3], [1.0, 0.04, -0.03, 0.02], 1.0),
]


@pytest.mark.parametrize("lat,pde,levels,n,state,dts", CASES)
def test_linearised_symbol_matches_oracle_jacobian(lat, pde, levels, n, state, dts):
    kw, prob = case(lat, pde, levels, n, dts)
    rc, lib = mmfd.mmfd_linear_stability(mmfd.make_desc(**kw, flags=mmfd.MMFD_FLAG_ALLOW_UNSTABLE), state)
    ref = oracle_max_amplification(prob, state)
    assert abs(lib - ref) <= 1e-8 * ref, (lib, ref)
    assert (rc == mmfd.MMFD_ERR_UNSTABLE) == (ref > 1 + 1e-6), (rc, ref)


def test_create_refuses_unstable_ncde():
    # the NCDE at its reference state phi = 0 with six times the stable time step
    kw, _ = case("D2Q9", "NCDE", 2, [64, 48], 6.0)
    with pytest.raises(mmfd.MMFDError) as e:
        mmfd.mmfd_describe(mmfd.make_desc(**kw))
    assert e.value.code == mmfd.MMFD_ERR_UNSTABLE
    info = mmfd.mmfd_describe(mmfd.make_desc(**kw, flags=mmfd.MMFD_FLAG_ALLOW_UNSTABLE))
    assert info.max_lambda > 1.5
    kw1, _ = case("D2Q9", "NCDE", 2, [64, 48], 1.0)
    assert mmfd.mmfd_describe(mmfd.make_desc(**kw1)).max_lambda <= 1 + 1e-9


def test_create_refuses_nse_unstable_at_rest():
    # two-level He-Luo sets a = abar = (1 - a0/2, a0, -a0/2): a0 = 0 (LBGK tau = 1) and 0.5 are
    # stable at rest, a0 = -1 is not
    for a0, stable in [(0.0, True), (0.5, True), (-1.0, False)]:
        a = P.two_level_from_a0(a0)
        kw = dict(pde="NSE", lattice="D2Q9", levels=2, n=[32, 32], dt=1.0, dx=[1.0, 1.0], a=a, abar=a)
        if stable:
            assert mmfd.mmfd_describe(mmfd.make_desc(**kw)).max_lambda <= 1 + 1e-9
        else:
            with pytest.raises(mmfd.MMFDError) as e:
                mmfd.mmfd_describe(mmfd.make_desc(**kw))
            assert e.value.code == mmfd.MMFD_ERR_UNSTABLE
            prob = P.problem_nse("D2Q9", 2, [6, 5], 1.0, [1.0, 1.0], a, a)
            assert oracle_max_amplification(prob, [1.0, 0.0, 0.0]) > 1.5


def test_linear_pdes_are_refused():
    kw = dict(pde="LCDE", lattice="D2Q9", levels=2, n=[16, 16], dt=1.0, dx=[1.0, 1.0], K=[[0.02, 0], [0, 0.02]],
              u=[0.1, 0.0], targets=[0, -1, -1, 0, 0.5])
    with pytest.raises(mmfd.MMFDError) as e:
        mmfd.mmfd_linear_stability(mmfd.make_desc(**kw), [1.0])
    assert e.value.code == mmfd.MMFD_ERR_UNSUPPORTED


def test_served_ncde_requests_stable_about_their_extreme_states():
    # the request generator's time step keeps every NCDE request of the seeded stream linearly
    # stable about each value its initial field spans (convection speed B'(phi) = phi), not only
    # about phi = 0 as mmfd_create checks
    from paper_2505_17057_gb300 import serving
    reqs = [r for r in serving.make_stream(60, seed=5) if r.desc["pde"] == "NCDE"]
    assert len(reqs) >= 10
    for r in reqs:
        m = float(np.abs(r.fields[0]).max())
        d = mmfd.make_desc(**r.desc)
        for v in np.linspace(-m, m, 5):
            rc, amp = mmfd.mmfd_linear_stability(d, [v])
            assert rc == mmfd.MMFD_OK and amp <= 1 + 1e-9, (r.desc["n"], r.desc["dt"], v, amp)
