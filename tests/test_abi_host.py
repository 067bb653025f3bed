"""CPU-only tests of the C-ABI library: it loads, exports every declared symbol, and its host
logic (parameter resolution, validation) agrees with the paper and with the oracle's own,
independently written, parameter mapping.  No compute call touches a GPU here."""
import os
import re
from fractions import Fraction
import json

import numpy as np
import pytest

from oracle import fourier as F
from oracle import oracle as orc
from oracle import params as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden", "coefficient_sets.json")


@pytest.fixture(scope="module")
def mm():
    from paper_2505_17057_gb300 import build
    build.build()
    from paper_2505_17057_gb300 import mmfd
    return mmfd


def _declared_functions():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", f)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(mmfd_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(mm):
    declared = _declared_functions()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(mm.lib, name), name
        assert name in mm.SIGNATURES, f"binding lacks {name}"


def test_strerror_covers_codes(mm):
    for code in range(-10, 2):
        assert mm.strerror(code) != "unknown status"


def test_eq_x_solver_matches_printed_sets(mm):
    sets = json.load(open(GOLDEN))["sets"]
    for s in sets:
        t = [float(Fraction(s["targets"][k])) for k in ("a0", "A10", "A11", "A21", "A22")]
        a, ah = mm.mmfd_solve_three_level(t)
        exp = s.get("reading", s["printed"])
        assert np.allclose(a, [float(Fraction(v)) for v in exp["a"]], atol=1e-15)
        assert np.allclose(ah, [float(Fraction(v)) for v in exp["ahat"]], atol=1e-15)


def _describe(mm, **kw):
    return mm.mmfd_describe(mm.make_desc(**kw))


def test_describe_lcde_quadratic_matches_oracle_mapping(mm):
    K = [[0.02, 0.005], [0.005, 0.01]]
    u = [0.1, 0.05]
    info = _describe(mm, pde="LCDE", lattice="D2Q9", levels=2, n=[64, 64], dt=1.0, dx=[1, 1], K=K, u=u)
    prob = P.problem_lcde("D2Q9", 2, [64, 64], 1.0, [1, 1], K, u, P.two_level_from_a0(0.0))
    assert np.allclose(np.array([list(r) for r in info.Cmat]).ravel(), np.asarray(prob.Cmat), atol=1e-15)
    assert np.allclose(list(info.a), prob.a)
    assert abs(info.max_lambda - F.max_amplification(prob)) < 1e-12


def test_describe_axis_lattice_d0(mm):
    K = [[0.02, 0.0], [0.0, 0.01]]
    u = [0.1, 0.05]
    info = _describe(mm, pde="LCDE", lattice="D2Q5", levels=2, n=[64, 64], dt=1.0, dx=[1, 1], K=K, u=u)
    prob = P.problem_lcde("D2Q5", 2, [64, 64], 1.0, [1, 1], K, u, P.two_level_from_a0(0.0))
    assert np.allclose(list(info.d0)[:2], prob.d0[:2], atol=1e-15)
    # App. A rD2Q5I weights
    d1, d2 = prob.d0[:2]
    assert np.allclose(list(info.w)[:5], [1 - d1 - d2, d1 / 2, d2 / 2, d1 / 2, d2 / 2], atol=1e-15)


def test_describe_three_level_ncde(mm):
    rows = {s["name"]: s for s in json.load(open(GOLDEN))["sets"]}
    t = [float(Fraction(rows["ex1_case3"]["targets"][k])) for k in ("a0", "A10", "A11", "A21", "A22")]
    dx = 2 * np.pi / 256
    dt = 1e-4
    info = _describe(mm, pde="NCDE", lattice="D2Q9", levels=3, n=[256, 256], dt=dt, dx=[dx, dx],
                     flux=[[0, 0, 0.5, 0], [0, 0, 0.5, 0]], diff=[0.01, 0, 0.01, 0], targets=t)
    prob = P.problem_ncde("D2Q9", 3, [256, 256], dt, [dx, dx], [[0, 0, 0.5, 0], [0, 0, 0.5, 0]],
                          [0.01, 0, 0.01], (7 / 8, 0, 1 / 8), (1 / 8, 0, -1 / 8))
    assert np.allclose(list(info.m2), prob.m2, rtol=1e-14)
    A = P.three_level_moments((7 / 8, 0, 1 / 8), (1 / 8, 0, -1 / 8))
    assert abs(info.A10 - A[(1, 0)]) < 1e-15 and abs(info.A22 - A[(2, 2)]) < 1e-15
    assert abs(info.A21 - A[(2, 1)]) < 1e-15 and abs(info.A20 - A[(2, 0)]) < 1e-15


def test_d3q19_weights(mm):
    info = _describe(mm, pde="NSE", lattice="D3Q19", levels=2, n=[8, 8, 8], dt=1.0, dx=[1, 1, 1],
                     a=(1, 0, 0))
    E, w, _ = orc.lattice("D3Q19", [1 / 3] * 3, [1, 1, 1])
    assert np.allclose(list(info.w), w, atol=1e-15)


def test_validation_errors(mm):
    K = [[0.02, 0.005], [0.005, 0.01]]
    with pytest.raises(mm.MMFDError) as e:
        _describe(mm, pde="LCDE", lattice="D2Q5", levels=2, n=[64, 64], dt=1.0, dx=[1, 1], K=K, u=[0.1, 0.05])
    assert e.value.code == mm.MMFD_ERR_UNREPRESENTABLE
    info = _describe(mm, pde="LCDE", lattice="D2Q5", levels=2, n=[64, 64], dt=1.0, dx=[1, 1], K=K,
                     u=[0.1, 0.05], flags=mm.MMFD_FLAG_DROP_OFFDIAG)
    assert info.max_lambda <= 1 + 1e-12
    with pytest.raises(mm.MMFDError) as e:
        _describe(mm, pde="NSE", lattice="D2Q5", levels=2, n=[8, 8], dt=1.0, dx=[1, 1], a=(1, 0, 0))
    assert e.value.code == mm.MMFD_ERR_UNSUPPORTED
    with pytest.raises(mm.MMFDError) as e:
        # Table 3's coarsest row: u^2/c_s^2 = 50/3 is unstable
        _describe(mm, pde="LCDE", lattice="D2Q9", levels=2, n=[20, 20], dt=1 / 6, dx=[0.1, 0.1],
                  K=[[0.01, 0], [0, 0.01]], u=[1.0, 1.0])
    assert e.value.code == mm.MMFD_ERR_UNSTABLE
    info = _describe(mm, pde="LCDE", lattice="D2Q9", levels=2, n=[20, 20], dt=1 / 6, dx=[0.1, 0.1],
                     K=[[0.01, 0], [0, 0.01]], u=[1.0, 1.0], flags=mm.MMFD_FLAG_ALLOW_UNSTABLE)
    assert info.max_lambda > 1
    with pytest.raises(mm.MMFDError) as e:
        _describe(mm, pde="LCDE", lattice="D2Q9", levels=2, n=[0, 20], dt=1.0, dx=[1, 1], K=np.eye(2) * 0.01)
    assert e.value.code == mm.MMFD_ERR_ARG
    with pytest.raises(mm.MMFDError) as e:
        # A_00 != 1
        _describe(mm, pde="LCDE", lattice="D2Q9", levels=2, n=[8, 8], dt=1.0, dx=[1, 1], K=np.eye(2) * 0.01,
                  a=(0.9, 0.0, 0.0))
    assert e.value.code == mm.MMFD_ERR_ARG


def test_stability_check_matches_oracle_symbol(mm):
    # the library's create-time max |lambda| equals the oracle's symbol on small grids (all wave numbers)
    for a0 in (0.0, 0.3, -0.4):
        for lat in ("D2Q5", "D2Q9"):
            K = [[0.03, 0.0], [0.0, 0.02]]
            u = [0.2, -0.1]
            info = _describe(mm, pde="LCDE", lattice=lat, levels=2, n=[24, 20], dt=1.0, dx=[1, 1], K=K, u=u,
                             targets=[a0, -1, -1, 0, 0.5], flags=mm.MMFD_FLAG_ALLOW_UNSTABLE)
            prob = P.problem_lcde(lat, 2, [24, 20], 1.0, [1, 1], K, u, P.two_level_from_a0(a0))
            assert abs(info.max_lambda - F.max_amplification(prob)) < 1e-12


def _corollary1_q(prob, shape):
    """max over wave numbers (theta = 0 excluded) of A^2 + B^2, Corollary 1's A and B."""
    up, um, E = F.ubar_split(prob)
    th = F.thetas(shape)
    dim = len(shape)
    A = np.zeros(shape)
    B = np.zeros(shape)
    for j in range(E.shape[0]):
        xi = sum(th[i] * E[j][dim - 1 - i] for i in range(dim))
        A += up[j] * np.cos(xi)
        B += um[j] * np.sin(xi)
    q = A * A + B * B
    q.flat[0] = 0.0
    return float(q.max())


def test_trt_coefficients(mm):
    for s in (0.3, 1.0, 1.7):
        w = 1.0 - s
        c = mm.mmfd_trt_coefficients(s)
        assert c == {"a": (1.0, 0.0, w), "ahat": (0.0, -w, 0.0), "abar": (1.0, 0.0, -w), "abarhat": (0.0, w, 0.0)}
    for bad in (0.0, 2.0, -0.5, float("nan")):
        with pytest.raises(mm.MMFDError) as e:
            mm.mmfd_trt_coefficients(bad)
        assert e.value.code == mm.MMFD_ERR_ARG


def test_stability_check_trt_is_corollary1(mm):
    # the library's create-time check with the TRT sets: its max |lambda| equals the oracle's
    # three-level roots, and it flags instability exactly where Corollary 1 (A^2 + B^2 > 1) does
    rng = np.random.default_rng(77)
    verdicts = []
    for _ in range(40):
        lat = ("D2Q5", "D2Q9")[rng.integers(2)]
        s = rng.uniform(0.2, 1.9)
        coef = mm.mmfd_trt_coefficients(s)
        # K in units of the TRT's natural diffusivity (1/s- - 1/2) dt: the derived c_s^2 is then
        # k0 + u_alpha^2 on D2Q5, below the App. A bound d_0x + d_0y < 1
        K = np.diag(rng.uniform(0.005, 0.2, 2)) * (1.0 / s - 0.5)
        ang = rng.uniform(0, 2 * np.pi)
        mag = rng.uniform(0.1, 0.7)
        u = [mag * np.cos(ang), mag * np.sin(ang)]
        info = _describe(mm, pde="LCDE", lattice=lat, levels=3, n=[20, 18], dt=1.0, dx=[1, 1], K=K, u=u,
                         a=coef["a"], ahat=coef["ahat"], flags=mm.MMFD_FLAG_ALLOW_UNSTABLE)
        prob = P.problem_lcde(lat, 3, [20, 18], 1.0, [1, 1], K, u, coef["a"], coef["ahat"])
        assert abs(info.max_lambda - F.max_amplification(prob)) < 1e-12
        q = _corollary1_q(prob, prob.shape)
        if abs(q - 1) < 1e-9:
            continue
        # the library's maximum includes theta = 0 (root exactly 1, the conserved mass)
        assert (info.max_lambda > 1 + 1e-12) == (q > 1), (lat, s, mag, q, info.max_lambda)
        verdicts.append(q > 1)
    assert len(verdicts) > 30 and 3 <= sum(verdicts) <= len(verdicts) - 3


def test_source_descriptor_validation(mm):
    K = np.eye(2) * 0.02
    base = dict(lattice="D2Q9", n=[32, 16], dt=1.0, dx=[1, 1])
    with pytest.raises(mm.MMFDError) as e:
        _describe(mm, pde="NSE", levels=2, a=(1, 0, 0), source="s", **base)
    assert e.value.code == mm.MMFD_ERR_UNSUPPORTED
    with pytest.raises(mm.MMFDError) as e:
        _describe(mm, pde="NCDE", levels=2, flux=[[0, 0.1, 0, 0], [0, 0.1, 0, 0]], diff=[0.1, 0, 0, 0],
                  source="su", **base)
    assert e.value.code == mm.MMFD_ERR_ARG
    with pytest.raises(mm.MMFDError) as e:
        _describe(mm, pde="LCDE", levels=2, K=K, u=[0.1, 0], source="s", bhat=(0.5, 0, 0), **base)
    assert e.value.code == mm.MMFD_ERR_ARG
    # compulsory bytes: FP32 levels (read one, write one) plus the source fields read once
    info = _describe(mm, pde="LCDE", levels=2, K=K, u=[0.1, 0], source="sm", storage="fp32", **base)
    assert info.bytes_per_lu == 4 * 2 + 4 * 3
    info = _describe(mm, pde="LCDE", levels=3, K=K, u=[0.1, 0], source="su", storage="fp64",
                     targets=[0, -1, -1, 0.25, 0.5], **base)
    assert info.bytes_per_lu == 8 * 3 + 8 * 2


def test_wave_descriptor(mm):
    c3 = mm.mmfd_wave_coefficients(3 / 8)
    assert c3 == {"a": (3 / 8, 5 / 4, 3 / 8), "ahat": (0.0, -1.0, 0.0)}
    with pytest.raises(mm.MMFDError):
        mm.mmfd_wave_coefficients(0.0)
    K = np.diag([0.5, 0.3])
    base = dict(pde="LWE", levels=3, n=[20, 18], dt=0.5, dx=[1.0, 1.0], K=K, flags=mm.MMFD_FLAG_ALLOW_UNSTABLE)
    for lat, gamma in [("D2Q5", 3 / 8), ("D2Q9", 3 / 8), ("D2Q9", 1 / 2)]:
        co = mm.mmfd_wave_coefficients(gamma)
        info = _describe(mm, lattice=lat, **co, **base)
        prob = P.problem_lwe(lat, [20, 18], 0.5, [1.0, 1.0], K, co["a"], co["ahat"])
        assert abs(info.A22 - gamma) < 1e-15 and abs(info.A20 + 1) < 1e-15 and abs(info.A10) < 1e-15
        assert np.allclose(list(info.d0)[:2], prob.d0[:2], rtol=1e-14)
        assert np.allclose(np.array([list(r) for r in info.Cmat]).ravel(), prob.Cmat, atol=1e-14)
        # the constant mode is a double root 1; the oracle's quadratic formula resolves it only to
        # O(sqrt(eps)), the library takes it exactly
        assert abs(info.max_lambda - F.max_amplification(prob)) < 1e-7
        assert info.max_lambda <= 1 + 1e-12
    co = mm.mmfd_wave_coefficients(3 / 8)
    for bad, code in [(dict(levels=2), mm.MMFD_ERR_ARG), (dict(u=[0.1, 0.0]), mm.MMFD_ERR_ARG),
                      (dict(a=(0.6, 1.0, 0.4), ahat=(0.0, -1.0, 0.0)), mm.MMFD_ERR_ARG),
                      (dict(source="s"), mm.MMFD_ERR_UNSUPPORTED)]:
        kw = dict(base, lattice="D2Q9", **co)
        kw.update(bad)
        with pytest.raises(mm.MMFDError) as e:
            _describe(mm, **kw)
        assert e.value.code == code, bad


def test_storage_reference_rules(mm):
    # NSE velocities have zero reference (their update is not affine in u); non-finite references
    # are rejected; FP64 levels hold values whatever the reference
    base = dict(pde="NSE", lattice="D2Q9", levels=2, n=[16, 16], dt=1.0, dx=[1, 1], a=(1, 0, 0), abar=(1, 0, 0))
    for st in ("fp32", "bf16"):
        mm.mmfd_describe(mm.make_desc(**base, storage=st, ref=[1.0, 0.0, 0.0]))
        with pytest.raises(mm.MMFDError) as e:
            mm.mmfd_describe(mm.make_desc(**base, storage=st, ref=[1.0, 0.01, 0.0]))
        assert e.value.code == mm.MMFD_ERR_ARG
    mm.mmfd_describe(mm.make_desc(**base, storage="fp64", ref=[1.0, 0.01, 0.0]))
    with pytest.raises(mm.MMFDError) as e:
        mm.mmfd_describe(mm.make_desc(pde="LCDE", lattice="D2Q9", levels=2, n=[16, 16], dt=1.0, dx=[1, 1],
                                      K=np.eye(2) * 0.01, storage="fp32", ref=[float("inf")]))
    assert e.value.code == mm.MMFD_ERR_ARG


def _theta_sweeps_from_oracle(prob, theta, eps):
    """Jacobi sweeps that take every mode's initial error ell / (1 - theta_1 ell) below eps when
    each sweep multiplies it by g = theta_1 (E - W0) / d, d = 1 + theta_1 (1 - W0); E and W0 from
    the oracle's explicit step (impulse response)."""
    delta = np.zeros(prob.shape)
    delta[(0,) * len(prob.shape)] = 1.0
    h = orc.step(prob, [delta])[0]
    W0 = h[(0,) * len(prob.shape)]
    E = np.fft.fftn(h)
    th1 = 1.0 - theta
    ell = E - 1.0
    g = np.abs(th1 * (E - W0) / (1.0 + th1 * (1.0 - W0)))
    b = np.abs(ell) / np.abs(1.0 - th1 * ell)
    m = (b > eps) & (g > 0)
    return max(1, int(np.ceil((np.log(eps / b[m]) / np.log(g[m])).max()))) if m.any() else 1


def test_theta_descriptor(mm):
    # the two-level theta-scheme (Eq. (GCN)): validation, the create-time check against
    # Eq. (Tcond1-1), and the Jacobi sweep count against the oracle's own symbol
    K = [[0.03, 0.004], [0.004, 0.02]]
    u = [0.15, -0.1]
    for lat in ("D2Q5", "D2Q9"):
        KK = np.diag(np.diag(K)) if lat == "D2Q5" else K
        for dt in (1.0, 3.0):
            prob = P.problem_lcde(lat, 2, [24, 20], dt, [1, 1], KK, u, P.two_level_from_a0(0.0))
            for theta in (0.0, 0.4, 0.5, 0.8):
                for st, es, eps in (("fp64", 8, 1e-15), ("fp32", 4, 6e-8)):
                    info = _describe(mm, pde="LCDE", lattice=lat, levels=2, n=[24, 20], dt=dt, dx=[1, 1], K=KK, u=u,
                                     a=P.two_level_from_a0(0.0), storage=st, theta=theta,
                                     flags=mm.MMFD_FLAG_ALLOW_UNSTABLE)
                    lam = np.abs(F.theta_lambda(prob, theta, prob.shape)).max()
                    assert abs(info.max_lambda - lam) < 1e-12, (lat, dt, theta)
                    k = _theta_sweeps_from_oracle(prob, theta, eps)
                    assert k <= info.sweeps <= k + 1, (lat, dt, theta, st, k, info.sweeps)
                    assert info.bytes_per_lu == es * (2 + 3 * info.sweeps)
    # theta = 1 is the explicit scheme: one sweep (x = rhs); no flag: no sweeps
    base = dict(pde="LCDE", lattice="D2Q9", levels=2, n=[32, 32], dt=1.0, dx=[1, 1], K=K, u=u)
    assert _describe(mm, **base, theta=1.0).sweeps == 1
    assert _describe(mm, **base).sweeps == 0
    # Theorem 2: heavily diffusive D2Q5 (a_0 = -2): theta <= 1/2 passes the check, the explicit end fails
    heavy = dict(pde="LCDE", lattice="D2Q5", levels=2, n=[16, 16], dt=1.0, dx=[1, 1], K=[[0.3, 0], [0, 0.25]],
                 u=[0.2, 0.1], a=P.two_level_from_a0(-2.0), storage="fp64")
    for theta in (0.0, 0.25, 0.5):
        assert _describe(mm, **heavy, theta=theta).max_lambda <= 1 + 1e-12
    with pytest.raises(mm.MMFDError) as e:
        _describe(mm, **heavy, theta=1.0)
    assert e.value.code == mm.MMFD_ERR_UNSTABLE
    # what the theta-scheme is not built for
    for bad, code in [(dict(theta=1.5), mm.MMFD_ERR_ARG), (dict(theta=-0.1), mm.MMFD_ERR_ARG),
                      (dict(theta=float("nan")), mm.MMFD_ERR_ARG),
                      (dict(theta=0.5, storage="bf16"), mm.MMFD_ERR_UNSUPPORTED),
                      (dict(theta=0.5, source="s"), mm.MMFD_ERR_UNSUPPORTED),
                      (dict(theta=0.5, levels=3, targets=[0, -1, -1, 0.25, 0.5]), mm.MMFD_ERR_UNSUPPORTED)]:
        kw = dict(base)
        kw.update(bad)
        with pytest.raises(mm.MMFDError) as e:
            _describe(mm, **kw)
        assert e.value.code == code, bad
    with pytest.raises(mm.MMFDError) as e:
        _describe(mm, pde="NCDE", lattice="D2Q9", levels=2, n=[16, 16], dt=1.0, dx=[1, 1],
                  flux=[[0, 0.1, 0, 0], [0, 0.1, 0, 0]], diff=[0.1, 0, 0, 0], theta=0.5)
    assert e.value.code == mm.MMFD_ERR_UNSUPPORTED


def test_theta_check_at_the_eq_tcond1_3_bound(mm):
    # the create-time check accepts theta just inside theta* = 1/2 + min (-A / (A^2 + B^2))
    # (Eq. (Tcond1-3), from the oracle's A and B) and refuses it just outside
    prob = P.problem_lcde("D2Q5", 2, [16, 16], 1.0, [1, 1], [[0.3, 0], [0, 0.25]], [0.2, 0.1],
                          P.two_level_from_a0(-2.0))
    A, B = F.theta_AB(prob, prob.shape)
    q = A * A + B * B
    m = q > 1e-14
    ts = 0.5 + float((-A[m] / q[m]).min())
    heavy = dict(pde="LCDE", lattice="D2Q5", levels=2, n=[16, 16], dt=1.0, dx=[1, 1], K=[[0.3, 0], [0, 0.25]],
                 u=[0.2, 0.1], a=P.two_level_from_a0(-2.0), storage="fp64")
    assert _describe(mm, **heavy, theta=ts - 1e-3).max_lambda <= 1 + 1e-12
    with pytest.raises(mm.MMFDError) as e:
        _describe(mm, **heavy, theta=ts + 1e-3)
    assert e.value.code == mm.MMFD_ERR_UNSTABLE


def test_dirichlet_descriptor(mm):
    base = dict(pde="LCDE", lattice="D2Q9", levels=2, n=[32, 16], dt=1.0, dx=[1, 1], K=np.eye(2) * 0.02,
                u=[0.1, 0.0])
    _describe(mm, **base, boundary="dirichlet")
    for bad, code in [(dict(n=[32, 2]), mm.MMFD_ERR_ARG), (dict(theta=0.5), mm.MMFD_ERR_UNSUPPORTED)]:
        kw = dict(base, boundary="dirichlet")
        kw.update(bad)
        with pytest.raises(mm.MMFDError) as e:
            _describe(mm, **kw)
        assert e.value.code == code, bad
    d = mm.make_desc(**base)
    d.boundary = 7
    with pytest.raises(mm.MMFDError) as e:
        mm.mmfd_describe(d)
    assert e.value.code == mm.MMFD_ERR_ARG
