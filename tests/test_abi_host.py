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
