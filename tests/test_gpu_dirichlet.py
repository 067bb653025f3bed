"""Dirichlet boundaries (MMFD_BC_DIRICHLET) on the GPU.

- Example 3 of Sec. IV run natively (the boundary values set before every step): Case 1 gives
  the GRE printed in Table 4 to its three digits, and every case equals the host-driven run of
  the same procedure on the oracle (tests/example3_dirichlet.py).
- Parity with the oracle for every PDE on 2D and 3D lattices and the three kernel families: the
  oracle takes a periodic step and then resets the boundary ring, which is the definition of
  the boundary treatment (interior stencils never reach past the ring).  FP64 1e-12, FP32 1e-5.
- Time-dependent boundary values from device memory; sources together with the boundary; a 3D
  heat problem with zero boundary values converging at second order to its closed form; the
  server refuses such requests.
"""
import json
import os

import numpy as np
import pytest

import example3_dirichlet as E3
import gpu_cases as G
from oracle import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_17057_gb300 import mmfd
    return mmfd


def _ring_mask(shape):
    m = np.zeros(shape, dtype=bool)
    for ax in range(len(shape)):
        idx = [slice(None)] * len(shape)
        idx[ax] = 0
        m[tuple(idx)] = True
        idx[ax] = -1
        m[tuple(idx)] = True
    return m


def test_example3_table4_native(mm):
    with open(os.path.join(os.path.dirname(__file__), "golden", "example3_table4.json")) as fh:
        t4 = json.load(fh)
    for case in (1, 2, 3):
        lat, _, gamma = E3.CASES[case]
        co = mm.mmfd_wave_coefficients(gamma)
        for nx, printed in zip(t4["nx"], t4["gre"][f"case{case}"]):
            prob, dx, dt, nt = E3.problem(case, nx)
            Y, X = E3._grid(nx)
            p0, p1 = E3.start_levels(nx, dx, dt)
            s = mm.Solver(mm.make_desc(pde="LWE", lattice=lat, levels=3, n=[nx + 1, nx + 1], dt=dt, dx=[dx, dx],
                                       K=0.5 * np.eye(2), storage="fp64", boundary="dirichlet", **co))
            try:
                s.set_fields([p1])
                s.set_fields([p0], level=1)
                for m in range(1, nt):
                    s.set_boundary([np.exp(X + Y + (m + 1) * dt)])
                    s.step(1)
                out = s.fields()[0]
            finally:
                s.close()
            ex = np.exp(X + Y + nt * dt)
            got = float(np.abs(out - ex)[1:-1, 1:-1].sum() / np.abs(ex)[1:-1, 1:-1].sum())
            want = E3.interior_gre(case, nx, lambda cur, prev: orc.step(prob, [cur], [prev])[0])
            assert abs(got - want) <= 1e-6 * want, (case, nx, got, want)
            if case == 1:
                assert float("%.2e" % got) == float(printed), (nx, got, printed)


CASES = [
    ("D2Q9", "LCDE", 2, [300, 130], "k_march2d"),
    ("D2Q9", "NSE", 2, [300, 130], "k_march2d"),
    ("D2Q9", "NCDE", 3, [300, 130], "k_march2d"),
    ("D2Q5", "LCDE", 3, [40, 30], "k_direct"),
    ("D3Q7", "LCDE", 2, [130, 20, 9], "k_march3d"),
    ("D3Q19", "NSE", 2, [130, 12, 7], "k_march3d"),
    ("D3Q19", "NCDE", 3, [20, 16, 12], "k_direct"),
]


@pytest.mark.parametrize("storage,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("lat,pde,levels,n,kernel", CASES)
def test_dirichlet_parity(mm, lat, pde, levels, n, kernel, storage, tol):
    rng = np.random.default_rng(G.RNG_SEED + 3)
    kw, prob = G.case(lat, pde, levels, n, storage)
    L0 = G.random_level(prob, rng)
    L1 = G.random_level(prob, rng) if levels == 3 else None
    ring = _ring_mask(prob.shape)
    s = mm.Solver(mm.make_desc(**kw, boundary="dirichlet", temporal_depth=0))
    try:
        info = s.get_info()
        assert info.kernel.decode() == kernel and info.temporal_depth == 1
        s.set_fields(L0)
        if L1 is not None:
            s.set_fields(L1, level=1)
        s.step(5)
        got = s.fields()
    finally:
        s.close()
    cur, prev = [f.copy() for f in L0], ([f.copy() for f in L1] if L1 is not None else None)
    for _ in range(5):
        new = orc.step(prob, cur, prev)
        for f_new, f0 in zip(new, L0):
            f_new[ring] = f0[ring]
        prev, cur = cur, new
    assert G.rel_err(got, cur) <= tol, (lat, pde, levels, n, storage, G.rel_err(got, cur))


def test_time_dependent_boundary_from_device(mm):
    import torch
    rng = np.random.default_rng(17)
    kw, prob = G.case("D2Q9", "LCDE", 2, [260, 70], "fp32")
    L0 = G.random_level(prob, rng)
    ring = _ring_mask(prob.shape)
    bvals = [1.0 + 0.1 * rng.standard_normal(prob.shape) for _ in range(4)]
    s = mm.Solver(mm.make_desc(**kw, boundary="dirichlet"))
    try:
        s.set_fields(L0)
        for b in bvals:
            s.set_boundary([torch.tensor(b, dtype=torch.float32, device="cuda")])
            s.step(1)
        got = s.fields()
    finally:
        s.close()
    cur = [f.copy() for f in L0]
    for b in bvals:
        cur = orc.step(prob, cur)
        cur[0][ring] = b.astype(np.float32).astype(np.float64)[ring]
    assert G.rel_err(got, cur) <= 1e-5


def test_server_refuses_dirichlet(mm):
    kw, prob = G.case("D2Q9", "LCDE", 2, [64, 64], "fp32")
    srv = mm.Server(hbm_budget=1 << 28)
    try:
        with pytest.raises(mm.MMFDError) as e:
            srv.submit(mm.make_desc(**kw, boundary="dirichlet"), [np.ones(prob.shape)], 10)
        assert e.value.code == mm.MMFD_ERR_UNSUPPORTED
    finally:
        srv.close()


def test_dirichlet_with_sources(mm):
    # source terms and a prescribed boundary together (FP64): the oracle steps with the same
    # sources and then resets the ring
    rng = np.random.default_rng(23)
    kw, prob = G.case("D2Q9", "LCDE", 3, [150, 40], "fp64")
    b3, b3h = (1.2, 0.1, 0.2), (-0.4, 0.0, -0.1)
    kw.update(source="s", b=b3, bhat=b3h)
    prob.source, prob.b, prob.bhat = "s", b3, b3h
    L0, L1 = G.random_level(prob, rng), G.random_level(prob, rng)
    srcs = [[0.3 + 0.2 * rng.standard_normal(prob.shape)] for _ in range(5)]
    ring = _ring_mask(prob.shape)
    s = mm.Solver(mm.make_desc(**kw, boundary="dirichlet"))
    try:
        s.set_fields(L0)
        s.set_fields(L1, level=1)
        s.set_source(srcs[0], level=1)
        for m in range(1, 4):
            s.set_source(srcs[m])
            s.step(1)
        got = s.fields()
    finally:
        s.close()
    cur, prev = L0, L1
    for m in range(1, 4):
        new = orc.step(prob, cur, prev, src=(srcs[m], srcs[m - 1]))
        new[0][ring] = L0[0][ring]
        prev, cur = cur, new
    assert G.rel_err(got, cur) <= 1e-12


def test_dirichlet_3d_heat_converges(mm):
    # D3Q7 LCDE with u = 0 on [0, 1]^3, zero boundary values: phi = sin(pi x) sin(pi y) sin(pi z)
    # decays as exp(-3 pi^2 kappa t); with dt proportional to dx^2 the error falls at second order
    kappa, t_end = 0.05, 0.1
    errs = []
    for nx in (16, 32):
        n = nx + 1
        dx = 1.0 / nx
        dt = 0.1 * dx * dx / kappa      # derived d_0 = 2 kappa dt / dx^2 = 0.2 per axis (App. A: sum < 1)
        steps = int(round(t_end / dt))
        dt = t_end / steps
        g = np.arange(n) * dx
        Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
        phi0 = np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)
        s = mm.Solver(mm.make_desc("LCDE", "D3Q7", 2, [n, n, n], dt, [dx] * 3, K=kappa * np.eye(3), u=[0.0] * 3,
                                   targets=[0, -1, -1, 0, 0.5], storage="fp64", boundary="dirichlet"))
        try:
            s.set_fields([phi0])
            s.step(steps)
            out = s.fields()[0]
        finally:
            s.close()
        errs.append(float(np.abs(out - phi0 * np.exp(-3 * np.pi ** 2 * kappa * t_end)).max()))
    order = np.log2(errs[0] / errs[1])
    assert 1.9 <= order <= 2.2 and errs[1] < 1e-3, (errs, order)
