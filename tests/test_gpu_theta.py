"""GPU parity of the two-level theta-scheme (Eq. (GCN)) through the C ABI.

The library solves (I - (1 - theta) L) phi^{n+1} = (I + theta L) phi^n by a right-hand-side
launch and a fixed number of Jacobi sweeps; the oracle solves the same system exactly in the DFT
basis.  Tolerances as elsewhere: FP64 1e-12, FP32 1e-5 relative to the field's max |value|.

- every lattice, both storages, the three kernel families (direct, 2D and 3D marching), grids
  spanning several tiles with ragged tails, theta in {0, 1/2, 0.7}, time steps beyond the
  explicit scheme's limit;
- theta = 1 gives the explicit solver's result bit for bit;
- the full-size workload (theta2d_4096): a plane wave is multiplied per step by Eq. (Tcond1-1)'s
  lambda (checked on sampled nodes) and the mass is conserved;
- the Jacobi sweeps fused per launch by the blocked 2D kernel (depths 2 .. 4, with blocked and
  single-sweep remainders) against the oracle;
- the solve server refuses theta-scheme requests; the autotuner keeps the result.
"""
import zlib

import numpy as np
import pytest

import gpu_cases as G
from oracle import fourier as F
from oracle import oracle as orc
from oracle import params as P

pytestmark = pytest.mark.gpu

A2 = P.two_level_from_a0(0.0)


@pytest.fixture(scope="module")
def mm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_17057_gb300 import mmfd
    return mmfd


def theta_case(lat, n, storage, dt, theta):
    dim = G.dims(lat)
    n = list(n) + [1] * (3 - len(n))
    dx = [1.0, 1.1, 0.9][:dim]
    if lat in ("D2Q5", "D3Q7"):
        K = np.diag([0.05, 0.04, 0.06][:dim])
    else:
        K = np.diag([0.05, 0.04, 0.06][:dim]) + 0.006 * (1 - np.eye(dim))
    u = [0.08, -0.05, 0.04][:dim]
    kw = dict(pde="LCDE", lattice=lat, levels=2, n=n[:2] if dim == 2 else n, dt=dt, dx=dx, K=K, u=u, a=A2,
              storage=storage, theta=theta)
    prob = P.problem_lcde(lat, 2, n, dt, dx, K, u, A2)
    return kw, prob


def smooth_level(prob, rng, modes=24):
    """1 + a sum of random Fourier modes (the workloads' field recipe) on the problem's grid."""
    shape = prob.shape
    grids = np.meshgrid(*[np.arange(m) for m in shape], indexing="ij")
    phi = np.ones(shape)
    for _ in range(modes):
        ph = rng.uniform(0, 2 * np.pi)
        arg = ph
        for g, m in zip(grids, shape):
            arg = arg + 2 * np.pi * rng.integers(-6, 7) * g / m
        phi += rng.uniform(0.02, 0.1) * np.cos(arg)
    return [phi]


CASES = [
    ("D2Q9", [300, 130], "fp64", 2.4, 0.5, "k_march2d_src"),
    ("D2Q9", [300, 130], "fp32", 2.4, 0.0, "k_march2d_src"),
    ("D2Q5", [257, 64], "fp32", 1.6, 0.7, "k_march2d_src"),
    ("D2Q5", [257, 64], "fp64", 1.6, 0.0, "k_march2d_src"),
    ("D2Q9", [40, 30], "fp64", 2.4, 0.5, "k_direct_src"),
    ("D2Q9", [37, 29], "fp32", 2.4, 0.5, "k_direct_src"),
    ("D3Q7", [130, 20, 9], "fp64", 1.6, 0.5, "k_march3d_src"),
    ("D3Q7", [20, 16, 12], "fp32", 1.6, 0.0, "k_direct_src"),
    ("D3Q19", [129, 12, 7], "fp32", 2.0, 0.5, "k_march3d_src"),
    ("D3Q19", [129, 12, 7], "fp64", 2.0, 0.7, "k_march3d_src"),
]


@pytest.mark.parametrize("lat,n,storage,dt,theta,kernel", CASES)
def test_theta_parity(mm, lat, n, storage, dt, theta, kernel):
    rng = np.random.default_rng(G.RNG_SEED)
    kw, prob = theta_case(lat, n, storage, dt, theta)
    L0 = smooth_level(prob, rng)
    s = mm.Solver(mm.make_desc(**kw))
    try:
        info = s.get_info()
        assert info.kernel.decode() == kernel
        assert info.sweeps >= 1 and info.temporal_depth == 1
        s.set_fields(L0)
        s.step(4)
        got = s.fields()
        assert s.get_info().steps_done == 4
    finally:
        s.close()
    want = orc.theta_run(prob, L0, 4, theta)
    tol = 1e-12 if storage == "fp64" else 1e-5
    assert G.rel_err(got, want) <= tol, (lat, n, storage, theta, G.rel_err(got, want))


# Jacobi sweeps fused per launch by the 2D blocked kernel: (case, temporal_depth asked, depth in
# use).  The sweep counts (10, 12, 19, 10, 15, 8) leave a blocked remainder, none, a single-sweep
# remainder, ...; ny = 8 is the smallest grid the depth-4 wavefront allows.
BLOCKED = [
    (("D2Q9", [300, 130], "fp32", 2.4, 0.5), 4, 4),
    (("D2Q5", [257, 64], "fp32", 1.6, 0.0), 3, 3),
    (("D2Q9", [300, 130], "fp64", 2.4, 0.5), 0, 2),
    (("D2Q9", [128, 8], "fp32", 2.4, 0.5), 4, 4),
    (("D2Q5", [200, 33], "fp64", 1.6, 0.7), 2, 2),
    (("D2Q9", [131, 70], "fp32", 2.4, 0.7), 0, 4),
]


@pytest.mark.parametrize("case,asked,depth", BLOCKED)
def test_theta_blocked_sweeps_parity(mm, case, asked, depth):
    lat, n, storage, dt, theta = case
    rng = np.random.default_rng(G.RNG_SEED + 1)
    kw, prob = theta_case(lat, n, storage, dt, theta)
    L0 = smooth_level(prob, rng)
    s = mm.Solver(mm.make_desc(**kw, temporal_depth=asked))
    try:
        info = s.get_info()
        assert info.kernel.decode() == "k_march2d_tb" and info.temporal_depth == depth
        s.set_fields(L0)
        s.step(4)
        got = s.fields()
        assert s.get_info().steps_done == 4
    finally:
        s.close()
    want = orc.theta_run(prob, L0, 4, theta)
    tol = 1e-12 if storage == "fp64" else 1e-5
    assert G.rel_err(got, want) <= tol, (case, asked, G.rel_err(got, want))


def test_theta_beyond_the_explicit_limit(mm):
    # at this step the explicit scheme is refused as unstable; Crank-Nicolson runs and matches
    kw, prob = theta_case("D2Q9", [160, 140], "fp64", 10.0, 0.5)
    with pytest.raises(mm.MMFDError) as e:
        mm.mmfd_describe(mm.make_desc(**dict(kw, theta=1.0)))
    assert e.value.code == mm.MMFD_ERR_UNSTABLE
    rng = np.random.default_rng(3)
    L0 = smooth_level(prob, rng)
    s = mm.Solver(mm.make_desc(**kw))
    try:
        s.set_fields(L0)
        s.step(6)
        got = s.fields()
    finally:
        s.close()
    want = orc.theta_run(prob, L0, 6, 0.5)
    assert G.rel_err(got, want) <= 1e-12


@pytest.mark.parametrize("lat,n", [("D2Q9", [300, 130]), ("D3Q19", [129, 12, 7])])
def test_theta_one_is_the_explicit_solver_bitwise(mm, lat, n):
    rng = np.random.default_rng(11)
    kw, prob = theta_case(lat, n, "fp32", 0.8, 1.0)
    L0 = smooth_level(prob, rng)
    out = []
    for extra in (dict(theta=1.0), dict(theta=None)):
        s = mm.Solver(mm.make_desc(**dict(kw, **extra), temporal_depth=1))
        try:
            s.set_fields(L0)
            s.step(5)
            out.append(s.fields()[0])
        finally:
            s.close()
    assert np.array_equal(out[0], out[1])


def test_theta_full_size_plane_wave(mm):
    # theta2d_4096 as the bench runs it (FP32, dt = 8, theta = 1/2): phi = 1 + eps cos(k . x) is
    # an eigenvector of the step, so after n steps it is 1 + Re(lambda^n eps e^{i k . x}) with
    # lambda of Eq. (Tcond1-1); checked on sampled nodes, with the mass
    import torch
    from paper_2505_17057_gb300 import configs
    desc, _, _ = configs.theta2d_4096()
    N = desc["n"][0]
    mx, my, eps = 16, 32, 0.1
    # the same wave numbers on a 256^2 grid: (1, 2) there
    small = P.problem_lcde("D2Q9", 2, [256, 256], desc["dt"], [1.0, 1.0], desc["K"], desc["u"], A2)
    lam = F.theta_lambda(small, desc["theta"], small.shape)[my // 16, mx // 16]
    steps = 6
    x = torch.arange(N, device="cuda", dtype=torch.float64)
    arg = 2 * np.pi * (mx * x[None, :] + my * x[:, None]) / N
    phi = (1.0 + eps * torch.cos(arg)).to(torch.float32)
    s = mm.Solver(mm.make_desc(**desc))
    try:
        s.set_fields([phi])
        m0 = s.reduce(mm.MMFD_RED_SUM)[0]
        s.step(steps)
        got = s.fields()[0]
        m1 = s.reduce(mm.MMFD_RED_SUM)[0]
    finally:
        s.close()
    rng = np.random.default_rng(5)
    iy = rng.integers(0, N, 4096)
    ix = rng.integers(0, N, 4096)
    a = 2 * np.pi * (mx * ix + my * iy) / N
    want = 1.0 + np.real(lam ** steps * eps * np.exp(1j * a))
    assert np.abs(got[iy, ix] - want).max() <= 1e-5
    assert abs(m0 - N * N) <= 1e-6 * N * N
    assert abs(m1 - m0) <= 1e-6 * abs(m0)


def test_server_refuses_theta_requests(mm):
    kw, prob = theta_case("D2Q9", [64, 64], "fp32", 0.8, 0.5)
    srv = mm.Server(hbm_budget=1 << 28)
    try:
        f = np.ones(prob.shape)
        with pytest.raises(mm.MMFDError) as e:
            srv.submit(mm.make_desc(**kw), [f], 10)
        assert e.value.code == mm.MMFD_ERR_UNSUPPORTED
    finally:
        srv.close()


def test_theta_autotune_keeps_the_result(mm):
    rng = np.random.default_rng(9)
    kw, prob = theta_case("D2Q9", [520, 300], "fp32", 2.4, 0.5)
    L0 = smooth_level(prob, rng)
    s = mm.Solver(mm.make_desc(**kw, temporal_depth=0))
    try:
        s.set_fields(L0)
        t = s.autotune(None)
        assert 1 <= t.temporal_depth <= 4
        s.set_fields(L0)
        s.step(3)
        got = s.fields()
    finally:
        s.close()
    want = orc.theta_run(prob, L0, 3, 0.5)
    assert G.rel_err(got, want) <= 1e-5


def _random_cases(count, seed=20250603):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        lat = ["D2Q5", "D2Q9", "D3Q7", "D3Q19"][rng.integers(4)]
        storage = ["fp32", "fp64"][rng.integers(2)]
        if lat.startswith("D2"):
            n = [int(rng.integers(128, 700)), int(rng.integers(8, 160))]
        else:
            n = [int(rng.integers(128, 220)), int(rng.integers(3, 24)), int(rng.integers(3, 12))]
        out.append((lat, n, storage, float(rng.choice([0.8, 1.6, 2.4] if lat != "D2Q5" and lat != "D3Q7" else [0.8, 1.6])),
                    float(rng.uniform(0.0, 0.9)), int(rng.integers(0, 5))))
    return out


@pytest.mark.parametrize("lat,n,storage,dt,theta,depth", _random_cases(16))
def test_theta_random_shapes(mm, lat, n, storage, dt, theta, depth):
    # seeded random lattices, storages, ragged grids, theta, time steps and fused-sweep depths
    rng = np.random.default_rng(zlib.crc32(repr((lat, n, storage, theta)).encode()))
    kw, prob = theta_case(lat, n, storage, dt, theta)
    L0 = smooth_level(prob, rng)
    s = mm.Solver(mm.make_desc(**kw, temporal_depth=depth))
    try:
        s.set_fields(L0)
        s.step(3)
        got = s.fields()
    finally:
        s.close()
    want = orc.theta_run(prob, L0, 3, theta)
    tol = 1e-12 if storage == "fp64" else 1e-5
    assert G.rel_err(got, want) <= tol, (lat, n, storage, dt, theta, depth, G.rel_err(got, want))
