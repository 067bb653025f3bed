"""Parity at the benchmark sizes, in the launch configuration bench.py times (same
descriptors, same kernels, the launcher's own tile choice): one step of the full grid on the
GPU, compared with the FP64 oracle on sampled nodes -- random interior nodes plus every
corner and samples of every edge row/column (and face) -- and, for the temporally blocked
path, with the unblocked GPU path on the whole grid (a property that holds at any size).

Tolerance: FP32 storage, 1e-5 relative to the field's max |value| (one step from the
FP32-rounded initial state, which is what the oracle is given); BF16-offset storage, one bf16
ulp of the stored offset (one step from the BF16-rounded state).
"""
import numpy as np
import pytest

from oracle import oracle as orc
from oracle import params as P
from paper_2505_17057_gb300 import configs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_17057_gb300 import mmfd
    return mmfd


def oracle_problem(kw):
    lat, n, dt, dx = kw["lattice"], kw["n"], kw["dt"], kw["dx"]
    if kw["pde"] == "NSE":
        return P.problem_nse(lat, 2, n, dt, dx, kw["a"], kw["abar"])
    a = P.two_level_from_a0(kw["targets"][0])
    return P.problem_lcde(lat, 2, n, dt, dx, np.asarray(kw["K"], dtype=float), kw["u"], a)


def sample_nodes(shape, rng, count=20000):
    """Flat indices (C order over `shape`, x fastest) of random nodes, all corners and
    samples of every boundary line / face."""
    shape = tuple(shape)
    idx = [rng.integers(0, int(np.prod(shape)), count)]
    dims = len(shape)
    for corner in np.ndindex(*([2] * dims)):
        c = tuple((s - 1) * b for s, b in zip(shape, corner))
        idx.append(np.array([np.ravel_multi_index(c, shape)]))
    for ax in range(dims):
        for side in (0, shape[ax] - 1):
            coords = [rng.integers(0, s, 500) for s in shape]
            coords[ax] = np.full(500, side)
            idx.append(np.ravel_multi_index(coords, shape))
    return np.unique(np.concatenate(idx))


def solve_one(mm, kw, fields, steps, depth):
    s = mm.Solver(mm.make_desc(**kw, temporal_depth=depth))
    try:
        info = s.get_info()
        s.set_fields(fields)
        stored = s.fields(0)
        s.step(steps)
        out = s.fields(0)
    finally:
        s.close()
    return info, stored, out


FULL = [("tgv2d", configs.tgv2d_4096, 4096, "k_march2d_nse_s"),
        ("lcde2d", configs.lcde2d_8192, 8192, "k_march2d"),
        ("cde3d", configs.cde3d_512, 512, "k_march3d"),
        ("nse3d", configs.nse3d_512, 512, "k_march3d_nse_s")]


@pytest.mark.parametrize("name,maker,n,kernel", FULL, ids=[f[0] for f in FULL])
def test_full_size_one_step_matches_oracle_on_samples(mm, name, maker, n, kernel):
    kw, fields, _ = maker(n=n, storage="fp32")
    info, stored, out = solve_one(mm, kw, fields, 1, 1)
    assert info.kernel.decode() == kernel
    prob = oracle_problem(kw)
    rng = np.random.default_rng(1234)
    nodes = sample_nodes(stored[0].shape, rng)
    ref = orc.step_nodes(prob, stored, None, nodes)
    for f in range(len(out)):
        got = out[f].reshape(-1)[nodes]
        scale = max(np.abs(ref[:, f]).max(), np.abs(out[f]).max())
        err = np.abs(got - ref[:, f]).max() / scale
        assert err < 1e-5, (name, f, err)
    assert all(np.isfinite(o).all() for o in out)


def test_full_size_blocked_matches_unblocked(mm):
    kw, fields, _ = configs.lcde2d_8192(n=8192, storage="fp32")
    info, _, blocked = solve_one(mm, kw, fields, 4, 4)
    assert info.kernel.decode() == "k_march2d_tb" and info.temporal_depth == 4
    _, _, plain = solve_one(mm, kw, fields, 4, 1)
    err = np.abs(blocked[0] - plain[0]).max() / np.abs(plain[0]).max()
    assert err < 1e-6, err


@pytest.mark.parametrize("depth", [2, 3])
def test_full_size_blocked_lean_nse_equals_unblocked(mm, depth):
    # the 4096^2 Taylor-Green vortex of the default benchmark, temporally blocked: the same bits
    # as the unblocked lean kernel after two launches
    kw, fields, _ = configs.tgv2d_4096(n=4096, storage="fp32")
    info, _, blocked = solve_one(mm, kw, fields, 2 * depth, depth)
    assert info.kernel.decode() == "k_march2d_tb_nse" and info.temporal_depth == depth
    _, _, plain = solve_one(mm, kw, fields, 2 * depth, 1)
    for f in range(3):
        assert np.array_equal(blocked[f], plain[f]), (f, np.abs(blocked[f] - plain[f]).max())


@pytest.mark.parametrize("lat,n", [("D2Q9", [65536, 32800]), ("D3Q7", [1300, 1300, 1300])])
def test_more_than_2_31_nodes(mm, lat, n):
    # node counts past 2^31 (every index in the kernels is 64-bit): one LCDE step of a single
    # Fourier mode phi0 = cos(theta . x), whose exact result is |lambda| cos(theta . x + arg lambda)
    # with the scheme's amplification factor lambda(theta) (Eq. (TforMMFD-3)), at sampled nodes
    # spread over the whole index range
    import torch
    from oracle import fourier as F
    dim = len(n)
    K = np.diag([0.02, 0.015, 0.01][:dim])
    u = [0.05, 0.03, 0.02][:dim]
    kw = dict(pde="LCDE", lattice=lat, levels=2, n=n, dt=1.0, dx=[1.0] * dim, K=K, u=u,
              targets=[0, -1, -1, 0, 0.5], storage="fp32")
    prob = P.problem_lcde(lat, 2, n, 1.0, [1.0] * dim, K, u, P.two_level_from_a0(0.0))
    modes = [3, 5, 2][:dim]
    theta = [2 * np.pi * m / nn for m, nn in zip(modes, n)]     # lattice axes x, y[, z]
    E, _, _ = orc.lattice(lat, prob.d0, prob.c)
    ub = F.ubar(prob)
    lam = sum(a * sum(ub[j] * np.exp(1j * k * sum(theta[ax] * E[j][ax] for ax in range(dim)))
                      for j in range(E.shape[0]))
              for k, a in zip((-1, 0, 1), prob.a))
    nodes = int(np.prod(n))
    assert nodes > 2 ** 31
    dev = torch.device("cuda")
    # phase of node (x, y[, z]) with x fastest, built plane by plane on the device
    field = torch.empty(nodes, dtype=torch.float32, device=dev)
    plane = n[0] * n[1]
    x = torch.arange(n[0], device=dev, dtype=torch.float64)
    y = torch.arange(n[1], device=dev, dtype=torch.float64)
    ph_xy = (theta[0] * x[None, :] + theta[1] * y[:, None]).reshape(-1)
    for z in range(n[2] if dim == 3 else 1):
        pz = theta[2] * z if dim == 3 else 0.0
        field[z * plane:(z + 1) * plane] = torch.cos(ph_xy + pz).to(torch.float32)
    shape = (n[1], n[0]) if dim == 2 else (n[2], n[1], n[0])
    s = mm.Solver(mm.make_desc(**kw))
    try:
        s.set_fields([field.view(shape)])
        s.step(1)
        out = s.fields(0, device=True, dtype=np.float32)[0].reshape(-1)
    finally:
        s.close()
    del field
    rng = np.random.default_rng(7)
    idx = np.unique(np.concatenate([rng.integers(0, nodes, 20000), [0, nodes - 1, 2 ** 31 - 1, 2 ** 31, 2 ** 31 + 1]]))
    got = out[torch.from_numpy(idx).to(dev)].double().cpu().numpy()
    xs = idx % n[0]
    ys = (idx // n[0]) % n[1]
    ph = theta[0] * xs + theta[1] * ys + (theta[2] * (idx // plane) if dim == 3 else 0.0)
    ref = np.abs(lam) * np.cos(ph + np.angle(lam))
    assert np.abs(got - ref).max() < 2e-6, np.abs(got - ref).max()


def bf16_ulp(x):
    """Spacing of bf16 numbers at |x| (8 significand bits)."""
    ax = np.maximum(np.abs(x), 1e-38)
    return 2.0 ** (np.floor(np.log2(ax)) - 7)


@pytest.mark.parametrize("name,maker,n,kernel", [FULL[0], FULL[3]], ids=["tgv2d", "nse3d"])
def test_full_size_bf16_one_step_matches_oracle_on_samples(mm, name, maker, n, kernel):
    # BF16-offset storage at the bench sizes, in the bench's launch configuration (on nse3d_512
    # the 16-row tiles with balanced per-group ranges, several of which run across y tiles):
    # within one bf16 ulp of the stored offset of the oracle's step from the stored state
    kw, fields, _ = maker(n=n, storage="bf16")
    info, stored, out = solve_one(mm, kw, fields, 1, 1)
    assert info.kernel.decode() == kernel
    if name == "nse3d":
        assert info.tile_rows == 16
    prob = oracle_problem(kw)
    rng = np.random.default_rng(4321)
    nodes = sample_nodes(stored[0].shape, rng)
    ref = orc.step_nodes(prob, stored, None, nodes)
    refs = kw["ref"]
    for f in range(len(out)):
        got = out[f].reshape(-1)[nodes]
        tol = bf16_ulp(ref[:, f] - refs[f]) + 2e-6 * (1 + np.abs(ref[:, f]))
        assert np.all(np.abs(got - ref[:, f]) <= tol), (name, f, np.abs(got - ref[:, f]).max())
