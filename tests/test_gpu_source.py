"""GPU parity of the source terms (Eq. (2-1), F_j = g_j^eq(S, M_1F, 0) of Eq. (SourceF)): the
CUDA path through the C ABI against the oracle on the same seeded inputs, with a source that
changes every step (set before each step) and with a source that stays constant.  Tolerances
as elsewhere: FP64 1e-12, FP32 1e-5 relative to the field's max |value|; BF16 within one bf16
ulp after one step.  Example 1 (isotropic CDE with a time-dependent source) runs on the GPU
and converges at second order.
"""
import numpy as np
import pytest

import gpu_cases as G
from oracle import oracle as orc
from oracle import params as P

pytestmark = pytest.mark.gpu

B2 = (0.8, 0.1, 0.1)
B3, B3H = (1.2, 0.1, 0.2), (-0.4, 0.0, -0.1)


@pytest.fixture(scope="module")
def mm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_17057_gb300 import mmfd
    return mmfd


def source_case(lat, pde, levels, n, storage, source, b=None, bhat=None):
    kw, prob = G.case(lat, pde, levels, n, storage)
    b = b if b is not None else (B2 if levels == 2 else B3)
    bhat = bhat if bhat is not None else ((0.0, 0.0, 0.0) if levels == 2 else B3H)
    kw.update(source=source, b=b, bhat=bhat)
    prob.source, prob.b, prob.bhat = source, b, bhat
    return kw, prob


def src_fields(prob, rng):
    return [0.3 + 0.2 * rng.standard_normal(prob.shape) for _ in range(prob.nsrc)]


def run_both(mm, kw, prob, rng, steps, static=False, storage_round=None, kernels=None):
    """GPU and oracle runs with the same sources; returns (gpu, oracle).  The name of the step
    kernel that ran is added to `kernels`."""
    L0 = G.random_level(prob, rng)
    L1 = G.random_level(prob, rng) if prob.levels == 3 else None
    srcs = {m: src_fields(prob, rng) for m in range(-1, steps)}
    if static:
        for m in srcs:
            srcs[m] = srcs[0]
    s = mm.Solver(mm.make_desc(**kw, flags=mm.MMFD_FLAG_ALLOW_UNSTABLE))
    try:
        kern = s.get_info().kernel.decode()
        assert kern in ("k_direct_src", "k_march2d_src", "k_march3d_src"), kern
        if kernels is not None:
            kernels.add(kern)
        s.set_fields(L0)
        if L1 is not None:
            s.set_fields(L1, level=1)
        stored0 = s.fields(0)
        stored1 = s.fields(1) if prob.levels == 3 else None
        if static:
            s.set_source(srcs[0])             # level 1 follows before the first step
            s.step(steps)
        else:
            if prob.levels == 3:
                s.set_source(srcs[-1], level=1)
            for m in range(steps):
                s.set_source(srcs[m])
                s.step(1)
        out = s.fields(0)
    finally:
        s.close()
    rnd = storage_round or (lambda f: f)
    ref, _ = orc.run_source(prob, stored0, stored1, steps, lambda m: [rnd(f) for f in srcs[m]], form="central")
    return out, ref


CASES = [("D2Q5", "LCDE", 2, "s"), ("D2Q5", "LCDE", 3, "su"), ("D2Q9", "LCDE", 2, "su"), ("D2Q9", "LCDE", 3, "sm"),
         ("D2Q9", "NCDE", 2, "sm"), ("D2Q9", "NCDE", 3, "s"), ("D3Q7", "LCDE", 2, "sm"), ("D3Q7", "LCDE", 3, "su"),
         ("D3Q19", "LCDE", 2, "s"), ("D3Q19", "LCDE", 3, "su"), ("D3Q19", "NCDE", 2, "s"), ("D3Q19", "NCDE", 3, "sm")]


@pytest.mark.parametrize("lat,pde,levels,source", CASES)
def test_source_fp64_matches_oracle(mm, lat, pde, levels, source):
    rng = np.random.default_rng(G.RNG_SEED + 100)
    # ragged strips and tails on the marching kernels (nx >= 128), and the direct kernel
    sizes = [[300, 70], [517, 131], [67, 45]] if G.dims(lat) == 2 else [[150, 21, 9], [131, 13, 7], [40, 21, 9]]
    kernels = set()
    for n in sizes:
        kw, prob = source_case(lat, pde, levels, n, "fp64", source)
        out, ref = run_both(mm, kw, prob, rng, 4, kernels=kernels)
        assert G.rel_err(out, ref) < 1e-12, (n, G.rel_err(out, ref))
    march = "k_march2d_src" if G.dims(lat) == 2 else "k_march3d_src"
    assert kernels == {"k_direct_src", march}, kernels


@pytest.mark.parametrize("lat,pde,levels,source", [("D2Q9", "LCDE", 3, "su"), ("D2Q9", "NCDE", 2, "sm"),
                                                   ("D3Q19", "NCDE", 3, "s"), ("D3Q7", "LCDE", 2, "sm")])
def test_source_fp32_matches_oracle(mm, lat, pde, levels, source):
    rng = np.random.default_rng(G.RNG_SEED + 101)
    n = [300, 70] if G.dims(lat) == 2 else [150, 21, 9]
    kw, prob = source_case(lat, pde, levels, n, "fp32", source)
    f32 = lambda f: f.astype(np.float32).astype(np.float64)
    out, ref = run_both(mm, kw, prob, rng, 3, storage_round=f32)
    assert G.rel_err(out, ref) < 1e-5


def test_source_bf16_one_step(mm):
    rng = np.random.default_rng(G.RNG_SEED + 102)
    kw, prob = source_case("D2Q9", "LCDE", 2, [260, 33], "bf16", "su")
    f32 = lambda f: f.astype(np.float32).astype(np.float64)
    out, ref = run_both(mm, kw, prob, rng, 1, storage_round=f32)
    tol = G.bf16_ulp(ref[0]) + 2e-6 * (1 + np.abs(ref[0]))
    assert np.all(np.abs(out[0] - ref[0]) <= tol)


@pytest.mark.parametrize("levels", [2, 3])
def test_static_source(mm, levels):
    # a source set once stays constant: level 1 follows level 0 before the first step, and
    # every later step reuses it
    rng = np.random.default_rng(G.RNG_SEED + 103)
    kw, prob = source_case("D2Q9", "LCDE", levels, [300, 70], "fp64", "su")
    out, ref = run_both(mm, kw, prob, rng, 5, static=True)
    assert G.rel_err(out, ref) < 1e-12


def test_source_mass_balance(mm):
    # periodic grid: sum phi' = sum_k a_k sum phi + dt sum_k b_k sum S (LCDE, two-level)
    rng = np.random.default_rng(G.RNG_SEED + 104)
    kw, prob = source_case("D2Q9", "LCDE", 2, [517, 131], "fp64", "sm")
    L0 = G.random_level(prob, rng)
    S = src_fields(prob, rng)
    s = mm.Solver(mm.make_desc(**kw))
    try:
        s.set_fields(L0)
        s.set_source(S)
        m0 = s.reduce(mm.MMFD_RED_SUM)[0]
        s.step(10)
        m1 = s.reduce(mm.MMFD_RED_SUM)[0]
    finally:
        s.close()
    expect = m0 + 10 * prob.dt * sum(prob.b) * S[0].sum()
    assert abs(m1 - expect) < 1e-11 * np.abs(L0[0]).sum()


def test_source_api_errors(mm):
    kw, _ = G.case("D2Q9", "LCDE", 2, [64, 32], "fp64")
    s = mm.Solver(mm.make_desc(**kw))
    try:
        with pytest.raises(mm.MMFDError) as e:
            s.set_source([np.zeros((32, 64))])
        assert e.value.code == mm.MMFD_ERR_STATE
    finally:
        s.close()
    kw, _ = source_case("D2Q9", "LCDE", 2, [64, 32], "fp64", "s")
    s = mm.Solver(mm.make_desc(**kw))
    try:
        with pytest.raises(mm.MMFDError) as e:
            s.set_source([np.zeros((32, 64))], level=1)    # two-level: no level t - dt
        assert e.value.code == mm.MMFD_ERR_ARG
    finally:
        s.close()
    srv = mm.Server(1 << 28, max_slots=2, steps_per_tick=1)
    try:
        with pytest.raises(mm.MMFDError) as e:
            srv.submit(mm.make_desc(**kw), [np.zeros((32, 64))], 1)
        assert e.value.code == mm.MMFD_ERR_UNSUPPORTED
    finally:
        srv.close()


def _example1_gpu(mm, case, nxu, ntu):
    import test_oracle_source as TS
    dx, dt = 1.0 / nxu, 1.0 / ntu
    n = 2 * nxu
    c = dx / dt
    kappa = c * c / 3.0 * dt / 2.0
    u = (0.1, 0.1)
    a, ah = TS.EX1_CASES[case]
    kw = dict(pde="LCDE", lattice="D2Q9", levels=3, n=[n, n], dt=dt, dx=[dx, dx], storage="fp64",
              K=kappa * np.eye(2), u=list(u), a=a, ahat=ah, source="su", b=(1.5, 0, 0), bhat=(-0.5, 0, 0))
    x = np.arange(n) * dx
    X, Y = np.meshgrid(x, x, indexing="xy")
    g = 1.0 - 2.0 * np.pi ** 2 * kappa
    exact = lambda t: np.exp(g * t) * np.sin(np.pi * (X + Y))
    R = lambda m: [np.exp(g * m * dt) * (np.sin(np.pi * (X + Y)) + np.pi * (u[0] + u[1]) * np.cos(np.pi * (X + Y)))]
    s = mm.Solver(mm.make_desc(**kw))
    try:
        s.set_fields([exact(0.0)])
        s.set_fields([exact(-dt)], level=1)
        s.set_source(R(-1), level=1)
        for m in range(ntu):
            s.set_source(R(m))
            s.step(1)
        out = s.fields(0)[0]
    finally:
        s.close()
    ref = exact(1.0)
    return float(np.abs(out - ref).sum() / np.abs(ref).sum()), TS.example1_gre(case, nxu, ntu)


@pytest.mark.parametrize("case", [1, 2, 3])
def test_example1_on_gpu(mm, case):
    res = [_example1_gpu(mm, case, nx, nt) for nx, nt in [(10, 6), (20, 24), (40, 96)]]
    for gpu, oracle in res:
        assert abs(gpu - oracle) < 1e-9 * oracle
    orders = [np.log2(res[i][0] / res[i + 1][0]) for i in range(2)]
    assert all(o >= 1.8 for o in orders), orders


@pytest.mark.parametrize("lat,n", [("D2Q9", [517, 131]), ("D3Q19", [150, 21, 9])])
@pytest.mark.parametrize("storage,tol", [("fp32", 1e-6), ("bf16", 0.0)])
def test_march_source_matches_direct(mm, monkeypatch, storage, tol, lat, n):
    # the fused epilogue of the marching kernels against the one-node-per-thread kernel, on a
    # grid with ragged strips, from the same stored state
    rng = np.random.default_rng(G.RNG_SEED + 105)
    kw, prob = source_case(lat, "NCDE", 3, n, storage, "sm")
    L0 = G.random_level(prob, rng)
    L1 = G.random_level(prob, rng)
    S0, S1 = src_fields(prob, rng), src_fields(prob, rng)
    outs = {}
    for force in ("", "direct"):
        monkeypatch.setenv("MMFD_FORCE_KERNEL", force)
        s = mm.Solver(mm.make_desc(**kw, flags=mm.MMFD_FLAG_ALLOW_UNSTABLE))
        try:
            outs[force] = s.get_info().kernel.decode()
            s.set_fields(L0)
            s.set_fields(L1, level=1)
            s.set_source(S1, level=1)
            s.set_source(S0)
            s.step(1)
            outs[force + "f"] = s.fields(0)[0]
        finally:
            s.close()
    assert outs[""] == ("k_march2d_src" if len(n) == 2 else "k_march3d_src") and outs["direct"] == "k_direct_src"
    a, b = outs["f"], outs["directf"]
    if storage == "bf16":
        # the two kernels round FP32 sums taken in different orders: at most one ulp apart
        assert np.all(np.abs(a - b) <= G.bf16_ulp(b) + 1e-6 * np.abs(b))
    else:
        assert np.abs(a - b).max() <= tol * np.abs(b).max()


@pytest.mark.parametrize("n", [[1, 7], [5, 1], [1, 1], [2, 3, 1], [1, 1, 3]])
def test_source_degenerate_grids(mm, n):
    # grids one node wide in some direction: every neighbour is a periodic image of the node
    rng = np.random.default_rng(G.RNG_SEED + 106)
    lat = "D2Q9" if len(n) == 2 else "D3Q19"
    kw, prob = source_case(lat, "LCDE", 3, n, "fp64", "sm")
    out, ref = run_both(mm, kw, prob, rng, 3)
    assert G.rel_err(out, ref) < 1e-12


def test_source_full_size_on_samples(mm):
    # the benchmark workload (Example 1's CDE with a time-dependent source at 4096^2, FP32) in the
    # bench's launch configuration: one step against the FP64 oracle on sampled nodes
    from paper_2505_17057_gb300 import configs
    import test_gpu_fullsize as FS
    kw, f0, fm1, source = configs.srccde2d_4096(n=4096, storage="fp32")
    s = mm.Solver(mm.make_desc(**kw))
    try:
        assert s.get_info().kernel.decode() == "k_march2d_src"
        s.set_fields(f0)
        s.set_fields(fm1, level=1)
        st0, st1 = s.fields(0), s.fields(1)
        S0, Sm1 = [np.float32(x).astype(np.float64) for x in source(0)], [np.float32(x).astype(np.float64) for x in source(-1)]
        s.set_source(source(-1), level=1)
        s.set_source(source(0))
        s.step(1)
        out = s.fields(0)[0]
    finally:
        s.close()
    a, ah = kw["a"], kw["ahat"]
    prob = P.problem_lcde("D2Q9", 3, kw["n"], kw["dt"], kw["dx"], kw["K"], kw["u"], a, ah)
    prob.source, prob.b, prob.bhat = "su", kw["b"], kw["bhat"]
    nodes = FS.sample_nodes(st0[0].shape, np.random.default_rng(99))
    ref = orc.step_nodes(prob, st0, st1, nodes, src=(S0, Sm1))[:, 0]
    got = out.reshape(-1)[nodes]
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-5
