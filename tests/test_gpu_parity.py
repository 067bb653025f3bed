"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances (relative to the field's max |value|): FP64 storage 1e-12; FP32 storage 1e-5;
BF16-offset storage: within one bf16 ulp of the offset (one step from bf16-exact input).
"""
import numpy as np
import pytest

import gpu_cases as G
from oracle import fourier as F
from oracle import oracle as orc
from oracle import params as P
from paper_2505_17057_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_17057_gb300 import mmfd
    return mmfd


def run_gpu(mm, kw, level0, level1=None, steps=1, **extra):
    d = mm.make_desc(**{**kw, **extra})
    s = mm.Solver(d)
    try:
        s.set_fields(level0)
        if level1 is not None:
            s.set_fields(level1, level=1)
        stored0 = s.fields(0)
        stored1 = s.fields(1) if kw["levels"] == 3 else None
        s.step(steps)
        out = s.fields(0)
        prev = s.fields(1) if kw["levels"] == 3 else None
    finally:
        s.close()
    return stored0, stored1, out, prev


SIZES_2D = [[300, 70], [67, 45]]
SIZES_3D = [[70, 37, 21], [150, 21, 9]]


@pytest.mark.parametrize("lat,pde,levels", G.SUPPORTED)
def test_parity_fp64(mm, lat, pde, levels):
    rng = np.random.default_rng(G.RNG_SEED)
    sizes = SIZES_2D if G.dims(lat) == 2 else SIZES_3D
    for n in sizes:
        kw, prob = G.case(lat, pde, levels, n, "fp64")
        L0 = G.random_level(prob, rng)
        L1 = G.random_level(prob, rng) if levels == 3 else None
        _, _, out, prev = run_gpu(mm, kw, L0, L1, steps=3)
        ref, refprev = orc.run(prob, L0, L1, nsteps=3)
        assert G.rel_err(out, ref) < 1e-12, (n, G.rel_err(out, ref))
        if levels == 3:
            assert G.rel_err(prev, refprev) < 1e-12


@pytest.mark.parametrize("lat,pde,levels", G.SUPPORTED)
def test_parity_fp32(mm, lat, pde, levels):
    rng = np.random.default_rng(G.RNG_SEED + 1)
    n = SIZES_2D[0] if G.dims(lat) == 2 else SIZES_3D[1]
    kw, prob = G.case(lat, pde, levels, n, "fp32")
    L0 = G.random_level(prob, rng)
    L1 = G.random_level(prob, rng) if levels == 3 else None
    s0, s1, out, _ = run_gpu(mm, kw, L0, L1, steps=3)
    # the oracle starts from the values the FP32 storage actually holds
    ref, _ = orc.run(prob, s0, s1, nsteps=3)
    assert G.rel_err(out, ref) < 1e-5, G.rel_err(out, ref)


@pytest.mark.parametrize("lat,pde,levels", [("D2Q9", "NSE", 2), ("D2Q9", "NCDE", 3), ("D2Q5", "LCDE", 2),
                                            ("D3Q19", "NSE", 2), ("D3Q7", "LCDE", 2)])
@pytest.mark.parametrize("sr", [False, True])
def test_parity_bf16_one_step(mm, lat, pde, levels, sr):
    rng = np.random.default_rng(G.RNG_SEED + 2)
    n = [260, 33] if G.dims(lat) == 2 else [140, 13, 7]
    kw, prob = G.case(lat, pde, levels, n, "bf16")
    refs = [1.0 if (pde == "NSE" and f == 0) else 0.0 for f in range(prob.nf)]
    L0 = G.random_level(prob, rng)
    L1 = G.random_level(prob, rng) if levels == 3 else None
    flags = mm.MMFD_FLAG_STOCHASTIC_ROUND if sr else 0
    s0, s1, out, _ = run_gpu(mm, kw, L0, L1, steps=1, flags=flags, ref=refs)
    ref, _ = orc.run(prob, s0, s1, nsteps=1)
    for f in range(prob.nf):
        off = ref[f] - refs[f]
        tol = G.bf16_ulp(off) + 2e-6 * (1 + np.abs(ref[f]))
        assert np.all(np.abs(out[f] - ref[f]) <= tol), (f, np.abs(out[f] - ref[f]).max())
    if not sr:
        # nearest rounding: the stored value is the bf16 rounding of the exact update in all but a few
        # nodes where the FP32 arithmetic lands on the other side of a rounding tie
        for f in range(prob.nf):
            hit = np.mean(out[f] == G.bf16_round(ref[f], refs[f]))
            assert hit > 0.99, (f, hit)


@pytest.mark.parametrize("n", [[1, 7], [5, 1], [2, 3], [1, 1], [3, 2]])
@pytest.mark.parametrize("lat,pde", [("D2Q9", "NSE"), ("D2Q9", "LCDE"), ("D2Q5", "LCDE"), ("D2Q9", "NCDE")])
def test_degenerate_2d_sizes(mm, n, lat, pde):
    rng = np.random.default_rng(7)
    kw, prob = G.case(lat, pde, 2, n, "fp64")
    L0 = G.random_level(prob, rng)
    _, _, out, _ = run_gpu(mm, kw, L0, None, steps=4)
    ref, _ = orc.run(prob, L0, None, nsteps=4)
    assert G.rel_err(out, ref) < 1e-12


@pytest.mark.parametrize("n", [[1, 1, 3], [4, 1, 2], [2, 3, 1], [5, 4, 3]])
@pytest.mark.parametrize("lat,pde", [("D3Q19", "NSE"), ("D3Q7", "LCDE")])
def test_degenerate_3d_sizes(mm, n, lat, pde):
    rng = np.random.default_rng(8)
    kw, prob = G.case(lat, pde, 2, n, "fp64")
    L0 = G.random_level(prob, rng)
    _, _, out, _ = run_gpu(mm, kw, L0, None, steps=3)
    ref, _ = orc.run(prob, L0, None, nsteps=3)
    assert G.rel_err(out, ref) < 1e-12


def test_config1_discrete_exact(mm):
    # 64x64 periodic LCDE, Gaussian hill sigma = 6, 200 steps, FP64: D2Q5 (K_xy dropped) and D2Q9
    # against the exact discrete solution lambda^n (Eq. (TforMMFD-7)) and the oracle.
    K = [[0.02, 0.005], [0.005, 0.01]]
    u = [0.1, 0.05]
    phi0 = inputs.gaussian_hill_2d(64, 64, 32, 32, 6.0)
    for lat in ("D2Q5", "D2Q9"):
        flags = mm.MMFD_FLAG_DROP_OFFDIAG if lat == "D2Q5" else 0
        kw = dict(pde="LCDE", lattice=lat, levels=2, n=[64, 64], dt=1.0, dx=[1, 1], K=K, u=u, storage="fp64",
                  targets=[0, -1, -1, 0, 0.5], flags=flags)
        _, _, out, _ = run_gpu(mm, kw, [phi0], None, steps=200)
        Kp = K if lat == "D2Q9" else [[0.02, 0], [0, 0.01]]
        prob = P.problem_lcde(lat, 2, [64, 64], 1.0, [1, 1], Kp, u, P.two_level_from_a0(0.0))
        ex = F.discrete_exact(prob, phi0, 200)
        assert np.abs(out[0] - ex).max() < 1e-12
        ref, _ = orc.run(prob, [phi0], None, nsteps=200)
        assert np.abs(out[0] - ref[0]).max() < 1e-12 * np.abs(ref[0]).max()


def test_three_level_equilibrium_start(mm):
    # setting level 0 only starts the three-level scheme from phi^{-1} := phi^0
    rng = np.random.default_rng(11)
    kw, prob = G.case("D2Q9", "NCDE", 3, [40, 30], "fp64")
    L0 = G.random_level(prob, rng)
    _, _, out, _ = run_gpu(mm, kw, L0, None, steps=5)
    ref, _ = orc.run(prob, L0, L0, nsteps=5)
    assert G.rel_err(out, ref) < 1e-12


def test_conservation_gpu(mm):
    # A_00 = 1: sum phi conserved (two- and three-level with sum ahat = 0); NSE also sum u
    rng = np.random.default_rng(12)
    for lat, pde, levels in [("D2Q9", "NCDE", 3), ("D2Q9", "NSE", 2), ("D3Q19", "NSE", 2), ("D2Q5", "LCDE", 2)]:
        n = [130, 66] if G.dims(lat) == 2 else [34, 18, 10]
        kw, prob = G.case(lat, pde, levels, n, "fp64")
        d = mm.make_desc(**kw)
        s = mm.Solver(d)
        L0 = G.random_level(prob, rng)
        s.set_fields(L0)
        before = s.reduce(mm.MMFD_RED_SUM)
        s.step(25)
        after = s.reduce(mm.MMFD_RED_SUM)
        scale = [np.abs(f).sum() for f in L0]
        for b, a, sc in zip(before, after, scale):
            assert abs(a - b) < 1e-12 * sc
        s.close()


@pytest.mark.parametrize("nx,storage", [(123, "fp32"), (128, "fp32"), (128, "bf16"), (128, "fp64")])
def test_reductions_match_numpy(mm, nx, storage):
    # nx = 128 takes the reduction's four-wide vector loads, nx = 123 the scalar ones; FP32 and
    # BF16 levels hold offsets from the density's reference rho0 = 1, which both must add back
    rng = np.random.default_rng(13)
    kw, prob = G.case("D2Q9", "NSE", 2, [nx, 77], storage)
    d = mm.make_desc(**kw)
    s = mm.Solver(d)
    s.set_fields(G.random_level(prob, rng))
    s.step(3)
    f = s.fields(0)
    sums = s.reduce(mm.MMFD_RED_SUM)
    mx = s.reduce(mm.MMFD_RED_MAXABS)
    for i in range(3):
        assert abs(sums[i] - f[i].sum()) < 1e-9 * np.abs(f[i]).sum()
        assert mx[i] == np.abs(f[i]).max()
    assert s.reduce(mm.MMFD_RED_NONFINITE)[0] == 0
    refv = f[1] + 1e-3 * rng.standard_normal(f[1].shape)
    gre, emax, rmax = s.error_norms(refv, field=1)
    assert abs(gre - np.abs(f[1] - refv).sum() / np.abs(refv).sum()) < 1e-9
    assert abs(emax - np.abs(f[1] - refv).max()) < 1e-12
    s.close()


def test_determinism_and_resume(mm):
    # bitwise identical reruns; n steps == n/2, export both levels, new solver, import, n/2
    rng = np.random.default_rng(14)
    kw, prob = G.case("D2Q9", "NCDE", 3, [200, 90], "fp32")
    L0 = G.random_level(prob, rng)
    L1 = G.random_level(prob, rng)
    _, _, a, _ = run_gpu(mm, kw, L0, L1, steps=40)
    _, _, b, _ = run_gpu(mm, kw, L0, L1, steps=40)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    d = mm.make_desc(**kw)
    s = mm.Solver(d)
    s.set_fields(L0)
    s.set_fields(L1, level=1)
    s.step(20)
    c0 = s.fields(0)
    c1 = s.fields(1)
    s.close()
    s2 = mm.Solver(mm.make_desc(**kw))
    s2.set_fields(c0)
    s2.set_fields(c1, level=1)
    s2.step(20)
    r = s2.fields(0)
    s2.close()
    assert all(np.array_equal(x, y) for x, y in zip(a, r))


def test_bounded_wait_reports_timeout(mm):
    # a wait that can never complete gives up after its budget and reports MMFD_ERR_TIMEOUT;
    # the context remains usable for a normal solve afterwards
    import torch
    s = torch.cuda.Stream()
    rc = mm.mmfd_selftest_wait_timeout(s.cuda_stream, 2_000_000)
    assert rc == mm.MMFD_ERR_TIMEOUT
    rng = np.random.default_rng(15)
    kw, prob = G.case("D2Q9", "NSE", 2, [140, 20], "fp64")
    L0 = G.random_level(prob, rng)
    _, _, out, _ = run_gpu(mm, kw, L0, None, steps=2)
    ref, _ = orc.run(prob, L0, None, nsteps=2)
    assert G.rel_err(out, ref) < 1e-12
