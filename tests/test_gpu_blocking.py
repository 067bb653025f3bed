"""GPU parity of the temporally blocked 2D path (two-level LCDE / NCDE, several steps per
launch): the blocked solver against the FP64 oracle and against the unblocked solver.

Tolerances as in the unblocked parity tests: FP64 1e-12, FP32 1e-5 relative to max |value|.
BF16: a blocked solver rounds to BF16 once per T steps, so T steps from a BF16-exact start
land within one bf16 ulp of the exact T-step update.
"""
import numpy as np
import pytest

import gpu_cases as G
from oracle import oracle as orc

pytestmark = pytest.mark.gpu

CASES = [("D2Q5", "LCDE"), ("D2Q9", "LCDE"), ("D2Q9", "NCDE")]
# ragged strips (nx not a multiple of the 120-column strip), the smallest grids the blocked
# kernel accepts (nx = 128, ny = 2T), and a grid taller than one item
SIZES = [[300, 70], [128, 8], [517, 131], [241, 37]]


@pytest.fixture(scope="module")
def mm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_17057_gb300 import mmfd
    return mmfd


def solve(mm, kw, L0, steps, depth, **extra):
    s = mm.Solver(mm.make_desc(**kw, temporal_depth=depth, **extra))
    try:
        info = s.get_info()
        s.set_fields(L0)
        stored = s.fields(0)
        s.step(steps)
        out = s.fields(0)
    finally:
        s.close()
    return info, stored, out


@pytest.mark.parametrize("lat,pde", CASES)
def test_blocked_fp64_matches_oracle(mm, lat, pde):
    rng = np.random.default_rng(G.RNG_SEED + 40)
    for n in SIZES:
        if n[1] < 4:
            continue
        kw, prob = G.case(lat, pde, 2, n, "fp64")
        L0 = G.random_level(prob, rng)
        # 5 steps = two blocked launches of depth 2 and one unblocked step
        info, _, out = solve(mm, kw, L0, 5, 2)
        assert info.temporal_depth == 2 and info.kernel.decode() == "k_march2d_tb", n
        ref, _ = orc.run(prob, L0, None, nsteps=5)
        assert G.rel_err(out, ref) < 1e-12, (n, G.rel_err(out, ref))


@pytest.mark.parametrize("depth", [2, 3, 4])
@pytest.mark.parametrize("lat,pde", CASES)
def test_blocked_fp32_matches_oracle_and_unblocked(mm, lat, pde, depth):
    rng = np.random.default_rng(G.RNG_SEED + 41 + depth)
    for n in SIZES:
        if n[1] < 2 * depth:
            continue
        kw, prob = G.case(lat, pde, 2, n, "fp32")
        L0 = G.random_level(prob, rng)
        steps = 2 * depth + 1
        info, stored, out = solve(mm, kw, L0, steps, depth)
        assert info.temporal_depth == depth and info.kernel.decode() == "k_march2d_tb", n
        ref, _ = orc.run(prob, stored, None, nsteps=steps)
        assert G.rel_err(out, ref) < 1e-5, (n, G.rel_err(out, ref))
        _, _, plain = solve(mm, kw, L0, steps, 1)
        assert G.rel_err(out, plain) < 1e-6, (n, G.rel_err(out, plain))


@pytest.mark.parametrize("depth", [3, 5])
@pytest.mark.parametrize("lat,pde", CASES)
def test_blocked_bf16_rounds_once_per_launch(mm, lat, pde, depth):
    rng = np.random.default_rng(G.RNG_SEED + 50 + depth)
    n = [260, 33]
    kw, prob = G.case(lat, pde, 2, n, "bf16")
    refs = [0.0]
    L0 = G.random_level(prob, rng)
    info, stored, out = solve(mm, kw, L0, depth, depth, ref=refs)
    assert info.temporal_depth == depth
    ref, _ = orc.run(prob, stored, None, nsteps=depth)
    tol = G.bf16_ulp(ref[0]) + 2e-6 * (1 + np.abs(ref[0]))
    assert np.all(np.abs(out[0] - ref[0]) <= tol), np.abs(out[0] - ref[0]).max()
    hit = np.mean(out[0] == G.bf16_round(ref[0], refs[0]))
    assert hit > 0.99, hit


def test_depth_selection(mm):
    kw, _ = G.case("D2Q9", "LCDE", 2, [300, 70], "fp32")
    s = mm.Solver(mm.make_desc(**kw, temporal_depth=9))
    assert s.get_info().temporal_depth == 4          # FP32 ghost columns hold 4 levels
    s.close()
    s = mm.Solver(mm.make_desc(**kw, temporal_depth=0))
    assert s.get_info().temporal_depth == 4
    s.close()
    kw64, _ = G.case("D2Q9", "LCDE", 2, [300, 70], "fp64")
    s = mm.Solver(mm.make_desc(**kw64, temporal_depth=0))
    assert s.get_info().temporal_depth == 2
    s.close()
    # the depth is clamped to what the rows allow (ny >= 2 T)
    kw7, _ = G.case("D2Q9", "LCDE", 2, [300, 7], "fp32")
    s = mm.Solver(mm.make_desc(**kw7, temporal_depth=4))
    assert s.get_info().temporal_depth == 3
    s.close()
    # unsupported: three-level, NSE, too few rows, narrow grids -> unblocked
    for args, depth in [(("D2Q9", "LCDE", 3, [300, 70]), 4), (("D2Q9", "NSE", 2, [300, 70]), 4),
                        (("D2Q9", "LCDE", 2, [300, 3]), 4), (("D2Q9", "LCDE", 2, [100, 70]), 4)]:
        kwu, _ = G.case(*args, "fp32")
        s = mm.Solver(mm.make_desc(**kwu, temporal_depth=depth))
        assert s.get_info().temporal_depth == 1, args
        s.close()


def test_blocked_conserves_mass(mm):
    # a_{-1} + a_0 + a_1 = 1 conserves sum(phi) for the LCDE (A_00 = 1); the blocked path keeps
    # it to FP64 rounding
    rng = np.random.default_rng(G.RNG_SEED + 60)
    kw, prob = G.case("D2Q9", "LCDE", 2, [517, 131], "fp64")
    L0 = G.random_level(prob, rng)
    s = mm.Solver(mm.make_desc(**kw, temporal_depth=2))
    try:
        s.set_fields(L0)
        m0 = s.reduce(mm.MMFD_RED_SUM)[0]
        s.step(40)
        m1 = s.reduce(mm.MMFD_RED_SUM)[0]
    finally:
        s.close()
    assert abs(m1 - m0) < 1e-12 * np.abs(L0[0]).sum()


# the lean He-Luo NSE (D2Q9, equal spacing, LBGK tau = 1: streaming momentum) has its own
# blocked kernel, k_march2d_tb_nse (three fields, depth 2 or 3)
def _lean_nse_case(n, storage):
    from oracle import params as P
    kw = dict(pde="NSE", lattice="D2Q9", levels=2, n=n, dt=1.0, dx=[1.0, 1.0], storage=storage,
              a=(1.0, 0.0, 0.0), abar=(1.0, 0.0, 0.0))
    prob = P.problem_nse("D2Q9", 2, n, 1.0, [1.0, 1.0], (1.0, 0.0, 0.0), (1.0, 0.0, 0.0))
    return kw, prob


@pytest.mark.parametrize("depth", [2, 3])
def test_blocked_lean_nse_fp32_matches_oracle_and_unblocked(mm, depth):
    # the blocked kernel runs the marching kernel's node update (lean_push_node2d) on the same
    # FP32 values: equal to the unblocked lean kernel to FP32 rounding (bit for bit on the 4096^2
    # benchmark grid and on these grids but 517 x 131, where nodes of the x-edge columns differ
    # by a few units in the last place of the stored offsets and spread from there)
    rng = np.random.default_rng(G.RNG_SEED + 70 + depth)
    for n in SIZES:
        if n[1] < 2 * depth:
            continue
        kw, prob = _lean_nse_case(n, "fp32")
        L0 = G.random_level(prob, rng)
        steps = 2 * depth + 1
        info, stored, out = solve(mm, kw, L0, steps, depth)
        assert info.temporal_depth == depth and info.kernel.decode() == "k_march2d_tb_nse", n
        ref, _ = orc.run(prob, stored, None, nsteps=steps)
        assert G.rel_err(out, ref) < 1e-5, (n, G.rel_err(out, ref))
        pinfo, _, plain = solve(mm, kw, L0, steps, 1)
        assert pinfo.kernel.decode() == "k_march2d_nse_s", n
        assert G.rel_err(out, plain) < 1e-6, (n, G.rel_err(out, plain))


@pytest.mark.parametrize("sr", [False, True])
def test_blocked_lean_nse_bf16_rounds_once_per_launch(mm, sr):
    rng = np.random.default_rng(G.RNG_SEED + 80)
    n = [260, 33]
    kw, prob = _lean_nse_case(n, "bf16")
    refs = [1.0, 0.0, 0.0]
    L0 = G.random_level(prob, rng)
    flags = mm.MMFD_FLAG_STOCHASTIC_ROUND if sr else 0
    info, stored, out = solve(mm, kw, L0, 3, 3, ref=refs, flags=flags)
    assert info.temporal_depth == 3 and info.kernel.decode() == "k_march2d_tb_nse"
    ref, _ = orc.run(prob, stored, None, nsteps=3)
    for f in range(3):
        tol = G.bf16_ulp(ref[f] - refs[f]) + 2e-6 * (1 + np.abs(ref[f]))
        assert np.all(np.abs(out[f] - ref[f]) <= tol), (f, np.abs(out[f] - ref[f]).max())


def test_blocked_lean_nse_depth_selection(mm):
    kw, _ = _lean_nse_case([300, 70], "fp32")
    for want, got in [(0, 3), (4, 3), (2, 2), (1, 1)]:
        s = mm.Solver(mm.make_desc(**kw, temporal_depth=want))
        info = s.get_info()
        s.close()
        assert info.temporal_depth == got, (want, info.temporal_depth)
        assert info.kernel.decode() == ("k_march2d_tb_nse" if got > 1 else "k_march2d_nse_s")
    # a general (non-streaming) momentum set keeps the unblocked kernel
    kwg = dict(kw, a=(0.95, 0.1, -0.05), abar=(0.9, 0.2, -0.1))
    s = mm.Solver(mm.make_desc(**kwg, temporal_depth=0))
    assert s.get_info().temporal_depth == 1
    s.close()
