"""GPU parity of the lean He-Luo NSE form of the marching kernels (k_march2d_nse_*, k_march3d_nse_*)
against the FP64 oracle and against the general pair form they replace.

The lean form applies with one speed on every axis on D2Q9 (any isotropic d_0) and on D3Q19
with d_0 = 1/3: there the uu terms of the EDF (Eq. (3-3)) reduce to |u|^2 and (e_p . u)^2, a+ and a- fold into the pair
parts, and when the momentum set is proportional to the scalar one (LBGK tau = 1) the momentum
contributions follow from the scalar ones.  Tolerances as in test_gpu_parity: FP32 storage 1e-5
relative to the field's max after three steps; BF16 one bf16 ulp of the offset after one step.
"""
import os

import numpy as np
import pytest

import gpu_cases as G
from oracle import oracle as orc
from oracle import params as P

pytestmark = pytest.mark.gpu

# (a, abar) per level count: LBGK tau = 1 (streaming momentum) and a general set (a_0 = 0.1,
# abar_0 = 0.2); three-level: the Example 2 set for rho with a momentum set that is not
# proportional to it, and the TRT special case at s- = 1.2 (proportional).
SETS = {
    ("s", 2): dict(a=(1.0, 0.0, 0.0), abar=(1.0, 0.0, 0.0)),
    ("g", 2): dict(a=(0.95, 0.1, -0.05), abar=(0.9, 0.2, -0.1)),
    ("g", 3): dict(a=G.THREE_A, ahat=G.THREE_AHAT, abar=(0.8, 0.0, 0.2), abarhat=(0.1, 0.0, -0.1)),
    ("s", 3): dict(a=(1.0, 0.0, -0.2), ahat=(0.0, 0.2, 0.0), abar=(1.0, 0.0, 0.2), abarhat=(0.0, -0.2, 0.0)),
}


@pytest.fixture(scope="module")
def mm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_17057_gb300 import mmfd
    return mmfd


def case(lat, mode, levels, n, storage, dt=1.0):
    dim = 2 if lat == "D2Q9" else 3
    co = SETS[(mode, levels)]
    kw = dict(pde="NSE", lattice=lat, levels=levels, n=n, dt=dt, dx=[1.0] * dim, storage=storage, **co)
    prob = P.problem_nse(lat, levels, n, dt, [1.0] * dim, co["a"], co["abar"], co.get("ahat", (0, 0, 0)),
                         co.get("abarhat", (0, 0, 0)))
    return kw, prob


def run(mm, kw, L0, L1=None, steps=3, force=None, **extra):
    old = os.environ.get("MMFD_FORCE_KERNEL")
    if force:
        os.environ["MMFD_FORCE_KERNEL"] = force
    try:
        s = mm.Solver(mm.make_desc(**{**kw, **extra}))
    finally:
        if force:
            if old is None:
                del os.environ["MMFD_FORCE_KERNEL"]
            else:
                os.environ["MMFD_FORCE_KERNEL"] = old
    try:
        kern = s.get_info().kernel.decode()
        s.set_fields(L0)
        if L1 is not None:
            s.set_fields(L1, level=1)
        s0 = s.fields(0)
        s1 = s.fields(1) if kw["levels"] == 3 else None
        s.step(steps)
        out = s.fields(0)
    finally:
        s.close()
    return kern, s0, s1, out


SHAPES = {"D2Q9": [[256, 37], [131, 5], [300, 1]], "D3Q19": [[128, 9, 5], [150, 21, 9], [131, 1, 3]]}


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
@pytest.mark.parametrize("mode,levels", [("s", 2), ("g", 2), ("g", 3), ("s", 3)])
def test_lean_fp32_vs_oracle(mm, lat, mode, levels):
    rng = np.random.default_rng(hash((lat, mode, levels)) % (1 << 31))
    for n in SHAPES[lat]:
        kw, prob = case(lat, mode, levels, n, "fp32")
        L0 = G.random_level(prob, rng)
        L1 = G.random_level(prob, rng) if levels == 3 else None
        kern, s0, s1, out = run(mm, kw, L0, L1)
        assert kern == f"k_march{len(n)}d_nse_{mode}", (kern, n)
        ref, _ = orc.run(prob, s0, s1, nsteps=3)
        assert G.rel_err(out, ref) < 1e-5, (n, G.rel_err(out, ref))


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
@pytest.mark.parametrize("mode,levels", [("s", 2), ("g", 3)])
@pytest.mark.parametrize("sr", [False, True])
def test_lean_bf16_one_step(mm, lat, mode, levels, sr):
    rng = np.random.default_rng(77 + levels)
    n = [260, 33] if lat == "D2Q9" else [140, 13, 7]
    kw, prob = case(lat, mode, levels, n, "bf16")
    refs = [1.0] + [0.0] * (prob.nf - 1)
    L0 = G.random_level(prob, rng)
    L1 = G.random_level(prob, rng) if levels == 3 else None
    flags = mm.MMFD_FLAG_STOCHASTIC_ROUND if sr else 0
    kern, s0, s1, out = run(mm, kw, L0, L1, steps=1, flags=flags, ref=refs)
    assert kern.endswith(f"_nse_{mode}"), kern
    ref, _ = orc.run(prob, s0, s1, nsteps=1)
    for f in range(prob.nf):
        tol = G.bf16_ulp(ref[f] - refs[f]) + 2e-6 * (1 + np.abs(ref[f]))
        assert np.all(np.abs(out[f] - ref[f]) <= tol), (f, np.abs(out[f] - ref[f]).max())


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
@pytest.mark.parametrize("mode,levels", [("s", 2), ("g", 2), ("g", 3), ("s", 3)])
def test_lean_matches_general_pair_form(mm, lat, mode, levels):
    # the same update as the general pair form, to FP32 rounding over ten steps
    rng = np.random.default_rng(11)
    n = [256, 24] if lat == "D2Q9" else [256, 24, 10]
    kw, prob = case(lat, mode, levels, n, "fp32")
    L0 = G.random_level(prob, rng)
    L1 = G.random_level(prob, rng) if levels == 3 else None
    k1, _, _, a = run(mm, kw, L0, L1, steps=10)
    k2, _, _, b = run(mm, kw, L0, L1, steps=10, force="generic")
    assert k1.endswith(f"_nse_{mode}") and k2 in ("k_march2d", "k_march3d"), (k1, k2)
    assert G.rel_err(a, b) < 2e-6, G.rel_err(a, b)


@pytest.mark.parametrize("mode", ["s", "g"])
def test_lean_d2q9_any_isotropic_d0(mm, mode):
    # on D2Q9 the lean shape holds for any isotropic d_0 (a diagonal pair spans both axes)
    rng = np.random.default_rng(23)
    n = [200, 30]
    co = SETS[(mode, 2)]
    kw = dict(pde="NSE", lattice="D2Q9", levels=2, n=n, dt=1.0, dx=[1.0, 1.0], storage="fp32", d0=[0.3, 0.3], **co)
    prob = P.problem_nse("D2Q9", 2, n, 1.0, [1.0, 1.0], co["a"], co["abar"], d0=[0.3, 0.3])
    L0 = G.random_level(prob, rng)
    kern, s0, _, out = run(mm, kw, L0)
    assert kern == f"k_march2d_nse_{mode}", kern
    ref, _ = orc.run(prob, s0, None, nsteps=3)
    assert G.rel_err(out, ref) < 1e-5, G.rel_err(out, ref)


# The 3D lean kernels stage 16-row tiles at one CTA per SM on large grids, 4-row tiles otherwise;
# MMFD_FORCE_KERNEL picks either on any grid.  Ragged shapes: partial x strips, partial 16-row
# tiles, one-row and few-plane grids.
WIDE_SHAPES = [[150, 21, 9], [131, 1, 3], [256, 40, 12], [130, 17, 33]]


@pytest.mark.parametrize("mode,levels", [("s", 2), ("g", 2), ("g", 3), ("s", 3)])
def test_lean3d_wide_tiles_fp32_vs_oracle(mm, mode, levels):
    rng = np.random.default_rng(hash(("wide", mode, levels)) % (1 << 31))
    for n in WIDE_SHAPES:
        kw, prob = case("D3Q19", mode, levels, n, "fp32")
        L0 = G.random_level(prob, rng)
        L1 = G.random_level(prob, rng) if levels == 3 else None
        kern, s0, s1, out = run(mm, kw, L0, L1, force="lean3d_rows16")
        assert kern == f"k_march3d_nse_{mode}", (kern, n)
        ref, _ = orc.run(prob, s0, s1, nsteps=3)
        assert G.rel_err(out, ref) < 1e-5, (n, G.rel_err(out, ref))


@pytest.mark.parametrize("mode,levels", [("s", 2), ("g", 3)])
@pytest.mark.parametrize("sr", [False, True])
def test_lean3d_wide_tiles_bf16_one_step(mm, mode, levels, sr):
    rng = np.random.default_rng(91 + levels)
    n = [140, 37, 7]
    kw, prob = case("D3Q19", mode, levels, n, "bf16")
    refs = [1.0] + [0.0] * (prob.nf - 1)
    L0 = G.random_level(prob, rng)
    L1 = G.random_level(prob, rng) if levels == 3 else None
    flags = mm.MMFD_FLAG_STOCHASTIC_ROUND if sr else 0
    kern, s0, s1, out = run(mm, kw, L0, L1, steps=1, force="lean3d_rows16", flags=flags, ref=refs)
    assert kern.endswith(f"_nse_{mode}"), kern
    ref, _ = orc.run(prob, s0, s1, nsteps=1)
    for f in range(prob.nf):
        tol = G.bf16_ulp(ref[f] - refs[f]) + 2e-6 * (1 + np.abs(ref[f]))
        assert np.all(np.abs(out[f] - ref[f]) <= tol), (f, np.abs(out[f] - ref[f]).max())


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_lean3d_wide_tiles_match_narrow(mm, storage):
    # the tile decides which warp computes a node, not the node's arithmetic: the two agree to
    # FP32 rounding over five steps (BF16: one step, within one bf16 ulp of the stored offset)
    rng = np.random.default_rng(5)
    n = [300, 37, 11]
    kw, prob = case("D3Q19", "s", 2, n, storage)
    extra = dict(ref=[1.0, 0.0, 0.0, 0.0]) if storage == "bf16" else {}
    L0 = G.random_level(prob, rng)
    steps = 5 if storage == "fp32" else 1
    _, _, _, a = run(mm, kw, L0, steps=steps, force="lean3d_rows16", **extra)
    _, _, _, b = run(mm, kw, L0, steps=steps, force="lean3d_rows4", **extra)
    if storage == "fp32":
        assert G.rel_err(a, b) < 1e-6, G.rel_err(a, b)
    else:
        for f in range(prob.nf):
            r = extra["ref"][f]
            tol = G.bf16_ulp(np.maximum(np.abs(a[f] - r), np.abs(b[f] - r)))
            assert np.all(np.abs(a[f] - b[f]) <= tol), (f, np.abs(a[f] - b[f]).max())


def test_lean3d_wide_bf16_ranges_crossing_tiles(mm):
    # 16-row BF16 tiles stream balanced ranges of (y tile, plane) pairs per group of strip CTAs;
    # on 300 x 50 x 120 (ragged strips and tiles) the ranges hold 9-10 planes and six of them run
    # from one y tile into the next.  One step against the oracle (one bf16 ulp) and against the
    # 4-row tiles (items of planes).
    rng = np.random.default_rng(404)
    n = [300, 50, 120]
    kw, prob = case("D3Q19", "s", 2, n, "bf16")
    refs = [1.0, 0.0, 0.0, 0.0]
    L0 = G.random_level(prob, rng)
    kern, s0, _, a = run(mm, kw, L0, steps=1, force="lean3d_rows16", ref=refs)
    assert kern == "k_march3d_nse_s", kern
    _, _, _, b = run(mm, kw, L0, steps=1, force="lean3d_rows4", ref=refs)
    ref, _ = orc.run(prob, s0, None, nsteps=1)
    for f in range(prob.nf):
        tol = G.bf16_ulp(ref[f] - refs[f]) + 2e-6 * (1 + np.abs(ref[f]))
        assert np.all(np.abs(a[f] - ref[f]) <= tol), (f, np.abs(a[f] - ref[f]).max())
        tab = G.bf16_ulp(np.maximum(np.abs(a[f] - refs[f]), np.abs(b[f] - refs[f])))
        assert np.all(np.abs(a[f] - b[f]) <= tab), (f, np.abs(a[f] - b[f]).max())
