"""Robustness of the C ABI's host validation (no GPU): seeded random descriptors, including
non-finite, negative, huge and out-of-range values, go through mmfd_describe.  Every call must
come back with a status (no crash, no exception other than the binding's MMFDError), and every
accepted descriptor must resolve to finite derived constants."""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def mm():
    from paper_2505_17057_gb300 import build
    build.build()
    from paper_2505_17057_gb300 import mmfd
    return mmfd


def _wild(rng, scale=1.0):
    r = rng.random()
    if r < 0.05:
        return float("nan")
    if r < 0.08:
        return float("inf") * (1 if rng.random() < 0.5 else -1)
    if r < 0.12:
        return 0.0
    if r < 0.16:
        return -abs(rng.normal()) * scale
    if r < 0.19:
        return 10.0 ** rng.integers(6, 300)
    return float(rng.uniform(0.0, 2.0) * scale)


def _random_desc(mm, rng):
    d = mm.mmfd_desc_init()
    d.pde = int(rng.integers(-1, 5))
    d.lattice = int(rng.integers(-1, 5))
    d.levels = int(rng.choice([2, 3, 2, 3, 1, 4]))
    d.dim = int(rng.choice([2, 3, 2, 3, 1]))
    for i in range(3):
        d.n[i] = int(rng.choice([1, 2, 7, 64, 130, 0, -3, 1 << 21, 1 << 40]))
    d.dt = _wild(rng)
    for i in range(3):
        d.dx[i] = _wild(rng)
        d.d0[i] = _wild(rng, 0.5)
        d.u[i] = _wild(rng, 0.2)
        for j in range(3):
            d.K[i][j] = _wild(rng, 0.05)
    for i in range(3):
        for k in range(4):
            d.flux[i][k] = _wild(rng, 0.3)
    for k in range(4):
        d.diff[k] = _wild(rng, 0.05)
    d.rho0 = _wild(rng)
    d.coef_mode = int(rng.integers(-1, 3))
    for arr in (d.a, d.ahat, d.abar, d.abarhat):
        for i in range(3):
            arr[i] = _wild(rng, 0.7) * (1 if rng.random() < 0.7 else -1)
    for i in range(5):
        d.targets[i] = _wild(rng) * (1 if rng.random() < 0.6 else -1)
        d.targets_bar[i] = d.targets[i]
    d.storage = int(rng.integers(-1, 4))
    d.flags = int(rng.integers(0, 64))
    for f in range(4):
        d.ref[f] = _wild(rng)
    d.temporal_depth = int(rng.integers(-2, 9))
    d.source = int(rng.integers(-1, 5))
    for i in range(3):
        d.b[i] = _wild(rng) if rng.random() < 0.3 else 0.0
        d.bhat[i] = _wild(rng) if rng.random() < 0.2 else 0.0
    d.theta = _wild(rng, 0.6)
    return d


def test_describe_never_crashes(mm):
    rng = np.random.default_rng(424242)
    accepted = 0
    for _ in range(3000):
        d = _random_desc(mm, rng)
        try:
            info = mm.mmfd_describe(d)
        except mm.MMFDError as e:
            assert e.code < 0
            continue
        accepted += 1
        assert info.nf in (1, 3, 4)
        for v in (info.A10, info.A20, info.A21, info.A22, info.bytes_per_lu, *info.c, *info.cs2, *info.w):
            assert math.isfinite(v), v
    # nearly every wild descriptor carries some invalid field and is refused with a status;
    # accepted ones are covered by the test below
    assert accepted < 3000


def test_plausible_descriptors_resolve(mm):
    # small perturbations of valid problems: accepted ones resolve to finite constants and a
    # finite amplification bound
    rng = np.random.default_rng(7)
    ok = 0
    for _ in range(300):
        lat = ["D2Q5", "D2Q9", "D3Q7", "D3Q19"][rng.integers(4)]
        dim = 2 if lat.startswith("D2") else 3
        K = np.diag(rng.uniform(0.005, 0.1, dim))
        if lat in ("D2Q9", "D3Q19"):
            K = K + 0.002 * (1 - np.eye(dim))
        try:
            info = mm.mmfd_describe(mm.make_desc(
                "LCDE", lat, int(rng.choice([2, 3])), [int(rng.integers(1, 300)) for _ in range(dim)],
                float(rng.uniform(0.2, 3.0)), [float(v) for v in rng.uniform(0.5, 2.0, dim)], K=K,
                u=[float(v) for v in rng.uniform(-0.3, 0.3, dim)], targets=[float(rng.uniform(-1, 0.5)), -1, -1, 0.25, 0.5],
                storage=["fp64", "fp32", "bf16"][rng.integers(3)], flags=mm.MMFD_FLAG_ALLOW_UNSTABLE,
                theta=None if rng.random() < 0.7 else float(rng.uniform(0, 1)), temporal_depth=int(rng.integers(0, 6))))
        except mm.MMFDError as e:
            assert e.code < 0
            continue
        ok += 1
        assert math.isfinite(info.max_lambda) and info.max_lambda >= 0
    assert ok > 100, ok
