"""Synthetic request streams for the solve server (seeded; config 5 of the workload list).

Each request: PDE uniform over {CDE, NCDE, NSE}; 2D with p = 0.7 (side log-uniform in
[32, 1024]) else 3D (side log-uniform in [32, 128]); steps log-uniform in [100, 5000];
storage FP32 or BF16 with p = 1/2 (BF16 requests use stochastic rounding: with
round-to-nearest, the small per-step changes of the slow three-level NCDE solves stall in
BF16); parameters as the single-solve workloads; initial fields from seeded Fourier series.
Arrivals: Poisson at a given rate.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List

import numpy as np

from . import inputs

STOCHASTIC_ROUND = 0x4   # MMFD_FLAG_STOCHASTIC_ROUND of the C ABI


@dataclass
class Request:
    desc: dict
    fields: list
    steps: int
    nodes: int
    arrival: float = 0.0


def _smooth_2d(rng, n, nmodes=6):
    modes = inputs.draw_fourier_modes_2d(rng, nmodes, 4, 0.05, 0.2)
    return inputs.fourier_field_2d(modes, n, n)


def _smooth_3d(rng, n):
    s = [inputs.normalised_series(rng, n, 4) for _ in range(3)]
    f = [inputs.cos_series_eval(x, n) for x in s]
    return f[2][:, None, None] * f[1][None, :, None] * f[0][None, None, :]


def make_request(rng: inputs.SplitMix64, storage_mix: bool = True, steps_scale: float = 1.0,
                 min_steps: int = 100, max_steps: int = 5000) -> Request:
    pde = ["LCDE", "NCDE", "NSE"][rng.randint(0, 2)]
    two_d = rng.uniform() < 0.7
    if two_d:
        n = int(round(math.exp(rng.uniform(math.log(32), math.log(1024)))))
    else:
        n = int(round(math.exp(rng.uniform(math.log(32), math.log(128)))))
    steps = int(round(math.exp(rng.uniform(math.log(min_steps), math.log(max_steps))) * steps_scale))
    storage = "bf16" if (storage_mix and rng.uniform() < 0.5) else "fp32"
    if two_d:
        base = _smooth_2d(rng, n)
        if pde == "LCDE":
            desc = dict(pde="LCDE", lattice="D2Q9", levels=2, n=[n, n], dt=1.0, dx=[1.0, 1.0],
                        K=[[0.02, 0.005], [0.005, 0.01]], u=[0.1, 0.05], targets=[0, -1, -1, 0, 0.5],
                        storage=storage, ref=[1.0])
            fields = [1.0 + base]
        elif pde == "NCDE":
            dx = 2 * math.pi / n
            phi = 0.5 * base
            dmax = 0.01 * (1 + float(np.abs(phi).max()) ** 2)
            # diffusive limit of config 2, a convective one (|B'| dt / dx <= 0.2) for coarse grids,
            # and dt <= 0.5 D_min / max|B'|^2 (B' = phi, D_min = 0.01): without the last bound the
            # three-level central scheme is linearly unstable about the field's extreme states on
            # coarse grids (amplification up to 1.03 per step), which BF16 rounding noise exposes
            dt = min(0.4 * dx * dx / (2 * dmax), 0.2 * dx / max(1e-12, float(np.abs(phi).max())),
                     0.5 * 0.01 / max(1e-12, float(np.abs(phi).max()) ** 2))
            desc = dict(pde="NCDE", lattice="D2Q9", levels=3, n=[n, n], dt=dt, dx=[dx, dx],
                        flux=[[0, 0, 0.5, 0], [0, 0, 0.5, 0]], diff=[0.01, 0, 0.01, 0],
                        a=(7 / 8, 0.0, 1 / 8), ahat=(1 / 8, 0.0, -1 / 8), storage=storage)
            fields = [phi]
        else:
            u0 = min(100 * (1 / 6) / n, 0.05)  # Re 100, capped at Ma ~ 0.09 on coarse grids
            rho, u, v = inputs.taylor_green_2d(n, n, u0, 1 / 6, 0.0)
            desc = dict(pde="NSE", lattice="D2Q9", levels=2, n=[n, n], dt=1.0, dx=[1.0, 1.0],
                        a=(1.0, 0.0, 0.0), abar=(1.0, 0.0, 0.0), storage=storage, ref=[1.0, 0.0, 0.0])
            fields = [rho, u, v]
        nodes = n * n
    else:
        base = _smooth_3d(rng, n)
        if pde == "LCDE":
            desc = dict(pde="LCDE", lattice="D3Q7", levels=2, n=[n, n, n], dt=1.0, dx=[1.0, 1.0, 1.0],
                        K=np.diag([0.02, 0.015, 0.01]), u=[0.05, 0.03, 0.02], targets=[0, -1, -1, 0, 0.5],
                        storage=storage, ref=[1.0])
            fields = [1.0 + 0.5 * base]
        elif pde == "NCDE":
            dx = 2 * math.pi / n
            phi = 0.5 * base
            dmax = 0.01 * (1 + float(np.abs(phi).max()) ** 2)
            dt = min(0.3 * dx * dx / (2 * dmax), 0.15 * dx / max(1e-12, float(np.abs(phi).max())),
                     0.5 * 0.01 / max(1e-12, float(np.abs(phi).max()) ** 2))   # as in 2D
            desc = dict(pde="NCDE", lattice="D3Q19", levels=3, n=[n, n, n], dt=dt, dx=[dx, dx, dx],
                        flux=[[0, 0, 0.5, 0]] * 3, diff=[0.01, 0, 0.01, 0],
                        a=(7 / 8, 0.0, 1 / 8), ahat=(1 / 8, 0.0, -1 / 8), storage=storage)
            fields = [phi]
        else:
            g = _smooth_3d(rng, n)
            rho = np.ones_like(base)
            desc = dict(pde="NSE", lattice="D3Q19", levels=2, n=[n, n, n], dt=1.0, dx=[1.0, 1.0, 1.0],
                        a=(1.0, 0.0, 0.0), abar=(1.0, 0.0, 0.0), storage=storage, ref=[1.0, 0.0, 0.0, 0.0])
            fields = [rho, 0.03 * base, 0.03 * g, 0.03 * np.transpose(base, (1, 2, 0))]
        nodes = n * n * n
    if storage == "bf16":
        desc["flags"] = STOCHASTIC_ROUND
    return Request(desc, fields, steps, nodes)


def make_stream(count: int, seed: int = 5, storage_mix: bool = True, steps_scale: float = 1.0) -> List[Request]:
    rng = inputs.SplitMix64(inputs.SEED_BASE + 4 + (seed << 32))
    return [make_request(rng, storage_mix, steps_scale) for _ in range(count)]


def poisson_arrivals(count: int, rate: float, seed: int = 5) -> np.ndarray:
    rng = inputs.SplitMix64(inputs.SEED_BASE + 4 + ((seed + 1) << 32))
    t, out = 0.0, []
    for _ in range(count):
        u = rng.uniform()
        t += -math.log(1.0 - u) / rate
        out.append(t)
    return np.array(out)
