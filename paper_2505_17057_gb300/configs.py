"""The benchmark and test workloads, stated as physical problems (sizes, PDE parameters,
scheme design targets) -- the same description feeds the CUDA path and the oracle.

Workload recipe (seeded, synthetic; the paper uses analytic test problems, no datasets):
  cde2d_64        64x64 periodic linear CDE, u = (0.1, 0.05), K = [[0.02, 0.005], [0.005, 0.01]],
                  Gaussian hill sigma = 6 cells, 200 steps, FP64, lattice units; D2Q5 (K_xy dropped)
                  and D2Q9 (full K).
  ncde2d_1024     1024x1024 periodic NCDE on [0, 2 pi)^2, B(phi) = (phi^2/2)(1, 1),
                  D(phi) = 0.01 (1 + phi^2), D2Q9 three-level (a_{-1}, a_0, a_1) = (7/8, 0, 1/8),
                  (ahat) = (1/8, 0, -1/8); phi0 = 32 seeded Fourier modes, amplitudes U(0.1, 0.5);
                  dt = 0.4 dx^2 / (2 D(max |phi0|)); 10k steps; FP32.
  lcde2d_8192     8192x8192 periodic linear CDE on D2Q9 (the scalar bandwidth probe), u and K as in
                  cde2d_64, two-level, targets (a_0, A10, A11, A21, A22) = (0, -1, -1, 0, 0.5),
                  phi0 = 1 + 32 seeded Fourier modes (amplitudes U(0.1, 0.5)); FP32.
  tgv2d_4096      4096x4096 periodic He-Luo NSE, D2Q9 two-level, a_0 = abar_0 = 0 (LBGK tau = 1,
                  nu = 1/6), Taylor-Green vortex with u0 = Re nu / N, Re = 100 or 1000; FP32 or BF16.
  cde3d_512       512^3 linear CDE on D3Q7, u = (0.05, 0.03, 0.02), K = diag(0.02, 0.015, 0.01),
                  phi0 = 1 + 0.5 Sx Sy Sz (16-mode seeded cosine series), 1k steps.
  nse3d_512       512^3 He-Luo NSE on D3Q19, LBGK tau = 1, rho0 = 1, divergence-free seeded
                  velocity with max |u| = 0.05, 1k steps.
  theta2d_4096    lcde2d_8192's LCDE and initial field on 4096^2, two-level theta-scheme (Eq. (GCN))
                  with theta = 1/2 (Crank-Nicolson) at dt = 8, a step at which the explicit scheme
                  (theta = 1) is unstable on this grid; FP32.
  srccde2d_4096   Example 1 (isotropic CDE with the time-dependent source R) scaled to 4096^2 on the
                  periodic [0, 2]^2: D2Q9 three-level Case 3 (a = (7/8, 0, 1/8), ahat = (1/8, 0, -1/8)),
                  b_{-1} = 3/2, bhat_{-1} = -1/2, F_j = w_j R (1 + c_j.u/c_s^2), u = (0.1, 0.1),
                  kappa = 0.01, dt = 1 / (0.06 N_x^2) with N_x = n / 2 (Example 1's N_t / N_x^2);
                  phi at t = 0 and -dt from the exact solution; FP32.
"""
from __future__ import annotations

import math

import numpy as np

from . import inputs

CONFIG_INDEX = {"cde2d_64": 0, "ncde2d_1024": 1, "lcde2d_8192": 1, "tgv2d_4096": 2, "cde3d_512": 3, "nse3d_512": 3,
                "serve": 4, "srccde2d_4096": 1, "theta2d_4096": 1}

NU_LBGK = 1.0 / 6.0          # -(Abar_22 / Abar_10) dt c_s^2 with a_0 = 0, c_s^2 = 1/3
THREE_LEVEL_A = (7 / 8, 0.0, 1 / 8)
THREE_LEVEL_AHAT = (1 / 8, 0.0, -1 / 8)


def cde2d_64(lattice: str = "D2Q9"):
    K = [[0.02, 0.005], [0.005, 0.01]]
    u = [0.1, 0.05]
    phi0 = inputs.gaussian_hill_2d(64, 64, 32, 32, 6.0)
    desc = dict(pde="LCDE", lattice=lattice, levels=2, n=[64, 64], dt=1.0, dx=[1.0, 1.0], K=K, u=u,
                targets=[0, -1, -1, 0, 0.5], storage="fp64")
    return desc, [phi0], 200


def ncde2d_1024(n: int = 1024, storage: str = "fp32"):
    rng = inputs.rng_for(CONFIG_INDEX["ncde2d_1024"])
    modes = inputs.draw_fourier_modes_2d(rng, 32, 8, 0.1, 0.5)
    phi0 = inputs.fourier_field_2d(modes, n, n)
    dx = 2 * math.pi / n
    dmax = 0.01 * (1 + float(np.abs(phi0).max()) ** 2)
    dt = 0.4 * dx * dx / (2 * dmax)
    desc = dict(pde="NCDE", lattice="D2Q9", levels=3, n=[n, n], dt=dt, dx=[dx, dx],
                flux=[[0, 0, 0.5, 0], [0, 0, 0.5, 0]], diff=[0.01, 0, 0.01, 0],
                a=THREE_LEVEL_A, ahat=THREE_LEVEL_AHAT, storage=storage)
    return desc, [phi0], 10000


def lcde2d_8192(n: int = 8192, storage: str = "fp32"):
    rng = inputs.rng_for(CONFIG_INDEX["lcde2d_8192"])
    modes = inputs.draw_fourier_modes_2d(rng, 32, 8, 0.1, 0.5)
    phi0 = 1.0 + inputs.fourier_field_2d(modes, n, n)
    desc = dict(pde="LCDE", lattice="D2Q9", levels=2, n=[n, n], dt=1.0, dx=[1.0, 1.0],
                K=[[0.02, 0.005], [0.005, 0.01]], u=[0.1, 0.05], targets=[0, -1, -1, 0, 0.5],
                storage=storage, ref=[1.0])
    return desc, [phi0], 1000


def theta2d_4096(n: int = 4096, storage: str = "fp32", theta: float = 0.5, dt: float = 8.0):
    rng = inputs.rng_for(CONFIG_INDEX["theta2d_4096"])
    modes = inputs.draw_fourier_modes_2d(rng, 32, 8, 0.1, 0.5)
    phi0 = 1.0 + inputs.fourier_field_2d(modes, n, n)
    desc = dict(pde="LCDE", lattice="D2Q9", levels=2, n=[n, n], dt=dt, dx=[1.0, 1.0],
                K=[[0.02, 0.005], [0.005, 0.01]], u=[0.1, 0.05], targets=[0, -1, -1, 0, 0.5],
                storage=storage, ref=[1.0], theta=theta)
    return desc, [phi0], 1000


def tgv2d_4096(n: int = 4096, re: float = 100.0, storage: str = "fp32"):
    u0 = re * NU_LBGK / n
    rho, u, v = inputs.taylor_green_2d(n, n, u0, NU_LBGK, 0.0)
    desc = dict(pde="NSE", lattice="D2Q9", levels=2, n=[n, n], dt=1.0, dx=[1.0, 1.0],
                a=(1.0, 0.0, 0.0), abar=(1.0, 0.0, 0.0), storage=storage, ref=[1.0, 0.0, 0.0])
    return desc, [rho, u, v], 5000


def tgv2d_reference(n: int, re: float, t: float):
    u0 = re * NU_LBGK / n
    return inputs.taylor_green_2d(n, n, u0, NU_LBGK, t)


def cde3d_512(n: int = 512, storage: str = "fp32"):
    phi0, _ = inputs.separable_scalar_3d(CONFIG_INDEX["cde3d_512"], n, n, n)
    desc = dict(pde="LCDE", lattice="D3Q7", levels=2, n=[n, n, n], dt=1.0, dx=[1.0, 1.0, 1.0],
                K=np.diag([0.02, 0.015, 0.01]), u=[0.05, 0.03, 0.02], targets=[0, -1, -1, 0, 0.5],
                storage=storage, ref=[1.0])
    return desc, [phi0], 1000


def nse3d_512(n: int = 512, storage: str = "fp32"):
    ux, uy, uz = inputs.solenoidal_velocity_3d(CONFIG_INDEX["nse3d_512"], n, n, n, 0.05)
    rho = np.ones_like(ux)
    desc = dict(pde="NSE", lattice="D3Q19", levels=2, n=[n, n, n], dt=1.0, dx=[1.0, 1.0, 1.0],
                a=(1.0, 0.0, 0.0), abar=(1.0, 0.0, 0.0), storage=storage, ref=[1.0, 0.0, 0.0, 0.0])
    return desc, [rho, ux, uy, uz], 1000


def srccde2d_4096(n: int = 4096, storage: str = "fp32"):
    """(desc, [phi(0)], [phi(-dt)], source) with source(m) = [R(x, m dt)] (Example 1)."""
    nx = n // 2
    dx = 2.0 / n
    dt = 1.0 / (0.06 * nx * nx)
    kappa = (dx / dt) ** 2 / 3.0 * dt / 2.0
    u = (0.1, 0.1)
    x = np.arange(n) * dx
    X, Y = np.meshgrid(x, x, indexing="xy")
    s_, c_ = np.sin(np.pi * (X + Y)), np.cos(np.pi * (X + Y))
    g = 1.0 - 2.0 * np.pi ** 2 * kappa
    desc = dict(pde="LCDE", lattice="D2Q9", levels=3, n=[n, n], dt=dt, dx=[dx, dx], K=np.eye(2) * kappa, u=list(u),
                a=THREE_LEVEL_A, ahat=THREE_LEVEL_AHAT, source="su", b=(1.5, 0.0, 0.0), bhat=(-0.5, 0.0, 0.0),
                storage=storage)
    base = s_ + np.pi * (u[0] + u[1]) * c_

    def source(m: int):
        return [np.exp(g * m * dt) * base]

    return desc, [s_.copy()], [np.exp(-g * dt) * s_], source
