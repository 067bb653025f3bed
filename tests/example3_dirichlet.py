"""Example 3 of Sec. IV (the wave equation d_t^2 phi = (1/2) lap phi on [0, 1]^2, exact solution
exp(x + y + t)) as the paper runs it: N_x intervals per axis (N_x + 1 nodes), N_t = 2 N_x steps
to t = 1, the second time level from the paper's Taylor start-up formula, and Dirichlet values
from the exact solution on the boundary nodes after every step.  The error is the GRE over the
interior nodes at t = 1.

The steppers it drives are periodic.  Every interior node's stencil stays inside the domain
(its neighbours are interior or boundary nodes), and the boundary nodes, which alone see the
periodic wrap, are overwritten with exact values after each step, so a periodic step followed by
the overwrite is the Dirichlet scheme.
"""
import math

import numpy as np

from oracle import params as P

# (lattice, beta, gamma) of Cases 1-3; alpha = gamma beta c_s^2 = 1/2 with c_s^2 = c^2 / 3
CASES = {1: ("D2Q5", 1.0, 3 / 8), 2: ("D2Q9", 1.0, 3 / 8), 3: ("D2Q9", 3 / 4, 1 / 2)}


def problem(case, nx):
    """(oracle Problem, dx, dt, number of steps) of one Table 4 row."""
    lat, _, gamma = CASES[case]
    dx = 1.0 / nx
    nt = 2 * nx
    dt = 1.0 / nt
    a, ah = P.wave_coefficients(gamma)
    return P.problem_lwe(lat, [nx + 1, nx + 1], dt, [dx, dx], 0.5 * np.eye(2), a, ah), dx, dt, nt


def _grid(nx):
    g = np.arange(nx + 1) / nx
    return np.meshgrid(g, g, indexing="ij")      # (Y, X), numpy order (y, x)


def _with_boundary(f, exact):
    out = f.copy()
    out[0, :], out[-1, :], out[:, 0], out[:, -1] = exact[0, :], exact[-1, :], exact[:, 0], exact[:, -1]
    return out


def start_levels(nx, dx, dt):
    """phi(x, 0) exact; phi(x, dt) = phi + dt phi_t + (dt / (2 dx))^2 times the sum over the two
    axes of the second differences of phi(., 0) (the paper's start-up), boundary exact."""
    Y, X = _grid(nx)
    p0 = np.exp(X + Y)
    second = np.zeros_like(p0)
    second[1:-1, :] += p0[2:, :] - 2 * p0[1:-1, :] + p0[:-2, :]
    second[:, 1:-1] += p0[:, 2:] - 2 * p0[:, 1:-1] + p0[:, :-2]
    p1 = p0 + dt * p0 + (dt / (2 * dx)) ** 2 * second    # phi_t = phi for exp(x + y + t)
    return p0, _with_boundary(p1, np.exp(X + Y + dt))


def interior_gre(case, nx, step):
    """Run one Table 4 row; step(cur, prev) returns the next level (numpy, (y, x) order)."""
    _, dx, dt, nt = problem(case, nx)
    Y, X = _grid(nx)
    prev, cur = start_levels(nx, dx, dt)
    for m in range(1, nt):
        prev, cur = cur, _with_boundary(step(cur, prev), np.exp(X + Y + (m + 1) * dt))
    ex = np.exp(X + Y + nt * dt)
    return float(np.abs(cur - ex)[1:-1, 1:-1].sum() / np.abs(ex)[1:-1, 1:-1].sum())


def orders(gres):
    return [math.log2(gres[i] / gres[i + 1]) for i in range(len(gres) - 1)]
