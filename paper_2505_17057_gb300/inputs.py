"""Seeded synthetic inputs for the MMFD solvers.

This module is shared by the CUDA path, the oracle-based tests and the
benchmark.  It only produces initial fields and closed-form reference
fields (Gaussian hill, random Fourier series, Taylor-Green vortex); it holds
none of the MMFD arithmetic (no equilibrium distribution, no stencil, no
scheme coefficients).

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), drawn on the host once and
fed to both the GPU and the oracle.

Array layout: every field is a numpy float64 array indexed [z][y][x] (3D) or
[y][x] (2D), x fastest, i.e. shape (ny, nx) or (nz, ny, nx).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MASK64 = (1 << 64) - 1
SEED_BASE = 0x4D4D4644  # "MMFD"


class SplitMix64:
    """SplitMix64 generator (64-bit state, golden-gamma increment)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        """Uniform double in [lo, hi) from the top 53 bits."""
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / 9007199254740992.0))

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive), by rejection-free modulo of 64 bits."""
        return lo + self.next_u64() % (hi - lo + 1)


def rng_for(config_index: int, salt: int = 0) -> SplitMix64:
    return SplitMix64(SEED_BASE + config_index + (salt << 32))


# --------------------------------------------------------------------------
# 2D fields
# --------------------------------------------------------------------------

def gaussian_hill_2d(nx: int, ny: int, cx: float, cy: float, sigma: float,
                     amp: float = 1.0) -> np.ndarray:
    """phi0 = amp * exp(-((x-cx)^2 + (y-cy)^2) / (2 sigma^2)), x, y in cell units."""
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    X, Y = np.meshgrid(x, y, indexing="xy")
    return amp * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2.0 * sigma * sigma))


@dataclass
class FourierModes2D:
    amps: np.ndarray    # (M,)
    kvec: np.ndarray    # (M, 2) integer wave vectors
    phases: np.ndarray  # (M,)


def draw_fourier_modes_2d(rng: SplitMix64, nmodes: int = 32, kmax: int = 8,
                          amp_lo: float = 0.1, amp_hi: float = 0.5) -> FourierModes2D:
    amps, ks, ph = [], [], []
    for _ in range(nmodes):
        amps.append(rng.uniform(amp_lo, amp_hi))
        while True:
            kx = rng.randint(-kmax, kmax)
            ky = rng.randint(-kmax, kmax)
            if kx != 0 or ky != 0:
                break
        ks.append((kx, ky))
        ph.append(rng.uniform(0.0, 2.0 * math.pi))
    return FourierModes2D(np.array(amps), np.array(ks, dtype=np.int64), np.array(ph))


def fourier_field_2d(modes: FourierModes2D, nx: int, ny: int) -> np.ndarray:
    """phi0(x, y) = sum_m A_m cos(k_m . (x, y) + theta_m) on the periodic box [0, 2 pi)^2."""
    x = 2.0 * math.pi * np.arange(nx, dtype=np.float64) / nx
    y = 2.0 * math.pi * np.arange(ny, dtype=np.float64) / ny
    # cos(kx x + ky y + t) = cos(ky y) cos(kx x + t) - sin(ky y) sin(kx x + t): the sum over modes
    # is one (ny x 2M) @ (2M x nx) product instead of M full-grid cosines
    cols, rows = [], []
    for a, (kx, ky), t in zip(modes.amps, modes.kvec, modes.phases):
        cols += [np.cos(ky * y), -np.sin(ky * y)]
        rows += [a * np.cos(kx * x + t), a * np.sin(kx * x + t)]
    return np.stack(cols, axis=1) @ np.stack(rows, axis=0)


def taylor_green_2d(nx: int, ny: int, u0: float, nu: float, t: float,
                    rho0: float = 1.0, cs2: float = 1.0 / 3.0):
    """Closed-form decaying Taylor-Green vortex on an nx x ny periodic lattice.

    u = -u0 cos(kx x) sin(ky y) e^{-nu (kx^2+ky^2) t},
    v =  u0 (kx/ky) sin(kx x) cos(ky y) e^{-nu (kx^2+ky^2) t},
    p = -(rho0 u0^2 / 4) (cos 2kx x + (kx/ky)^2 cos 2ky y) e^{-2 nu (kx^2+ky^2) t},
    rho = rho0 + p / cs2, with kx = 2 pi / nx, ky = 2 pi / ny (lattice units).
    Returns (rho, u, v) as float64 arrays of shape (ny, nx).
    """
    kx = 2.0 * math.pi / nx
    ky = 2.0 * math.pi / ny
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    X, Y = np.meshgrid(x, y, indexing="xy")
    decay = math.exp(-nu * (kx * kx + ky * ky) * t)
    u = -u0 * np.cos(kx * X) * np.sin(ky * Y) * decay
    v = u0 * (kx / ky) * np.sin(kx * X) * np.cos(ky * Y) * decay
    p = -(rho0 * u0 * u0 / 4.0) * (np.cos(2 * kx * X) + (kx / ky) ** 2 * np.cos(2 * ky * Y)) * decay * decay
    rho = rho0 + p / cs2
    return rho, u, v


# --------------------------------------------------------------------------
# 3D fields
# --------------------------------------------------------------------------

@dataclass
class CosSeries1D:
    amps: np.ndarray    # (M,)
    phases: np.ndarray  # (M,)
    norm: float         # 1 / max |S| on the grid it was normalised on


def draw_cos_series(rng: SplitMix64, nmodes: int = 16, amp_lo: float = 0.1,
                    amp_hi: float = 0.5) -> CosSeries1D:
    amps = np.array([rng.uniform(amp_lo, amp_hi) for _ in range(nmodes)])
    ph = np.array([rng.uniform(0.0, 2.0 * math.pi) for _ in range(nmodes)])
    return CosSeries1D(amps, ph, 1.0)


def cos_series_eval(s: CosSeries1D, n: int, deriv: int = 0) -> np.ndarray:
    """S(x) = norm * sum_{m=1}^{M} A_m cos(m x + theta_m) on x = 2 pi i / n (or its derivative in x)."""
    x = 2.0 * math.pi * np.arange(n, dtype=np.float64) / n
    out = np.zeros(n)
    for m, (a, t) in enumerate(zip(s.amps, s.phases), start=1):
        arg = m * x + t
        if deriv == 0:
            out += a * np.cos(arg)
        elif deriv == 1:
            out += -a * m * np.sin(arg)
        else:
            raise ValueError("deriv must be 0 or 1")
    return s.norm * out


def normalised_series(rng: SplitMix64, n: int, nmodes: int = 16) -> CosSeries1D:
    s = draw_cos_series(rng, nmodes)
    s.norm = 1.0 / float(np.max(np.abs(cos_series_eval(s, n))))
    return s


def separable_scalar_3d(config_index: int, nx: int, ny: int, nz: int, nmodes: int = 16):
    """phi0 = 1 + 0.5 * Sx(x) Sy(y) Sz(z), each S a seeded cosine series with max |S| = 1.

    Returns (phi0, (Sx, Sy, Sz)) where the series objects allow an exact
    separable reference solution to be built by the caller.
    """
    rng = rng_for(config_index)
    sx = normalised_series(rng, nx, nmodes)
    sy = normalised_series(rng, ny, nmodes)
    sz = normalised_series(rng, nz, nmodes)
    fx, fy, fz = cos_series_eval(sx, nx), cos_series_eval(sy, ny), cos_series_eval(sz, nz)
    phi = 1.0 + 0.5 * fz[:, None, None] * fy[None, :, None] * fx[None, None, :]
    return phi, (sx, sy, sz)


def solenoidal_velocity_3d(config_index: int, nx: int, ny: int, nz: int,
                           umax: float = 0.05, nmodes: int = 16):
    """Divergence-free velocity u = curl(psi) from separable cosine series, scaled to max |u| = umax.

    psi = (P(y) Q(z), R(x) T(z), U(x) V(y)), so
    u_x = U(x) V'(y) - R(x) T'(z), u_y = P(y) Q'(z) - U'(x) V(y), u_z = R'(x) T(z) - P'(y) Q(z).
    Returns (u, v, w) float64 arrays of shape (nz, ny, nx).
    """
    rng = rng_for(config_index, salt=1)
    P, Q, R, T, U, V = (normalised_series(rng, m, nmodes) for m in (ny, nz, nx, nz, nx, ny))
    Px, Qx, Rx, Tx, Ux, Vx = (cos_series_eval(s, m) for s, m in
                              ((P, ny), (Q, nz), (R, nx), (T, nz), (U, nx), (V, ny)))
    dP, dQ, dR, dT, dU, dV = (cos_series_eval(s, m, 1) for s, m in
                              ((P, ny), (Q, nz), (R, nx), (T, nz), (U, nx), (V, ny)))
    ux = Ux[None, None, :] * dV[None, :, None] - Rx[None, None, :] * dT[:, None, None]
    uy = Px[None, :, None] * dQ[:, None, None] - dU[None, None, :] * Vx[None, :, None]
    uz = dR[None, None, :] * Tx[:, None, None] - dP[None, :, None] * Qx[:, None, None]
    ux = np.broadcast_to(ux, (nz, ny, nx)).copy()
    uy = np.broadcast_to(uy, (nz, ny, nx)).copy()
    uz = np.broadcast_to(uz, (nz, ny, nx)).copy()
    scale = umax / float(max(np.abs(ux).max(), np.abs(uy).max(), np.abs(uz).max()))
    return ux * scale, uy * scale, uz * scale


def random_field(config_index: int, shape, lo: float = -1.0, hi: float = 1.0, salt: int = 7) -> np.ndarray:
    """Uniform random field from SplitMix64 (vectorised: one draw per element, in C order)."""
    rng = rng_for(config_index, salt)
    n = int(np.prod(shape))
    # Vectorised SplitMix64: the k-th output uses state seed + (k+1) * gamma.
    k = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(rng.state) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return (lo + (hi - lo) * u).reshape(shape)
