"""Pins of the two-level theta-scheme Eq. (GCN) in the oracle (CPU only).

The oracle solves (I - theta_1 L) phi^{n+1} = (I + theta L) phi^n exactly in the DFT basis of the
circulant difference operator L (oracle.theta_run).  What fixes it from outside:

- a dense linear solve of the same system, with L assembled column by column from the explicit
  oracle step (catches a wrong FFT convention, axis order or a transposed operand);
- theta = 1 is the explicit scheme Eq. (2-2-2);
- a single Fourier mode is multiplied per step by Eq. (Tcond1-1)'s lambda, built from
  Eq. (Tcond1-2)'s A and B (ubar^+- of the EDF, not the step code);
- D2Q5 with u = 0 is the textbook theta-method on the five-point Laplacian (theta = 1/2:
  Crank-Nicolson), written out here in closed form, and it converges at second order to the
  exact heat-equation solution with dt proportional to dx;
- mass is conserved, and Theorem 2 holds: theta <= 1/2 does not amplify at a time step where
  the explicit end (theta = 1) blows up.
"""
import numpy as np
import pytest

from oracle import fourier as F
from oracle import oracle as orc
from oracle import params as P

RNG = np.random.default_rng(20250517)


def aniso_problem(lattice, n, dt=1.0, a0=0.0):
    dim = len(n)
    if dim == 2:
        K = [[0.02, 0.005], [0.005, 0.01]] if lattice == "D2Q9" else [[0.02, 0.0], [0.0, 0.01]]
        u = [0.1, 0.05]
    else:
        K = np.diag([0.02, 0.015, 0.01]) if lattice == "D3Q7" else [[0.02, 0.004, 0.0], [0.004, 0.015, 0.003],
                                                                     [0.0, 0.003, 0.01]]
        u = [0.05, 0.03, 0.02]
    return P.problem_lcde(lattice, 2, list(n), dt, [1.0] * dim, K, u, P.two_level_from_a0(a0))


def rand_field(prob):
    return 1.0 + 0.5 * RNG.standard_normal(prob.shape)


def dense_L(prob):
    """The matrix of L = E - I, one column per unit vector (E: the explicit oracle step)."""
    N = int(np.prod(prob.shape))
    M = np.empty((N, N))
    for c in range(N):
        e = np.zeros(N)
        e[c] = 1.0
        M[:, c] = orc.step(prob, [e.reshape(prob.shape)])[0].ravel() - e
    return M


CASES = [("D2Q9", (5, 6)), ("D2Q5", (4, 5)), ("D3Q7", (3, 4, 5)), ("D3Q19", (3, 3, 4))]


@pytest.mark.parametrize("lattice,shape", CASES)
def test_theta_matches_dense_solve(lattice, shape):
    prob = aniso_problem(lattice, shape[::-1])
    L = dense_L(prob)
    I = np.eye(L.shape[0])
    phi = rand_field(prob)
    for theta in (0.0, 0.3, 0.5):
        want = phi.ravel()
        for _ in range(3):
            want = np.linalg.solve(I - (1 - theta) * L, (I + theta * L) @ want)
        got = orc.theta_run(prob, [phi], 3, theta)[0]
        assert np.abs(got.ravel() - want).max() <= 1e-12 * np.abs(want).max(), (lattice, theta)


@pytest.mark.parametrize("lattice,n", [("D2Q9", (24, 20)), ("D3Q7", (12, 10, 8))])
def test_theta_one_is_the_explicit_scheme(lattice, n):
    prob = aniso_problem(lattice, n)
    phi = rand_field(prob)
    want, _ = orc.run(prob, [phi], None, 5)
    got = orc.theta_run(prob, [phi], 5, 1.0)
    assert np.abs(got[0] - want[0]).max() <= 1e-13 * np.abs(want[0]).max()


@pytest.mark.parametrize("lattice", ["D2Q9", "D2Q5"])
def test_theta_mode_amplification_is_eq_tcond1_1(lattice):
    n = (32, 24)
    prob = aniso_problem(lattice, n)
    ny, nx = prob.shape
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    for (mx, my) in ((1, 0), (3, 2), (7, 5), (16, 12)):
        th = 2 * np.pi * mx * x / nx + 2 * np.pi * my * y / ny
        for theta in (0.0, 0.5, 0.8):
            lam = F.theta_lambda(prob, theta, prob.shape)[my, mx]
            got = orc.theta_run(prob, [np.cos(th)], 4, theta)[0]
            want = np.real(lam ** 4 * np.exp(1j * th))
            assert np.abs(got - want).max() <= 1e-12, (lattice, mx, my, theta)


def heat_problem(n, dt, kx, ky):
    dx = 2 * np.pi / n
    return P.problem_lcde("D2Q5", 2, [n, n], dt, [dx, dx], [[kx, 0], [0, ky]], [0.0, 0.0],
                          P.two_level_from_a0(0.0)), dx


def test_theta_on_d2q5_is_the_textbook_theta_method():
    # u = 0 on D2Q5: E = I + dt (kx d_xx + ky d_yy) with the three-point second differences, so the
    # theta-scheme multiplies a mode by (1 + theta dt s) / (1 - (1 - theta) dt s),
    # s = -(4 kx / dx^2) sin^2(xi_x / 2) - (4 ky / dy^2) sin^2(xi_y / 2)
    n, kx, ky = 32, 0.3, 0.2
    dt = 0.4
    prob, dx = heat_problem(n, dt, kx, ky)
    phi = rand_field(prob)
    xi = F.thetas(prob.shape)              # (xi_y, xi_x), index units
    s = -4 * kx / dx ** 2 * np.sin(xi[1] / 2) ** 2 - 4 * ky / dx ** 2 * np.sin(xi[0] / 2) ** 2
    for theta in (0.0, 0.5, 1.0):
        mult = (1 + theta * dt * s) / (1 - (1 - theta) * dt * s)
        want = np.real(np.fft.ifft2(np.fft.fft2(phi) * mult ** 3))
        got = orc.theta_run(prob, [phi], 3, theta)[0]
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max(), theta


def test_crank_nicolson_converges_at_second_order():
    # theta = 1/2 on D2Q5, u = 0: phi = sin(x) sin(2y) decays as exp(-(kx + 4 ky) t); with dt
    # proportional to dx (far beyond the explicit limit dt <= dx^2 / (2 (kx + ky))) the error
    # falls as dx^2
    kx, ky, T = 0.3, 0.2, 1.0
    errs = []
    for n in (16, 32, 64):
        dx = 2 * np.pi / n
        steps = n // 4
        dt = T / steps
        prob, _ = heat_problem(n, dt, kx, ky)
        g = np.arange(n) * dx
        Y, X = np.meshgrid(g, g, indexing="ij")
        phi0 = np.sin(X) * np.sin(2 * Y)
        got = orc.theta_run(prob, [phi0], steps, 0.5)[0]
        errs.append(np.abs(got - phi0 * np.exp(-(kx + 4 * ky) * T)).max())
        assert dt > dx * dx / (2 * (kx + ky))
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.9 <= o <= 2.2 for o in orders), (errs, orders)


def test_crank_nicolson_d2q9_converges_at_second_order():
    # the same heat problem on D2Q9 (quadratic EDF, d_0 = 1/3): not the five-point scheme, but
    # still second order with dt proportional to dx
    kx, ky, T = 0.3, 0.2, 1.0
    errs = []
    for n in (32, 64, 128):
        dx = 2 * np.pi / n
        steps = n // 4
        prob = P.problem_lcde("D2Q9", 2, [n, n], T / steps, [dx, dx], [[kx, 0], [0, ky]], [0.0, 0.0],
                              P.two_level_from_a0(0.0))
        g = np.arange(n) * dx
        Y, X = np.meshgrid(g, g, indexing="ij")
        phi0 = np.sin(X) * np.sin(2 * Y)
        got = orc.theta_run(prob, [phi0], steps, 0.5)[0]
        errs.append(np.abs(got - phi0 * np.exp(-(kx + 4 * ky) * T)).max())
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.9 <= o <= 2.1 for o in orders), (errs, orders)


def test_theta_conserves_mass():
    prob = aniso_problem("D2Q9", (40, 30))
    phi = rand_field(prob)
    for theta in (0.0, 0.5):
        out = orc.theta_run(prob, [phi], 10, theta)[0]
        assert abs(out.sum() - phi.sum()) <= 1e-12 * np.abs(phi).sum()


def test_theorem2_at_a_large_time_step():
    # heavily diffusive D2Q5 (a_0 = -2, so A_22 = 3/2): the explicit end blows up, theta <= 1/2
    # never amplifies (Theorem 2 (1))
    prob = P.problem_lcde("D2Q5", 2, [16, 16], 1.0, [1, 1], [[0.3, 0], [0, 0.25]], [0.2, 0.1],
                          P.two_level_from_a0(-2.0))
    phi = rand_field(prob)
    n0 = np.linalg.norm(phi)
    for theta in (0.0, 0.25, 0.5):
        out = orc.theta_run(prob, [phi], 50, theta)[0]
        assert np.linalg.norm(out) <= n0 * (1 + 1e-12), theta
    assert np.linalg.norm(orc.theta_run(prob, [phi], 50, 1.0)[0]) > 1e3 * n0


def theta_star(prob):
    """The stability bound of Eq. (Tcond1-3) for A <= 0: |lambda| <= 1 on every mode iff
    theta <= theta* = 1/2 + min over modes with A^2 + B^2 > 0 of (-A) / (A^2 + B^2)."""
    A, B = F.theta_AB(prob, prob.shape)
    q = A * A + B * B
    m = q > 1e-14
    assert (A[m] <= 1e-14).all()      # condition (a)
    return 0.5 + float((-A[m] / q[m]).min())


def heavy_problem():
    return P.problem_lcde("D2Q5", 2, [16, 16], 1.0, [1, 1], [[0.3, 0], [0, 0.25]], [0.2, 0.1],
                          P.two_level_from_a0(-2.0))


def test_theta_bound_just_inside_and_outside():
    # conditional stability for theta > 1/2 (Theorem 2 (2)): bounded just inside theta*, and just
    # outside the oracle's growth rate per step tends to max |lambda| of Eq. (Tcond1-1)
    prob = heavy_problem()
    ts = theta_star(prob)
    assert 0.5 < ts < 1.0, ts
    phi = rand_field(prob)
    n0 = np.linalg.norm(phi)
    inside = orc.theta_run(prob, [phi], 400, ts - 0.01)[0]
    assert np.linalg.norm(inside) <= n0 * (1 + 1e-10)
    th = ts + 0.01
    lam = np.abs(F.theta_lambda(prob, th, prob.shape)).max()
    assert lam > 1.0
    a = orc.theta_run(prob, [phi], 300, th)[0]
    b = orc.theta_run(prob, [a], 1, th)[0]
    assert abs(np.linalg.norm(b) / np.linalg.norm(a) - lam) <= 1e-6 * lam
