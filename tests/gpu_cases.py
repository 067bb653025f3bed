"""Shared problem definitions for the GPU parity tests: one physical description, turned
into an mmfd_desc for the CUDA path and, independently, into an oracle Problem."""
import numpy as np

from oracle import oracle as orc
from oracle import params as P

RNG_SEED = 20250517

# Example 1 Case 3 / Example 2 Case 2 set (Eq. (X) with a_0 = 0, A_10 = A_11 = -1, A_21 = 1/4, A_22 = 1/2)
THREE_A = (7 / 8, 0.0, 1 / 8)
THREE_AHAT = (1 / 8, 0.0, -1 / 8)


def dims(lat):
    return 2 if lat.startswith("D2") else 3


def shape_of(n, lat):
    return (n[1], n[0]) if dims(lat) == 2 else (n[2], n[1], n[0])


def case(lat, pde, levels, n, storage="fp64", generic=True, coeffs=None):
    """(desc kwargs, oracle Problem) for a generic stable problem on the given grid.

    coeffs: optional dict overriding "a", "ahat" (and, for the NSE, "abar", "abarhat"); the
    oracle problem is then built from them (its EDF parameters follow the scheme's moments)."""
    dim = dims(lat)
    n = list(n) + [1] * (3 - len(n))
    dt = 0.8
    dx = [1.0, 1.1, 0.9][:dim]
    a2 = (0.95, 0.1, -0.05)      # a_0 = 0.1 two-level: a_{-1} = 1 - a_0/2, a_1 = -a_0/2
    a3, ah3 = THREE_A, THREE_AHAT
    a = a2 if levels == 2 else a3
    ah = (0.0, 0.0, 0.0) if levels == 2 else ah3
    coeffs = coeffs or {}
    a = tuple(coeffs.get("a", a))
    ah = tuple(coeffs.get("ahat", ah))
    kw = dict(pde=pde, lattice=lat, levels=levels, n=n[:dim] if dim == 3 else n[:2], dt=dt, dx=dx, storage=storage)
    if dim == 3:
        kw["n"] = n
    if pde == "LCDE":
        if lat in ("D2Q5", "D3Q7"):
            K = np.diag([0.05, 0.04, 0.06][:dim])
        else:
            K = np.diag([0.05, 0.04, 0.06][:dim]) + 0.006 * (1 - np.eye(dim))
        u = [0.08, -0.05, 0.04][:dim]
        kw.update(K=K, u=u, a=a, ahat=ah)
        prob = P.problem_lcde(lat, levels, n, dt, dx, K, u, a, ah)
    elif pde == "NCDE":
        # diffusion-dominated (|B'|^2 <= 2 alpha / dt) so that every NCDE case stays stable
        flux = [[0, 0.05, 0.1, 0], [0, -0.03, 0.1, 0], [0, 0, 0.06, 0.02]][:dim]
        diff = [0.15, 0, 0.05, 0]
        kw.update(flux=flux, diff=diff, a=a, ahat=ah)
        prob = P.problem_ncde(lat, levels, n, dt, dx, flux, diff[:3], a, ah)
    else:
        ab = (0.9, 0.2, -0.1) if levels == 2 else (0.8, 0.0, 0.2)
        abh = (0.0, 0.0, 0.0) if levels == 2 else (0.1, 0.0, -0.1)
        ab = tuple(coeffs.get("abar", ab))
        abh = tuple(coeffs.get("abarhat", abh))
        kw.update(a=a, ahat=ah, abar=ab, abarhat=abh)
        prob = P.problem_nse(lat, levels, n, dt, dx, a, ab, ah, abh)
    return kw, prob


def random_level(prob, rng, nse_u=0.03):
    shape = prob.shape
    if prob.pde == "NSE":
        return [1.0 + 0.01 * rng.standard_normal(shape)] + [nse_u * rng.standard_normal(shape) for _ in range(prob.dim)]
    if prob.pde == "NCDE":
        return [0.5 + 0.2 * rng.standard_normal(shape)]
    return [1.0 + 0.3 * rng.standard_normal(shape)]


SUPPORTED = [
    ("D2Q5", "LCDE", 2), ("D2Q5", "LCDE", 3), ("D2Q9", "LCDE", 2), ("D2Q9", "LCDE", 3),
    ("D2Q9", "NCDE", 2), ("D2Q9", "NCDE", 3), ("D2Q9", "NSE", 2), ("D2Q9", "NSE", 3),
    ("D3Q7", "LCDE", 2), ("D3Q7", "LCDE", 3), ("D3Q19", "LCDE", 2), ("D3Q19", "LCDE", 3),
    ("D3Q19", "NCDE", 2), ("D3Q19", "NCDE", 3), ("D3Q19", "NSE", 2), ("D3Q19", "NSE", 3),
]


def rel_err(gpu, ref):
    return max(float(np.abs(g - r).max() / max(1e-300, np.abs(r).max())) for g, r in zip(gpu, ref))


def bf16_round(x, ref=0.0):
    """Round ref + bf16(x - ref) (nearest even), as the BF16-offset storage does."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x - ref, dtype=np.float32)).to(torch.bfloat16)
    return t.to(torch.float64).numpy() + ref


def bf16_ulp(x):
    ax = np.maximum(np.abs(x), 1e-38)
    return 2.0 ** (np.floor(np.log2(ax)) - 7)
