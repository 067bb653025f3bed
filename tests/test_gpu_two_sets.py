"""GPU parity of the multiple-parameter-set scheme, Eq. (2-2-1b) (MMFD_FLAG_TWO_SETS): the CUDA
path against the oracle's central form with the same sets, on the direct, marching, blocked and
batched (server) kernels.  Tolerances as for the one-set scheme: FP64 1e-12, FP32 1e-5
relative to the field's max |value|.  The TRT MesoFD scheme of Eq. (2-1b) is the special case
whose zeroth-order set is the even set (momentum: the odd set); it is checked against the
oracle's form 4, which builds f_j per direction.
"""
import numpy as np
import pytest

import gpu_cases as G
from oracle import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_17057_gb300 import mmfd
    return mmfd


def two_set_case(lat, pde, levels, n, storage, rng, trt=False):
    kw, prob = G.case(lat, pde, levels, n, storage)
    a = tuple(prob.a)
    ah = tuple(prob.ahat)
    ab = tuple(prob.abar) if prob.pde == "NSE" else a
    abh = tuple(prob.abarhat) if prob.pde == "NSE" else ah
    def pert(t):
        # zero-sum perturbations keep sum_k a_k (A_00 = 1 when the set is the zeroth-order one)
        d = 0.04 * rng.standard_normal(3)
        return tuple(x + y for x, y in zip(t, d - d.mean()))
    sets = {"d2": (pert(a), pert(ah) if levels == 3 else (0.0, 0.0, 0.0)),
            "d1": (pert(a), pert(ah) if levels == 3 else (0.0, 0.0, 0.0)),
            "bar_d2": (pert(ab), pert(abh) if levels == 3 else (0.0, 0.0, 0.0)),
            "bar_d1": (pert(ab), pert(abh) if levels == 3 else (0.0, 0.0, 0.0))}
    if trt:
        # Eq. (2-1b): the zeroth-order set is the even set, the momentum's the odd set; the
        # problem is rebuilt from them, since EDF parameters (the NCDE second moment, the LCDE
        # diffusion mapping) follow the moments of the zeroth-order set
        coeffs = {"a": sets["d2"][0], "ahat": sets["d2"][1]}
        if pde == "NSE":
            coeffs.update(abar=sets["bar_d2"][0], abarhat=sets["bar_d2"][1])
        kw, prob = G.case(lat, pde, levels, n, storage, coeffs=coeffs)
    kw["sets"] = sets
    prob.sets = sets
    return kw, prob


def run(mm, kw, L0, L1, steps, **extra):
    s = mm.Solver(mm.make_desc(**kw, flags=mm.MMFD_FLAG_ALLOW_UNSTABLE, **extra))
    try:
        s.set_fields(L0)
        if L1 is not None:
            s.set_fields(L1, level=1)
        stored0 = s.fields(0)
        stored1 = s.fields(1) if kw["levels"] == 3 else None
        s.step(steps)
        out = s.fields(0)
        kern = s.get_info().kernel.decode()
    finally:
        s.close()
    return stored0, stored1, out, kern


SIZES_2D = [[300, 70], [67, 45]]
SIZES_3D = [[150, 21, 9], [70, 37, 21]]


@pytest.mark.parametrize("lat,pde,levels", G.SUPPORTED)
def test_two_sets_fp64(mm, lat, pde, levels):
    rng = np.random.default_rng(G.RNG_SEED + 80)
    kernels = set()
    for n in (SIZES_2D if G.dims(lat) == 2 else SIZES_3D):
        kw, prob = two_set_case(lat, pde, levels, n, "fp64", rng)
        L0 = G.random_level(prob, rng)
        L1 = G.random_level(prob, rng) if levels == 3 else None
        _, _, out, kern = run(mm, kw, L0, L1, 3)
        kernels.add(kern)
        ref, _ = orc.run(prob, L0, L1, nsteps=3, form="central")
        assert G.rel_err(out, ref) < 1e-12, (n, kern, G.rel_err(out, ref))
    assert len(kernels) == 2, kernels   # the direct and the marching kernel both ran


@pytest.mark.parametrize("lat,pde,levels", [("D2Q9", "NSE", 2), ("D2Q9", "LCDE", 2), ("D2Q9", "NCDE", 3),
                                            ("D3Q19", "NSE", 2), ("D3Q7", "LCDE", 2)])
def test_two_sets_fp32(mm, lat, pde, levels):
    rng = np.random.default_rng(G.RNG_SEED + 81)
    n = [300, 70] if G.dims(lat) == 2 else [150, 21, 9]
    kw, prob = two_set_case(lat, pde, levels, n, "fp32", rng)
    L0 = G.random_level(prob, rng)
    L1 = G.random_level(prob, rng) if levels == 3 else None
    s0, s1, out, _ = run(mm, kw, L0, L1, 3)
    ref, _ = orc.run(prob, s0, s1, nsteps=3, form="central")
    assert G.rel_err(out, ref) < 1e-5


def test_two_sets_blocked(mm):
    rng = np.random.default_rng(G.RNG_SEED + 82)
    kw, prob = two_set_case("D2Q9", "LCDE", 2, [300, 70], "fp32", rng)
    L0 = G.random_level(prob, rng)
    s0, _, out, kern = run(mm, kw, L0, None, 9, temporal_depth=4)
    assert kern == "k_march2d_tb"
    ref, _ = orc.run(prob, s0, None, nsteps=9, form="central")
    assert G.rel_err(out, ref) < 1e-5


@pytest.mark.parametrize("lat,pde,levels", [("D2Q9", "NSE", 2), ("D2Q9", "NSE", 3), ("D2Q9", "NCDE", 3),
                                            ("D3Q19", "NSE", 2)])
def test_trt_mesofd_special_case(mm, lat, pde, levels):
    rng = np.random.default_rng(G.RNG_SEED + 83)
    n = [67, 45] if G.dims(lat) == 2 else [40, 21, 9]
    kw, prob = two_set_case(lat, pde, levels, n, "fp64", rng, trt=True)
    L0 = G.random_level(prob, rng)
    L1 = G.random_level(prob, rng) if levels == 3 else None
    _, _, out, _ = run(mm, kw, L0, L1, 3)
    ref, _ = orc.run(prob, L0, L1, nsteps=3, form="mesofd_trt")
    assert G.rel_err(out, ref) < 1e-12


def test_two_sets_in_the_server(mm):
    rng = np.random.default_rng(G.RNG_SEED + 84)
    reqs = []
    for lat, pde, levels, n in [("D2Q9", "NSE", 2, [96, 70]), ("D2Q9", "LCDE", 2, [400, 200]),
                                ("D3Q19", "NCDE", 3, [24, 20, 18])]:
        kw, prob = two_set_case(lat, pde, levels, n, "fp64", rng)
        reqs.append((kw, prob, G.random_level(prob, rng), 7))
    srv = mm.Server(1 << 30, max_slots=8, steps_per_tick=4)
    tickets = [srv.submit(mm.make_desc(**kw, flags=mm.MMFD_FLAG_ALLOW_UNSTABLE), L0, steps)
               for kw, _, L0, steps in reqs]
    srv.drain()
    for t, (kw, prob, L0, steps) in zip(tickets, reqs):
        rc, r = srv.poll(t)
        assert rc == mm.MMFD_OK and r.status == 0
        out = srv.result(t)
        srv.release(t)
        ref, _ = orc.run(prob, L0, L0 if prob.levels == 3 else None, nsteps=steps, form="central")
        assert G.rel_err(out, ref) < 1e-12
    srv.close()
