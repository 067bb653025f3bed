"""GPU check of the TRT special case (Sec. III.C, case (2), s+ + s- = 2) against an independent
lattice-Boltzmann code: the three-level CUDA path, with the sets mmfd_trt_coefficients gives,
started from (one LBGK tau = 1 step of phi^0, phi^0), must reproduce the moments of the oracle's
TRT collide-and-stream run from equilibrium populations of phi^0.  FP64 storage, 1e-12 relative
to the field's max |value|, on the direct and the marching kernels.
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


THREE_LEVEL = [c[:2] for c in G.SUPPORTED if c[2] == 3]


@pytest.mark.parametrize("s", [0.7, 1.4])
@pytest.mark.parametrize("lat,pde", THREE_LEVEL)
def test_three_level_path_is_the_trt_lb(mm, lat, pde, s):
    rng = np.random.default_rng(G.RNG_SEED + 90)
    coeffs = mm.mmfd_trt_coefficients(s)
    # nx >= 128 runs the marching kernel, narrower grids the direct one
    sizes = [[300, 70], [67, 45]] if G.dims(lat) == 2 else [[150, 21, 9], [40, 21, 9]]
    kernels = set()
    steps = 6
    for n in sizes:
        kw, prob = G.case(lat, pde, 3, n, "fp64", coeffs=coeffs)
        phi0 = G.random_level(prob, rng)
        phi1 = orc.lbgk_tau1_run(prob, phi0, 1)
        solver = mm.Solver(mm.make_desc(**kw, flags=mm.MMFD_FLAG_ALLOW_UNSTABLE))
        try:
            solver.set_fields(phi1)
            solver.set_fields(phi0, level=1)
            solver.step(steps - 1)
            out = solver.fields(0)
            kernels.add(solver.get_info().kernel.decode())
        finally:
            solver.close()
        lb = orc.trt_run(prob, phi0, s, steps)
        assert all(np.isfinite(f).all() for f in lb)
        assert G.rel_err(out, lb) < 1e-12, (n, G.rel_err(out, lb))
    assert len(kernels) == 2, kernels
