"""mmfd_check_fields on the GPU: the frozen-coefficient check about the extreme states of a
solver's current level (field maxima from the device reductions) agrees with mmfd_linear_stability
at those states and flags a level whose flow is too fast for the scheme."""
import numpy as np
import pytest

from paper_2505_17057_gb300 import mmfd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return mmfd


@pytest.mark.parametrize("storage", ["fp64", "fp32", "bf16"])
def test_check_fields_nse(mm, storage):
    rng = np.random.default_rng(3)
    n = [140, 20]
    kw = dict(pde="NSE", lattice="D2Q9", levels=2, n=n, dt=1.0, dx=[1.0, 1.0], a=(1.0, 0.0, 0.0),
              abar=(1.0, 0.0, 0.0), storage=storage)
    s = mm.Solver(mm.make_desc(**kw))
    try:
        for umax, stable in [(0.05, True), (0.45, False)]:
            u = rng.uniform(-umax, umax, (n[1], n[0]))
            v = rng.uniform(-umax, umax, (n[1], n[0]))
            u.flat[0], v.flat[1] = umax, -umax        # the maxima the reduction must find
            s.set_fields([np.ones((n[1], n[0])), u, v])
            rc, amp = mm.mmfd_check_fields(s.h)
            stored = s.fields(0)
            mu, mv = np.abs(stored[1]).max(), np.abs(stored[2]).max()
            want = max(mm.mmfd_linear_stability(mm.make_desc(**kw), [1.0, su * mu, sv * mv])[1]
                       for su in (-1, 1) for sv in (-1, 1))
            assert abs(amp - max(want, 1.0)) <= 1e-9 * amp, (umax, amp, want)
            assert (rc == mm.MMFD_OK) == stable, (umax, rc, amp)
    finally:
        s.close()


def test_check_fields_ncde(mm):
    n = [130, 16]
    kw = dict(pde="NCDE", lattice="D2Q9", levels=3, n=n, dt=0.8, dx=[1.0, 1.1], flux=[[0, 0.05, 0.1, 0], [0, -0.03, 0.1, 0]],
              diff=[0.15, 0, 0.05, 0], a=(7 / 8, 0.0, 1 / 8), ahat=(1 / 8, 0.0, -1 / 8), storage="fp32")
    s = mm.Solver(mm.make_desc(**kw))
    try:
        phi = 0.5 + 0.2 * np.cos(2 * np.pi * np.arange(n[0]) / n[0])[None, :] * np.ones((n[1], 1))
        s.set_fields([phi])
        rc, amp = mm.mmfd_check_fields(s.h)
        assert rc == mm.MMFD_OK and abs(amp - 1.0) < 1e-9, (rc, amp)
        # a much larger amplitude drives D(phi) = 0.15 + 0.05 phi^2 past the explicit limit
        s.set_fields([5.0 * phi])
        rc, amp = mm.mmfd_check_fields(s.h)
        assert rc == mm.MMFD_ERR_UNSTABLE and amp > 1.0, (rc, amp)
    finally:
        s.close()
