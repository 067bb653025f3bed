"""The autotuner: it picks a (temporal depth, work-item height) pair by timing, leaves the
fields untouched, and the tuned solver still matches the oracle; a cache file replays the
choice without timing."""
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


@pytest.mark.parametrize("lat,pde,levels,n,depth", [
    ("D2Q9", "LCDE", 2, [300, 70], 0),     # depth and height tuned
    ("D2Q9", "NSE", 2, [260, 33], 1),      # height only
    ("D3Q19", "NSE", 2, [150, 21, 9], 1),  # 3D marching kernel
    ("D2Q9", "NCDE", 3, [67, 45], 1),      # direct kernel: nothing to vary but the timing runs
])
def test_autotune_keeps_fields_and_parity(mm, tmp_path, lat, pde, levels, n, depth):
    rng = np.random.default_rng(G.RNG_SEED + 70)
    kw, prob = G.case(lat, pde, levels, n, "fp64")
    L0 = G.random_level(prob, rng)
    L1 = G.random_level(prob, rng) if levels == 3 else None
    cache = str(tmp_path / "tune.txt")
    s = mm.Solver(mm.make_desc(**kw, temporal_depth=depth))
    try:
        s.set_fields(L0)
        if L1 is not None:
            s.set_fields(L1, level=1)
        before = s.fields(0)
        info = s.autotune(cache)
        assert info.from_cache == 0 and info.candidates >= 1 and info.ms_per_step > 0
        assert s.get_info().temporal_depth == info.temporal_depth
        after = s.fields(0)
        assert all(np.array_equal(a, b) for a, b in zip(before, after))
        assert s.get_info().steps_done == 0
        s.step(7)
        out = s.fields(0)
    finally:
        s.close()
    ref, _ = orc.run(prob, L0, L1, nsteps=7)
    assert G.rel_err(out, ref) < 1e-12
    # a second solver of the same problem takes the choice from the cache
    s2 = mm.Solver(mm.make_desc(**kw, temporal_depth=depth))
    try:
        info2 = s2.autotune(cache)
        assert info2.from_cache == 1 and info2.candidates == 0
        assert (info2.temporal_depth, info2.rows_per_item) == (info.temporal_depth, info.rows_per_item)
    finally:
        s2.close()
