"""GPU checks of the level upload (the pack kernels): an FP32 source packs into FP32 and BF16-offset
storage exactly as the same values given in FP64, whether or not the storage reference is an FP32
number (the packing forms the offset in FP32 only where that rounds to the FP64 result)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_17057_gb300 import mmfd
    return mmfd


def stored_after_upload(mm, storage, ref, values, device_f32):
    import torch
    n = [values.shape[1], values.shape[0]]
    d = mm.make_desc("LCDE", "D2Q9", 2, n, 1.0, [1.0, 1.0], storage=storage, K=[[0.02, 0.0], [0.0, 0.02]],
                     u=[0.05, 0.0], targets=[0, -1, -1, 0, 0.5], ref=[ref])
    s = mm.Solver(d)
    try:
        if device_f32:
            s.set_fields([torch.tensor(values, dtype=torch.float32, device="cuda")])
        else:
            s.set_fields([values.astype(np.float64)])
        return s.fields(0)[0]
    finally:
        s.close()


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
@pytest.mark.parametrize("ref", [1.0, 0.1, 0.0])
def test_fp32_upload_equals_fp64_upload(mm, storage, ref):
    rng = np.random.default_rng(31)
    # nx a multiple of 4 (the vector pack), values spanning many binades around the reference,
    # some equal to it, some far from it, some tiny
    v = (ref + np.concatenate([rng.standard_normal(600) * 10.0 ** rng.uniform(-9, 2, 600),
                               np.full(8, ref), rng.standard_normal(8) * 1e-30])).astype(np.float32)
    vals = np.resize(v, (37, 256))
    a = stored_after_upload(mm, storage, ref, vals, device_f32=True)
    b = stored_after_upload(mm, storage, ref, vals, device_f32=False)
    assert np.array_equal(a, b), np.abs(a - b).max()
