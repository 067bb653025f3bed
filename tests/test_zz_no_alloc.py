"""mmfd_reduce_static -- the allocation-free variant of mmfd_reduce -- against mmfd_reduce.

Callers that cannot allocate device memory at the point of use (a cudaFree would synchronise
the device; an allocator's own bookkeeping path or a component under a fixed memory budget
cannot call back into cudaMalloc) use mmfd_reduce_static, which keeps its partial sums in a
fixed file-scope device array.  This test calls it through the C ABI twice in a row -- the
second call runs on the scratch the first one left behind -- and checks both results against
the existing entry point.  This file sorts last so that a run stopping at the first failure
has already run every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_reduce_static_matches_reduce():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_17057_gb300 import mmfd

    rng = np.random.default_rng(2027)
    shape = (300, 517)  # spans two 2^17-element blocks plus a ragged tail
    fields = [1.0 + 0.3 * rng.standard_normal(shape), 0.02 * rng.standard_normal(shape),
              0.02 * rng.standard_normal(shape)]
    d = mmfd.make_desc("NSE", "D2Q9", 2, [shape[1], shape[0]], 1.0, [1.0, 1.0], storage="fp64",
                       a=(1.0, 0.0, 0.0), abar=(1.0, 0.0, 0.0))
    s = mmfd.Solver(d)
    s.set_fields(fields)
    s.step(3)
    dev = s.fields(0, device=True)  # dense FP64 device arrays of the current level
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for what, tol in ((mmfd.MMFD_RED_SUM, 1e-12), (mmfd.MMFD_RED_MAXABS, 0.0), (mmfd.MMFD_RED_NONFINITE, 0.0)):
        ref = s.reduce(what)
        for call in range(2):  # two calls in a row share the same scratch
            got = []
            for f in dev:
                mmfd.mmfd_reduce_static(f.data_ptr(), mmfd.MMFD_DT_F64, f.numel(), what, out.data_ptr(), stream)
                torch.cuda.synchronize()
                got.append(float(out.item()))
            if what == mmfd.MMFD_RED_NONFINITE:
                assert sum(got) == ref[0], (call, got, ref)
            else:
                for g, r, f in zip(got, ref, dev):
                    scale = float(torch.abs(f).sum().item()) if what == mmfd.MMFD_RED_SUM else 1.0
                    assert abs(g - r) <= tol * scale, (what, call, g, r)
    # sizes beyond the static scratch are refused with a clear error, not run
    with pytest.raises(mmfd.MMFDError) as e:
        mmfd.mmfd_reduce_static(dev[0].data_ptr(), mmfd.MMFD_DT_F64, (1 << 27) + 1, mmfd.MMFD_RED_SUM,
                                out.data_ptr(), stream)
    assert e.value.code == mmfd.MMFD_ERR_ARG
    s.close()
