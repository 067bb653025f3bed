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


def test_reduce_static_fp32_and_nonfinite():
    # the FP32 load path and a non-zero non-finite count, against mmfd_reduce of an FP32 solver
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_17057_gb300 import mmfd

    rng = np.random.default_rng(2028)
    shape = (260, 1031)  # three 2^17-element blocks with a ragged tail
    phi = 1.0 + 0.3 * rng.standard_normal(shape)
    bad = phi.copy()
    where = rng.choice(bad.size, 37, replace=False)
    bad.reshape(-1)[where[:20]] = np.nan
    bad.reshape(-1)[where[20:30]] = np.inf
    bad.reshape(-1)[where[30:]] = -np.inf
    d = mmfd.make_desc("LCDE", "D2Q9", 2, [shape[1], shape[0]], 1.0, [1.0, 1.0], storage="fp32",
                       K=[[0.02, 0.0], [0.0, 0.02]], u=[0.05, 0.0], targets=[0, -1, -1, 0, 0.5], ref=[1.0])
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    s = mmfd.Solver(d)
    try:
        s.set_fields([phi])
        s.step(2)
        dev = s.fields(0, device=True, dtype=np.float32)[0]
        for what in (mmfd.MMFD_RED_SUM, mmfd.MMFD_RED_MAXABS, mmfd.MMFD_RED_NONFINITE):
            ref = s.reduce(what)[0]
            for call in range(2):
                mmfd.mmfd_reduce_static(dev.data_ptr(), mmfd.MMFD_DT_F32, dev.numel(), what, out.data_ptr(), stream)
                torch.cuda.synchronize()
                got = float(out.item())
                # the solver reduces the stored FP32 offsets plus the reference in FP64; the dense
                # copy holds the FP32-rounded values
                scale = float(torch.abs(dev.double()).sum().item()) if what == mmfd.MMFD_RED_SUM else abs(ref)
                assert abs(got - ref) <= 1e-7 * max(scale, 1.0), (what, call, got, ref)
        s.set_fields([bad])
        dev = s.fields(0, device=True, dtype=np.float32)[0]
        ref = s.reduce(mmfd.MMFD_RED_NONFINITE)[0]
        assert ref == 37
        for call in range(2):
            mmfd.mmfd_reduce_static(dev.data_ptr(), mmfd.MMFD_DT_F32, dev.numel(), mmfd.MMFD_RED_NONFINITE,
                                    out.data_ptr(), stream)
            torch.cuda.synchronize()
            assert float(out.item()) == ref, (call, out.item())
    finally:
        s.close()


def test_reduce_static_rejects_host_pointers():
    # host memory (pageable or page-locked) is refused before anything is launched: out keeps
    # its sentinel value
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_17057_gb300 import mmfd

    stream = torch.cuda.current_stream().cuda_stream
    out = torch.full((1,), -7.0, dtype=torch.float64, device="cuda")
    dev = torch.ones(1000, dtype=torch.float64, device="cuda")
    host = np.ones(1000)
    pinned = torch.ones(1000, dtype=torch.float64).pin_memory()
    host_out = np.zeros(1)
    cases = [(host.ctypes.data, out.data_ptr()), (pinned.data_ptr(), out.data_ptr()),
             (dev.data_ptr(), host_out.ctypes.data)]
    for field, dst in cases:
        with pytest.raises(mmfd.MMFDError) as e:
            mmfd.mmfd_reduce_static(field, mmfd.MMFD_DT_F64, 1000, mmfd.MMFD_RED_SUM, dst, stream)
        assert e.value.code == mmfd.MMFD_ERR_ARG
    torch.cuda.synchronize()
    assert float(out.item()) == -7.0 and host_out[0] == 0.0
    mmfd.mmfd_reduce_static(dev.data_ptr(), mmfd.MMFD_DT_F64, 1000, mmfd.MMFD_RED_SUM, out.data_ptr(), stream)
    torch.cuda.synchronize()
    assert float(out.item()) == 1000.0
