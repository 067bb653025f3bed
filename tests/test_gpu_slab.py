"""Slab decomposition of one solve on the GPU, emulated on one device: R solvers each step their
slab plus one halo row (plane) as a periodic grid and swap halo rows through mmfd_get_rows /
mmfd_set_rows between steps (paper_2505_17057_gb300/slab.py bookkeeping).  The stitched slabs
equal the single-domain solver bit for bit: every owned node is updated by the same kernel from
the same neighbour values in the same order.  Plus the row-range transfers against full-level
ones."""
import numpy as np
import pytest

import gpu_cases as G
from paper_2505_17057_gb300 import slab as SL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_17057_gb300 import mmfd
    return mmfd


def _dt(mm, storage):
    return (np.float64, mm.MMFD_DT_F64) if storage == "fp64" else (np.float32, mm.MMFD_DT_F32)


def run_slabs(mm, kw, L0, L1, nranks, steps):
    import torch
    storage = kw["storage"]
    npdt, _ = _dt(mm, storage)
    # halo rows travel as FP64 values: exact for every storage (an FP32 offset from the reference
    # state, or a BF16 one, comes back unchanged), so the slabs stay bitwise equal to one grid
    dt, tdt = mm.MMFD_DT_F64, torch.float64
    n_axis = L0[0].shape[0]
    slabs = [SL.make_slab(r, nranks, n_axis, 1) for r in range(nranks)]
    solvers = []
    for sl in slabs:
        n_local = list(kw["n"][:-1]) + [sl.local_rows]
        s = mm.Solver(mm.make_desc(**{**kw, "n": n_local}))
        rows = sl.global_rows()
        s.set_fields([f[rows] for f in L0])
        if L1 is not None:
            s.set_fields([f[rows] for f in L1], level=1)
        solvers.append(s)
    levels = [0, 1] if L1 is not None else [0]
    row_shape = L0[0].shape[1:]
    nf = len(L0)

    def buf():
        return [torch.empty(row_shape, dtype=tdt, device="cuda") for _ in range(nf)]

    for _ in range(steps):
        for lv in levels:
            # first / last owned row of every slab, then into the neighbours' halo rows
            lo = [buf() for _ in slabs]
            hi = [buf() for _ in slabs]
            for k, (sl, s) in enumerate(zip(slabs, solvers)):
                mm.mmfd_get_rows(s.h, lv, 1, 1, [t.data_ptr() for t in lo[k]], mm.MMFD_DEVICE, dt)
                mm.mmfd_get_rows(s.h, lv, sl.rows, 1, [t.data_ptr() for t in hi[k]], mm.MMFD_DEVICE, dt)
            for k, (sl, s) in enumerate(zip(slabs, solvers)):
                mm.mmfd_set_rows(s.h, lv, 0, 1, [t.data_ptr() for t in hi[sl.prev]], mm.MMFD_DEVICE, dt)
                mm.mmfd_set_rows(s.h, lv, sl.rows + 1, 1, [t.data_ptr() for t in lo[sl.next]], mm.MMFD_DEVICE, dt)
        for s in solvers:
            s.step(1)
    out = []
    for sl, s in zip(slabs, solvers):
        f = s.fields(0, dtype=npdt)
        out.append([x[1:1 + sl.rows] for x in f])
        s.close()
    return [np.concatenate([o[f] for o in out], axis=0) for f in range(nf)]


CASES = [
    ("D2Q9", "NSE", 2, [256, 21], "fp32", None),                    # lean kernel (streaming momentum)
    ("D2Q9", "NSE", 2, [300, 19], "fp32", {"dx": [1.0, 1.1]}),      # general pair form
    ("D2Q9", "LCDE", 3, [200, 17], "fp64", None),                   # three-level: both levels exchanged
    ("D2Q9", "NCDE", 3, [130, 12], "bf16", None),
    ("D3Q19", "NSE", 2, [140, 9, 11], "fp32", None),                # z slabs
    ("D3Q7", "LCDE", 2, [128, 6, 9], "fp32", None),
]


@pytest.mark.parametrize("nranks", [2, 3])
@pytest.mark.parametrize("lat,pde,levels,n,storage,over", CASES)
def test_slabs_equal_single_domain(mm, lat, pde, levels, n, storage, over, nranks):
    rng = np.random.default_rng(40 + levels)
    kw, prob = G.case(lat, pde, levels, n, storage)
    if pde == "NSE" and over is None:
        kw.update(dx=[1.0] * len(n), a=(1.0, 0.0, 0.0), abar=(1.0, 0.0, 0.0), ahat=(0, 0, 0), abarhat=(0, 0, 0))
    if over:
        kw.update(over)
    L0 = G.random_level(prob, rng)
    L1 = G.random_level(prob, rng) if levels == 3 else None
    npdt, _ = _dt(mm, storage)
    s = mm.Solver(mm.make_desc(**kw))
    try:
        s.set_fields(L0)
        if L1 is not None:
            s.set_fields(L1, level=1)
        s.step(5)
        ref = s.fields(0, dtype=npdt)
    finally:
        s.close()
    got = run_slabs(mm, kw, L0, L1, nranks, 5)
    for f in range(len(ref)):
        assert np.array_equal(got[f], ref[f]), (f, np.abs(got[f] - ref[f]).max())


@pytest.mark.parametrize("storage", ["fp64", "fp32", "bf16"])
def test_rows_match_full_level(mm, storage):
    rng = np.random.default_rng(9)
    kw, prob = G.case("D3Q19", "NSE", 2, [130, 7, 6], storage)
    L0 = G.random_level(prob, rng)
    s = mm.Solver(mm.make_desc(**kw))
    try:
        s.set_fields(L0)
        full = s.fields(0)
        part = [np.empty((2,) + f.shape[1:]) for f in full]
        mm.mmfd_get_rows(s.h, 0, 3, 2, [p.ctypes.data for p in part], mm.MMFD_HOST, mm.MMFD_DT_F64)
        for p, f in zip(part, full):
            assert np.array_equal(p, f[3:5])
        # overwrite planes 4 and 5 (the periodic image of the last plane follows)
        new = [rng.standard_normal((2,) + f.shape[1:]) * 0.01 + f[:2] for f in full]
        mm.mmfd_set_rows(s.h, 0, 4, 2, [np.ascontiguousarray(x).ctypes.data for x in new], mm.MMFD_HOST,
                         mm.MMFD_DT_F64)
        after = s.fields(0)
        for f, a in zip(full, after):
            assert np.array_equal(a[:4], f[:4])
        # the stored values, and their periodic images (a step reads them), are those set_fields of
        # the same values stores
        s.step(2)
        stepped = s.fields(0)
        expect = [np.concatenate([f[:4], x], axis=0) for f, x in zip(full, new)]
        s.set_fields(expect)
        for a, w in zip(after, s.fields(0)):
            assert np.array_equal(a, w)
        s.step(2)
        for a, w in zip(stepped, s.fields(0)):
            assert np.array_equal(a, w)
        with pytest.raises(mm.MMFDError):
            mm.mmfd_get_rows(s.h, 0, 5, 2, [p.ctypes.data for p in part], mm.MMFD_HOST, mm.MMFD_DT_F64)
    finally:
        s.close()
