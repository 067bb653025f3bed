"""Slab decomposition of a single solve (paper_2505_17057_gb300.slab), world sizes 2 and 3 over
gloo on the CPU: every rank steps its slab plus T halo rows with the FP64 oracle, exchanging T
halo rows every T steps (both levels, T = 1, for three-level schemes), and the stitched slabs
equal the single-domain oracle run bit for bit (every owned node sees the same neighbours in the
same order)."""
import os
import socket

import numpy as np
import pytest

import gpu_cases as G
from oracle import oracle as orc
from paper_2505_17057_gb300 import slab as SL

CASES = [
    ("D2Q9", "NSE", 2, [13, 11], 1),
    ("D2Q9", "NSE", 2, [13, 11], 2),
    ("D2Q9", "NCDE", 3, [10, 9], 1),
    ("D3Q19", "NSE", 2, [6, 5, 8], 2),
    ("D3Q7", "LCDE", 3, [5, 4, 7], 1),
]
STEPS = 6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _level(prob, seed, which):
    return G.random_level(prob, np.random.default_rng(seed + which))


def _worker(rank, world, port, case, outdir):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        lat, pde, levels, n, T = case
        _, prob = G.case(lat, pde, levels, n, "fp64")
        L0 = _level(prob, 91, 0)
        L1 = _level(prob, 91, 1) if levels == 3 else None
        sl = SL.make_slab(rank, world, prob.shape[0], T)
        rows = sl.global_rows()
        n_local = list(n[:-1]) + [sl.local_rows]
        _, lprob = G.case(lat, pde, levels, n_local, "fp64")
        cur = [f[rows].copy() for f in L0]
        prev = [f[rows].copy() for f in L1] if L1 is not None else None
        done = 0
        while done < STEPS:
            # owned rows are local rows T .. T + rows - 1
            lv = [cur] + ([prev] if prev is not None else [])
            send_lo = [torch.from_numpy(np.ascontiguousarray(f[T:2 * T])) for L in lv for f in L]
            send_hi = [torch.from_numpy(np.ascontiguousarray(f[sl.rows:sl.rows + T])) for L in lv for f in L]
            recv_lo = [torch.empty_like(t) for t in send_hi]
            recv_hi = [torch.empty_like(t) for t in send_lo]
            SL.exchange(sl, send_lo, send_hi, recv_lo, recv_hi)
            k = 0
            for L in lv:
                for f in L:
                    f[:T] = recv_lo[k].numpy()
                    f[T + sl.rows:] = recv_hi[k].numpy()
                    k += 1
            cur, prev = orc.run(lprob, cur, prev, nsteps=T)
            done += T
        own = [f[T:T + sl.rows] for f in cur]
        np.save(os.path.join(outdir, f"slab{rank}.npy"), np.stack(own))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-{c[1]}-{c[2]}L-T{c[4]}" for c in CASES])
def test_slabs_match_single_domain(tmp_path, world, case):
    import torch.multiprocessing as mp
    lat, pde, levels, n, T = case
    _, prob = G.case(lat, pde, levels, n, "fp64")
    if prob.shape[0] // world < T:
        pytest.skip("slab thinner than its halo")
    mp.spawn(_worker, args=(world, _free_port(), case, str(tmp_path)), nprocs=world, join=True)
    L0 = _level(prob, 91, 0)
    L1 = _level(prob, 91, 1) if levels == 3 else None
    ref, _ = orc.run(prob, L0, L1, nsteps=STEPS)
    got = np.concatenate([np.load(tmp_path / f"slab{r}.npy") for r in range(world)], axis=1)
    for f in range(prob.nf):
        assert np.array_equal(got[f], ref[f]), (f, np.abs(got[f] - ref[f]).max())


def test_partition():
    assert SL.partition(10, 3) == [(0, 4), (4, 7), (7, 10)]
    sl = SL.make_slab(0, 3, 10, 2)
    assert sl.global_rows() == [8, 9, 0, 1, 2, 3, 4, 5]
    assert (sl.prev, sl.next) == (2, 1)
    with pytest.raises(ValueError):
        SL.make_slab(1, 4, 5, 2)
