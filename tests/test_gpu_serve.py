"""GPU tests of the solve server: continuous batching of mixed requests, admission by HBM
footprint, and 'the same result alone and in the mix' (bitwise for the batched kernel, within
the storage tolerance against the single-solve kernels)."""
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


MIX = [
    ("D2Q9", "NSE", 2, [96, 70], "fp32", 37),
    ("D2Q9", "NCDE", 3, [130, 64], "fp32", 25),
    ("D2Q5", "LCDE", 2, [64, 40], "fp64", 50),
    ("D2Q9", "LCDE", 2, [200, 33], "bf16", 19),
    ("D3Q19", "NSE", 2, [24, 20, 18], "fp32", 12),
    ("D3Q7", "LCDE", 3, [30, 17, 9], "fp64", 21),
    ("D2Q9", "NSE", 3, [40, 40], "fp64", 9),
    ("D3Q19", "NCDE", 2, [16, 16, 16], "bf16", 14),
    ("D2Q9", "NSE", 2, [300, 90], "fp32", 3),
    ("D2Q9", "NCDE", 2, [70, 70], "fp32", 0),
    ("D2Q9", "NCDE", 3, [260, 260], "fp32", 7),   # large enough for its own march launches
    ("D2Q9", "NSE", 2, [512, 160], "bf16", 6),
    ("D2Q9", "LCDE", 2, [400, 200], "fp32", 11),  # own launches, temporally blocked
    ("D2Q5", "LCDE", 2, [320, 224], "bf16", 13),  # own launches, temporally blocked
]


def _requests(seed=3):
    rng = np.random.default_rng(seed)
    out = []
    for lat, pde, levels, n, st, steps in MIX:
        kw, prob = G.case(lat, pde, levels, n, st)
        out.append((kw, prob, G.random_level(prob, rng), steps))
    return out


def _serve(mm, reqs, budget=1 << 30, slots=64, spt=8, graphs=True):
    srv = mm.Server(budget, max_slots=slots, steps_per_tick=spt, use_graphs=graphs)
    tickets = [srv.submit(mm.make_desc(**kw), L0, steps) for kw, _, L0, steps in reqs]
    srv.drain()
    res = []
    for t in tickets:
        rc, r = srv.poll(t)
        assert rc == mm.MMFD_OK and r.status == 0
        res.append(srv.result(t))
        srv.release(t)
    st = srv.stats()
    srv.close()
    return res, st


def test_mix_equals_alone_bitwise(mm):
    reqs = _requests()
    mixed, st = _serve(mm, reqs)
    assert st["submitted"] == len(reqs) and st["finished"] == len(reqs)
    assert st["graph_replays"] > 0
    for i, r in enumerate(reqs):
        # the same steps per tick: requests stepped with their own blocked launches split each
        # tick into blocks, so their rounding depends on the tick length
        alone, _ = _serve(mm, [r], spt=8, graphs=False)
        for a, b in zip(mixed[i], alone[0]):
            assert np.array_equal(a, b), MIX[i]


def test_mix_matches_single_solve_and_oracle(mm):
    reqs = _requests(seed=4)
    mixed, _ = _serve(mm, reqs)
    for (kw, prob, L0, steps), out, spec in zip(reqs, mixed, MIX):
        st = spec[4]
        d = mm.make_desc(**kw)
        s = mm.Solver(d)
        s.set_fields(L0)
        stored0 = s.fields(0)
        s.step(steps)
        single = s.fields(0)
        s.close()
        tol = {"fp64": 1e-12, "fp32": 1e-5, "bf16": 2e-2}[st]
        assert G.rel_err(out, single) < tol, (spec, G.rel_err(out, single))
        if st == "fp64":
            ref, _ = orc.run(prob, L0, L0 if prob.levels == 3 else None, nsteps=steps)
            assert G.rel_err(out, ref) < 1e-12, spec
        elif st == "fp32":
            # served FP32 requests against the FP64 oracle, started from the values FP32 storage holds
            ref, _ = orc.run(prob, stored0, stored0 if prob.levels == 3 else None, nsteps=steps)
            assert G.rel_err(out, ref) < 1e-5, (spec, G.rel_err(out, ref))


def test_admission_by_footprint(mm):
    reqs = _requests(seed=5)[:6]
    # budget that fits only a few requests at a time: the rest wait in the queue
    d0 = mm.make_desc(**reqs[0][0])
    info = mm.mmfd_describe(d0)
    budget = 3 * max(1, info.bytes_per_lu) * 96 * 70 * 4
    res_small, st = _serve(mm, reqs, budget=int(budget), slots=2)
    res_big, _ = _serve(mm, reqs)
    for a, b in zip(res_small, res_big):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    srv = mm.Server(1 << 16, max_slots=4)
    kw, prob, L0, steps = reqs[0]
    with pytest.raises(mm.MMFDError) as e:
        srv.submit(mm.make_desc(**kw), L0, steps)
    assert e.value.code == mm.MMFD_ERR_ADMISSION
    srv.close()


def test_arrivals_while_running(mm):
    reqs = _requests(seed=6)
    srv = mm.Server(1 << 30, max_slots=4, steps_per_tick=4)
    first = [srv.submit(mm.make_desc(**kw), L0, steps) for kw, _, L0, steps in reqs[:3]]
    for _ in range(3):
        for t in first:
            srv.poll(t)
    later = [srv.submit(mm.make_desc(**kw), L0, steps) for kw, _, L0, steps in reqs[3:]]
    pending = set(first + later)
    guard = 0
    while pending and guard < 100000:
        for t in list(pending):
            rc, r = srv.poll(t)
            if rc == mm.MMFD_OK:
                assert r.finish_s >= r.admit_s >= r.submit_s
                pending.discard(t)
                srv.release(t)
        guard += 1
    assert not pending
    st = srv.stats()
    assert st["finished"] == len(reqs) and st["ticks"] > 0
    srv.close()


@pytest.mark.parametrize("graphs", [True, False])
def test_work_queue_equals_per_step_batch(mm, monkeypatch, graphs):
    # MMFD_SERVE_QUEUE=1: every batched class runs all steps of a tick as one launch of the
    # device-resident work queue (k_batch_queue), each tile waiting for its request's previous
    # step; the node update is the per-step kernel's, so the results are equal bit for bit
    reqs = _requests(seed=8)
    per_step, st1 = _serve(mm, reqs, graphs=graphs)
    monkeypatch.setenv("MMFD_SERVE_QUEUE", "1")
    queued, st2 = _serve(mm, reqs, graphs=graphs)
    assert st2["launches"] < st1["launches"], (st1["launches"], st2["launches"])
    for a, b, spec in zip(queued, per_step, MIX):
        for x, y in zip(a, b):
            assert np.array_equal(x, y), spec


def test_work_queue_wait_runs_out_and_reports(mm, monkeypatch):
    # failure detection without a GPU fault: with MMFD_SERVE_QUEUE_STALL=1 no tile's wait for its
    # request's previous step can be met, so every wait gives up after its bounded budget (about a
    # second), the kernel records the timeout in the server's device flag and the result call
    # reports MMFD_ERR_TIMEOUT; the context stays usable
    monkeypatch.setenv("MMFD_SERVE_QUEUE", "1")
    monkeypatch.setenv("MMFD_SERVE_QUEUE_STALL", "1")
    kw, prob = G.case("D2Q9", "LCDE", 2, [64, 40], "fp32")
    L0 = G.random_level(prob, np.random.default_rng(1))
    srv = mm.Server(1 << 30, max_slots=4, steps_per_tick=4)
    t = srv.submit(mm.make_desc(**kw), L0, 6)
    srv.drain()
    with pytest.raises(mm.MMFDError) as e:
        srv.result(t)
    assert e.value.code == mm.MMFD_ERR_TIMEOUT
    srv.release(t)
    srv.close()
    monkeypatch.delenv("MMFD_SERVE_QUEUE_STALL")
    res, _ = _serve(mm, _requests(seed=8)[:3])
    assert len(res) == 3
