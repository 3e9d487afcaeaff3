"""Batched and served solves: every member's result is the same alone and in
the mix (same kernels, same per-member controller), and matches the oracle.
"""
import numpy as np
import pytest

from paper_1111_6583_gb300 import workloads as wl
from tests.gpu_util import FP64_TOL, oracle_evolve, rel_maxnorm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _ensemble(sizes, t_end):
    rng = np.random.Generator(np.random.PCG64(11))
    specs = []
    for k, n in enumerate(sizes):
        sp = wl.elasticity_member(n, float(rng.uniform(0.1, 0.5)), float(rng.uniform(1, 5)),
                                  t_end=t_end * (1.0 + 0.3 * k / len(sizes)))
        specs.append(sp)
    return specs


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_equals_alone(orc, prec, use_graph):
    import torch
    from paper_1111_6583_gb300 import claw
    specs = _ensemble([64, 100, 1000, 4096, 5003, 9000], t_end=2.0)
    b = claw.Batch(specs, prec)
    infos = b.evolve(use_graph=use_graph)
    torch.cuda.synchronize()
    for k, sp in enumerate(specs):
        s = claw.Solver(sp, prec)
        ia = s.evolve(sp["t_end"])
        qa = s.q.double().cpu().numpy()
        qb = b.q[k].double().cpu().numpy()
        assert infos[k]["steps"] == ia["steps"] and infos[k]["t"] == ia["t"] == sp["t_end"]
        assert np.array_equal(qa, qb), k
        s.close()
        if prec == "fp64" and k < 3:
            qo, io = oracle_evolve(orc, sp, sp["t_end"])
            assert io["steps"] == ia["steps"]
            assert rel_maxnorm(qb, qo) <= FP64_TOL
    b.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("budget_mb", [4096, 3])
@pytest.mark.parametrize("sched", [("all", 0), ("srw", 1 << 22), ("srw", 2500)])
def test_server_equals_alone(orc, prec, budget_mb, sched):
    """Requests of different sizes and final times through the continuous-
    batching server (a 3 MB budget admits one or two at a time; every running
    request stepped per attempt, or the least remaining work first with a
    cell threshold that picks one or two of them) give the same states as
    solving each alone."""
    import torch
    from paper_1111_6583_gb300 import claw
    reqs = [(48, [(0.5, 0.1, 0.4, 0.5)], 0.3), (96, [(0.3, 0.2, 0.6, 0.6)], 0.5),
            (64, [(0.8, 0.05, 0.5, 0.3), (0.2, 0.3, 0.3, 0.7)], 0.2),
            (120, [(0.4, 0.15, 0.5, 0.5)], 0.4)]
    specs = [wl.sw_humps_2d(n, humps, t) for n, humps, t in reqs]
    sv = claw.Server(specs[0], prec, budget_bytes=budget_mb << 20, max_slots=8)
    sv.schedule(*sched)
    tickets = [sv.submit(sp) for sp in specs]
    results = {}
    guard = 0
    while len(results) < len(tickets):
        sv.pump(4)
        for t in tickets:
            if t not in results:
                r = sv.poll(t)
                if r is not None:
                    results[t] = r
        guard += 1
        assert guard < 100000
    sv.close()
    for t, sp in zip(tickets, specs):
        r = results[t]
        assert r["status"] == "ok" and r["t"] == sp["t_end"]
        s = claw.Solver(sp, prec)
        ia = s.evolve(sp["t_end"])
        qa = s.q.double().cpu().numpy()
        s.close()
        assert ia["steps"] == r["steps"]
        assert np.array_equal(qa, r["q"].astype(np.float64))
        if prec == "fp64":
            qo, io = oracle_evolve(orc, sp, sp["t_end"])
            assert rel_maxnorm(r["q"], qo) <= FP64_TOL


def test_server_rejects_request_beyond_budget():
    from paper_1111_6583_gb300 import claw
    sp = wl.sw_humps_2d(256, [(0.5, 0.1, 0.5, 0.5)], 0.1)
    sv = claw.Server(sp, "fp32", budget_bytes=1 << 20, max_slots=4)
    with pytest.raises(claw.ClawError) as ei:
        sv.submit(sp)
    assert ei.value.status == claw.CLAW_EBUDGET
    sv.close()


def _host_pair(spec, prec):
    import torch
    dt = torch.float64 if prec == "fp64" else torch.float32
    hin = torch.as_tensor(spec["q0"], dtype=dt).pin_memory()
    return hin, torch.empty_like(hin).pin_memory()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(64, 41), (128, 7), (64, 3)])
def test_step_host_equals_device_steps(prec, shape):
    """claw_step_host from host buffers: two calls of one attempt give the same
    bits as one call of two attempts and as the device-resident solver."""
    import torch
    from paper_1111_6583_gb300 import claw
    spec = wl.random_smooth_2d("sw_roe", 131, 29 if shape[1] == 3 else 70)
    a = claw.Solver(spec, prec)
    a.tune(*shape)
    b = claw.Solver(spec, prec)
    b.tune(*shape)
    c = claw.Solver(spec, prec)
    c.tune(*shape)
    ain, aout = _host_pair(spec, prec)
    bin_, bout = _host_pair(spec, prec)
    for _ in range(3):
        assert a.step_host(ain, aout, 1) == 0
        assert a.step_host(aout, ain, 1) == 0
        assert b.step_host(bin_, bout, 2) == 0
        bin_, bout = bout, bin_
        c.step()
        c.step()
    c.sync()
    torch.cuda.synchronize()
    assert np.array_equal(ain.numpy(), bin_.numpy())
    assert np.array_equal(ain.numpy(), c.q.cpu().numpy())
    for s in (a, b, c):
        s.close()


def test_step_host_rejected_attempt():
    """A first dt far above the stable one: the single attempt is rejected and
    the output is the input; the next call takes the shrunk dt.  Two calls
    equal one call of two attempts."""
    from paper_1111_6583_gb300 import claw
    spec = wl.random_smooth_2d("sw_roe", 131, 70, dt_initial=0.5)
    a = claw.Solver(spec, "fp64")
    a.tune(64, 41)
    b = claw.Solver(spec, "fp64")
    b.tune(64, 41)
    ain, aout = _host_pair(spec, "fp64")
    bin_, bout = _host_pair(spec, "fp64")
    assert a.step_host(ain, aout, 1) == 0
    assert np.array_equal(aout.numpy(), ain.numpy())
    assert a.info()["rejects"] == 1 and a.info()["steps"] == 0
    assert a.step_host(aout, ain, 1) == 0
    assert b.step_host(bin_, bout, 2) == 0
    assert np.array_equal(ain.numpy(), bout.numpy())
    assert a.info()["steps"] == 1
    a.close()
    b.close()


@pytest.mark.parametrize("policy", ["all", "srw"])
def test_server_schedule_order(policy):
    """A small grid with a long final time (more steps, less work) beside a
    larger grid with a short one: stepping every request per attempt finishes
    the larger (fewer steps) first; the shortest-remaining-work schedule, with
    a threshold the small grid meets alone, finishes the small one first.
    Both end at their t_end either way."""
    from paper_1111_6583_gb300 import claw
    big = wl.sw_humps_2d(96, [(0.2, 0.1, 0.5, 0.5)], 0.3)
    small = wl.sw_humps_2d(32, [(0.2, 0.1, 0.5, 0.5)], 1.5)
    sv = claw.Server(big, "fp32", budget_bytes=1 << 30, max_slots=4)
    sv.schedule(policy, 32 * 32)
    tb, ts = sv.submit(big), sv.submit(small)
    done = {}
    guard = 0
    while len(done) < 2:
        sv.pump(2)
        for t in (tb, ts):
            if t not in done:
                r = sv.poll(t, want_state=False)
                if r is not None:
                    done[t] = (r, len(done))
        guard += 1
        assert guard < 100000
    sv.close()
    first = ts if policy == "srw" else tb
    assert done[first][1] == 0
    assert done[ts][0]["status"] == "ok" and done[tb][0]["status"] == "ok"
    assert done[tb][0]["t"] == 0.3 and done[ts][0]["t"] == 1.5
    assert done[ts][0]["steps"] > done[tb][0]["steps"]


def test_server_schedule_rejects_bad_arguments():
    from paper_1111_6583_gb300 import claw
    sv = claw.Server(wl.sw_humps_2d(32, [], 0.1), "fp32", budget_bytes=1 << 26, max_slots=2)
    with pytest.raises(RuntimeError):
        sv.schedule("srw", 0)
    lib = claw.load()
    assert lib.claw_server_schedule(sv.h, 7, 1) != 0
    sv.close()


def test_server_take_done_lists_each_finished_request_once():
    from paper_1111_6583_gb300 import claw
    specs = [wl.sw_humps_2d(n, [(0.3, 0.1, 0.5, 0.5)], t) for n, t in ((32, 0.1), (48, 0.2),
                                                                     (40, 0.05))]
    sv = claw.Server(specs[0], "fp32", budget_bytes=1 << 28, max_slots=4)
    tickets = [sv.submit(sp) for sp in specs]
    seen = []
    guard = 0
    while len(seen) < len(tickets):
        sv.pump(4)
        got = sv.take_done(cap=1)  # at most one per call; the rest wait
        while got:
            seen += got
            got = sv.take_done(cap=1)
        guard += 1
        assert guard < 100000
    assert sorted(seen) == sorted(tickets) and len(set(seen)) == len(seen)
    assert sv.take_done() == []
    for t, sp in zip(tickets, specs):
        r = sv.poll(t, want_state=False)
        assert r["status"] == "ok" and r["t"] == sp["t_end"]
    sv.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_server_1d_requests_match_single_solves(orc, prec):
    """1D requests (elasticity in the layered medium, uneven sizes, a budget
    that admits a few at a time) through the pipelined server: each result
    equals its single solve bit for bit, and the FP64 ones the oracle."""
    from paper_1111_6583_gb300 import claw
    specs = [wl.elasticity_member(n, a, w, t_end=t)
             for n, a, w, t in ((300, 0.3, 2.0, 3.0), (1000, 0.2, 3.0, 2.0),
                                (4099, 0.4, 1.5, 1.0), (777, 0.25, 2.5, 4.0))]
    sv = claw.Server(specs[0], prec, budget_bytes=1 << 20, max_slots=8)
    tickets = [sv.submit(sp) for sp in specs]
    results, guard = {}, 0
    while len(results) < len(tickets):
        sv.pump(3)
        for t in sv.take_done():
            results[t] = sv.poll(t)
        guard += 1
        assert guard < 100000
    sv.close()
    for t, sp in zip(tickets, specs):
        r = results[t]
        assert r["status"] == "ok" and r["t"] == sp["t_end"]
        s = claw.Solver(sp, prec)
        ia = s.evolve(sp["t_end"])
        qa = s.q.double().cpu().numpy()
        s.close()
        assert ia["steps"] == r["steps"]
        assert np.array_equal(qa, r["q"].astype(np.float64))
        if prec == "fp64":
            qo, io = oracle_evolve(orc, sp, sp["t_end"])
            assert rel_maxnorm(r["q"], qo) <= FP64_TOL


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_step_host_rejected_attempt_returns_qn(prec):
    """claw_step_host whose only attempt is rejected (a first dt far above the
    stable one, no retries): CLAW_ECFL, and the state copied back is Q^n
    (the device moves it into the slot the host reads)."""
    import torch
    from paper_1111_6583_gb300 import claw
    spec = wl.random_smooth_2d("sw_roe", 96, 64, dt_initial=0.5, max_retries=0)
    s = claw.Solver(spec, prec)
    hin, hout = _host_pair(spec, prec)
    st = s.step_host(hin, hout, 1)
    torch.cuda.synchronize()
    s.close()
    assert st == claw.CLAW_ECFL
    assert torch.equal(hout, hin)
