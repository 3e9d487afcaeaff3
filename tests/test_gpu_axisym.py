"""GPU parity of the axisymmetric shock-bubble pieces (Sec. 7.2) against the
oracle: the Euler Roe solver with a passive tracer (classic and SharpClaw),
dimensionally split classic steps, and the geometric source applied after
accepted steps only (Godunov splitting), alone and in batches.
"""
import numpy as np
import pytest

from paper_1111_6583_gb300 import workloads as wl
from tests.gpu_util import (FP32_SHOCK_L1_TOL, FP64_TOL, gpu_evolve, gpu_fixed_steps,
                            oracle_evolve, oracle_fixed_steps, rel_l1, rel_maxnorm)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("transverse", [0, 1, 2])
def test_tracer_classic2d_fixed_dt(orc, transverse):
    spec = wl.random_smooth_2d("euler_tracer", 131, 70, transverse=transverse)
    dt = 0.25 / 131
    qo, co = oracle_fixed_steps(orc, spec, dt, 4)
    qg, cg = gpu_fixed_steps(spec, "fp64", dt, 4)
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    assert np.allclose(cg, co, rtol=1e-13, atol=0)


@pytest.mark.parametrize("scheme,char", [("classic", 0), ("sharpclaw", 0), ("sharpclaw", 1)])
def test_tracer_1d(orc, scheme, char):
    spec = wl.random_1d("euler_tracer", 300, scheme=scheme, char_decomp=char)
    dt = 0.15 / 300
    qo, _ = oracle_fixed_steps(orc, spec, dt, 3)
    qg, _ = gpu_fixed_steps(spec, "fp64", dt, 3)
    assert rel_maxnorm(qg, qo) <= FP64_TOL


@pytest.mark.parametrize("char", [0, 1])
def test_tracer_sharpclaw2d(orc, char):
    spec = wl.random_smooth_2d("euler_tracer", 70, 37, scheme="sharpclaw", char_decomp=char)
    dt = 0.1 / 70
    qo, _ = oracle_fixed_steps(orc, spec, dt, 3)
    qg, _ = gpu_fixed_steps(spec, "fp64", dt, 3)
    assert rel_maxnorm(qg, qo) <= FP64_TOL


@pytest.mark.parametrize("rp", ["advection", "acoustics", "sw_roe", "euler_roe", "euler_tracer"])
@pytest.mark.parametrize("order", [1, 2])
def test_dimensional_splitting_fixed_dt(orc, rp, order):
    spec = wl.random_smooth_2d(rp, 131, 70, order=order, dim_split=1, transverse=0)
    dt = 0.25 / 131
    qo, co = oracle_fixed_steps(orc, spec, dt, 4)
    qg, cg = gpu_fixed_steps(spec, "fp64", dt, 4)
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    assert np.allclose(cg, co, rtol=1e-13, atol=0)


def test_dimensional_splitting_controller(orc):
    """Split steps through the controller (three state buffers, the result
    two slots on): the dam break to t = 0.4."""
    spec = wl.sw_dambreak_2d(n=128, t_end=0.4)
    spec.update(dim_split=1, transverse=0)
    qo, io = oracle_evolve(orc, spec, 0.4)
    for graph in (True, False):
        qg, ig = gpu_evolve(spec, "fp64", 0.4, use_graph=graph)
        assert ig["steps"] == io["steps"] and ig["t"] == io["t"] == 0.4
        assert rel_maxnorm(qg, qo) <= FP64_TOL


@pytest.mark.parametrize("dim_split", [0, 1])
def test_axisymmetric_shock_bubble(orc, dim_split):
    spec = wl.shock_bubble_axisym(nx=160, ny=40, t_end=0.1, sub=4, dim_split=dim_split)
    if dim_split:
        spec["transverse"] = 0
    qo, io = oracle_evolve(orc, spec, 0.1)
    assert io["status"] == "ok"
    for graph in (True, False):
        qg, ig = gpu_evolve(spec, "fp64", 0.1, use_graph=graph)
        assert ig["status"] == 0 and ig["steps"] == io["steps"] and ig["t"] == 0.1
        assert rel_maxnorm(qg, qo) <= FP64_TOL
    q32, i32 = gpu_evolve(spec, "fp32", 0.1)
    assert i32["status"] == 0 and rel_l1(q32, qo) <= FP32_SHOCK_L1_TOL


def test_source_follows_accepted_steps_only(orc):
    """A first dt far above the stable one is rejected and retried; the
    source step runs once per accepted step (steps, rejects and state as the
    oracle's)."""
    spec = wl.shock_bubble_axisym(nx=80, ny=20, t_end=0.05, sub=4)
    spec["dt_initial"] = 0.02
    qo, io = oracle_evolve(orc, spec, 0.05)
    qg, ig = gpu_evolve(spec, "fp64", 0.05)
    assert io["rejects"] >= 1 and ig["rejects"] == io["rejects"]
    assert ig["steps"] == io["steps"]
    assert rel_maxnorm(qg, qo) <= FP64_TOL


def test_axisymmetric_batch_equals_alone(orc):
    import torch
    from paper_1111_6583_gb300 import claw
    specs = [wl.shock_bubble_axisym(nx=nx, ny=ny, t_end=t, sub=4)
             for nx, ny, t in ((80, 20, 0.05), (120, 30, 0.04), (64, 16, 0.06))]
    b = claw.Batch(specs, "fp64")
    infos = b.evolve()
    torch.cuda.synchronize()
    for k, sp in enumerate(specs):
        s = claw.Solver(sp, "fp64")
        ia = s.evolve(sp["t_end"])
        qa = s.q.double().cpu().numpy()
        s.close()
        assert infos[k]["steps"] == ia["steps"] and infos[k]["t"] == sp["t_end"]
        assert np.array_equal(qa, b.q[k].double().cpu().numpy())
        if k == 0:
            qo, io = oracle_evolve(orc, sp, sp["t_end"])
            assert io["steps"] == ia["steps"] and rel_maxnorm(qa, qo) <= FP64_TOL
    b.close()


@pytest.mark.parametrize("split", ["godunov", "strang"])
@pytest.mark.parametrize("budget_kb", [512 << 10, 300])
@pytest.mark.parametrize("sched", [("all", 0), ("srw", 1500)])
def test_server_with_source_equals_alone(orc, split, budget_kb, sched):
    """Axisymmetric shock-bubble requests of different sizes and final times
    through the continuous-batching server (a 300 KB budget admits about one
    at a time; Strang requests carry their half-step buffer) give the same
    states as solving each alone."""
    from paper_1111_6583_gb300 import claw
    specs = [wl.shock_bubble_axisym(nx=nx, ny=ny, t_end=t, sub=2, source_split=split)
             for nx, ny, t in ((64, 16, 0.06), (96, 24, 0.05), (80, 20, 0.07))]
    sv = claw.Server(specs[0], "fp64", budget_bytes=budget_kb << 10, max_slots=4)
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
    for k, (t, sp) in enumerate(zip(tickets, specs)):
        r = results[t]
        assert r["status"] == "ok" and r["t"] == sp["t_end"]
        s = claw.Solver(sp, "fp64")
        ia = s.evolve(sp["t_end"])
        qa = s.q.double().cpu().numpy()
        s.close()
        assert ia["steps"] == r["steps"]
        assert np.array_equal(qa, r["q"].astype(np.float64))
        if k == 0:
            qo, io = oracle_evolve(orc, sp, sp["t_end"])
            assert rel_maxnorm(r["q"], qo) <= FP64_TOL


# --------------------------------------------------------------------------
# Strang splitting of the source: half before the step, half after it
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim_split", [0, 1])
def test_strang_axisymmetric_shock_bubble(orc, dim_split):
    spec = wl.shock_bubble_axisym(nx=160, ny=40, t_end=0.1, sub=4, dim_split=dim_split,
                                  source_split="strang")
    if dim_split:
        spec["transverse"] = 0
    qo, io = oracle_evolve(orc, spec, 0.1)
    assert io["status"] == "ok"
    for graph in (True, False):
        qg, ig = gpu_evolve(spec, "fp64", 0.1, use_graph=graph)
        assert ig["status"] == 0 and ig["steps"] == io["steps"] and ig["t"] == 0.1
        assert rel_maxnorm(qg, qo) <= FP64_TOL
    q32, i32 = gpu_evolve(spec, "fp32", 0.1)
    assert i32["status"] == 0 and rel_l1(q32, qo) <= FP32_SHOCK_L1_TOL


def test_strang_fixed_dt_differs_from_godunov(orc):
    """Fixed steps, long enough for the shock to reach the bubble (before
    that the radial momentum is at rounding level and a per-field relative
    norm means nothing): each splitting matches its own oracle run, and the
    two differ (the source is active)."""
    out = {}
    for split in ("godunov", "strang"):
        spec = wl.shock_bubble_axisym(nx=96, ny=24, t_end=0.05, sub=4, source_split=split)
        dt = 0.2 / 96
        qo, co = oracle_fixed_steps(orc, spec, dt, 40)
        qg, cg = gpu_fixed_steps(spec, "fp64", dt, 40)
        assert rel_maxnorm(qg, qo) <= FP64_TOL
        assert np.allclose(cg, co, rtol=1e-13, atol=0)
        out[split] = qg
    assert np.abs(out["godunov"] - out["strang"]).max() > 1e-3


def test_strang_rejected_attempt_keeps_qn(orc):
    """A first dt far above the stable one: the rejected attempt has already
    written the half-source state, but into its own buffer, so the retry
    starts from Q^n (steps, rejects and state as the oracle's)."""
    spec = wl.shock_bubble_axisym(nx=80, ny=20, t_end=0.05, sub=4, source_split="strang")
    spec["dt_initial"] = 0.02
    qo, io = oracle_evolve(orc, spec, 0.05)
    for graph in (True, False):
        qg, ig = gpu_evolve(spec, "fp64", 0.05, use_graph=graph)
        assert io["rejects"] >= 1 and ig["rejects"] == io["rejects"]
        assert ig["steps"] == io["steps"]
        assert rel_maxnorm(qg, qo) <= FP64_TOL


@pytest.mark.parametrize("integrator", ["ssp_rk3", "ssp104"])
def test_strang_sharpclaw(orc, integrator):
    """SharpClaw stages read the half-source state wherever they read Q^n
    (run until the shock has reached the bubble, so that every field is well
    above rounding level)."""
    spec = wl.shock_bubble_axisym(nx=96, ny=24, t_end=0.06, sub=4, scheme="sharpclaw",
                                  source_split="strang")
    spec.update(char_decomp=1, time_integrator=integrator, cfl_desired=0.5, cfl_max=0.6)
    qo, io = oracle_evolve(orc, spec, 0.06)
    qg, ig = gpu_evolve(spec, "fp64", 0.06)
    assert ig["status"] == 0 and ig["steps"] == io["steps"]
    assert rel_maxnorm(qg, qo) <= FP64_TOL


def test_strang_batch_equals_alone(orc):
    import torch
    from paper_1111_6583_gb300 import claw
    specs = [wl.shock_bubble_axisym(nx=nx, ny=ny, t_end=t, sub=4, source_split="strang")
             for nx, ny, t in ((80, 20, 0.07), (120, 30, 0.06))]
    b = claw.Batch(specs, "fp64")
    infos = b.evolve()
    torch.cuda.synchronize()
    for k, sp in enumerate(specs):
        s = claw.Solver(sp, "fp64")
        ia = s.evolve(sp["t_end"])
        qa = s.q.double().cpu().numpy()
        s.close()
        assert infos[k]["steps"] == ia["steps"] and infos[k]["t"] == sp["t_end"]
        assert np.array_equal(qa, b.q[k].double().cpu().numpy())
        if k == 0:
            qo, io = oracle_evolve(orc, sp, sp["t_end"])
            assert io["steps"] == ia["steps"] and rel_maxnorm(qa, qo) <= FP64_TOL
    b.close()
