"""GPU parity of acoustics in a varying medium and of the capacity function
kappa (Eq. (conslaw)) against the oracle: the 1D row kernel, the per-face
classic path (capacity; 2D media-aware transverse splits), SharpClaw, and a
controller run of the heterogeneous 2D acoustics workload.
"""
import numpy as np
import pytest

from paper_1111_6583_gb300 import workloads as wl
from tests.gpu_util import (FP32_SHOCK_L1_TOL, FP32_SMOOTH_TOL, FP64_TOL, gpu_evolve,
                            gpu_fixed_steps, oracle_evolve, oracle_fixed_steps, rel_l1,
                            rel_maxnorm)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("bc", [("periodic", "periodic"), ("wall", "extrap")])
@pytest.mark.parametrize("capa", [-1, 2])
def test_vc_1d_classic(orc, bc, capa):
    kw = {"capa_index": 2} if capa >= 0 else {"num_aux": 2}
    spec = wl.random_1d("acoustics_vc", 700, bc=bc, **kw)
    if capa < 0:
        spec["aux"] = spec["aux"][:2].copy()
    dt = 0.4 / 700
    qo, co = oracle_fixed_steps(orc, spec, dt, 5)
    qg, cg = gpu_fixed_steps(spec, "fp64", dt, 5)
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    assert np.allclose(cg, co, rtol=1e-13, atol=0)


@pytest.mark.parametrize("transverse", [0, 1, 2])
@pytest.mark.parametrize("capa", [-1, 2])
def test_vc_2d_classic_faces(orc, transverse, capa):
    kw = {"capa_index": 2} if capa >= 0 else {"num_aux": 2}
    spec = wl.random_smooth_2d("acoustics_vc", 131, 70, transverse=transverse, **kw)
    if capa < 0:
        spec["aux"] = spec["aux"][:2].copy()
    dt = 0.3 / 131
    qo, co = oracle_fixed_steps(orc, spec, dt, 4)
    qg, cg = gpu_fixed_steps(spec, "fp64", dt, 4)
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    assert np.allclose(cg, co, rtol=1e-13, atol=0)


@pytest.mark.parametrize("ndim", [1, 2])
@pytest.mark.parametrize("rp", ["sw_roe", "euler_roe"])
def test_capacity_classic_conservative_systems(orc, ndim, rp):
    if ndim == 1:
        spec = wl.random_1d(rp, 400, bc=("wall", "extrap"))
        x = (np.arange(400) + 0.5) / 400
        kap = (1.0 + 0.4 * np.sin(2 * np.pi * x))[None]
    else:
        spec = wl.random_smooth_2d(rp, 90, 61, bc="wall")
        X, Y = np.meshgrid((np.arange(90) + 0.5) / 90, (np.arange(61) + 0.5) / 61,
                           indexing="xy")
        kap = (1.0 + 0.4 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y))[None]
    spec.update(num_aux=1, capa_index=0, aux=np.ascontiguousarray(kap))
    dt = 0.2 / spec["n"][0]
    qo, co = oracle_fixed_steps(orc, spec, dt, 4)
    qg, cg = gpu_fixed_steps(spec, "fp64", dt, 4)
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    assert np.allclose(cg, co, rtol=1e-13, atol=0)


@pytest.mark.parametrize("ndim", [1, 2])
@pytest.mark.parametrize("capa", [-1, 2])
def test_vc_sharpclaw(orc, ndim, capa):
    kw = {"capa_index": 2} if capa >= 0 else {"num_aux": 2}
    if ndim == 1:
        spec = wl.random_1d("acoustics_vc", 300, scheme="sharpclaw", **kw)
    else:
        spec = wl.random_smooth_2d("acoustics_vc", 70, 37, scheme="sharpclaw", **kw)
    if capa < 0:
        spec["aux"] = spec["aux"][:2].copy()
    dt = 0.15 / spec["n"][0]
    qo, co = oracle_fixed_steps(orc, spec, dt, 3)
    qg, cg = gpu_fixed_steps(spec, "fp64", dt, 3)
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    assert np.allclose(cg, co, rtol=1e-13, atol=0)


def test_vc_2d_workload_controller(orc):
    """The heterogeneous 2D acoustics workload (impedance jump, stretched
    grid as a capacity, walls) through the controller."""
    spec = wl.acoustics_vc_2d(n=128, t_end=0.3)
    qo, io = oracle_evolve(orc, spec, 0.3)
    for graph in (True, False):
        qg, ig = gpu_evolve(spec, "fp64", 0.3, use_graph=graph)
        assert ig["steps"] == io["steps"] and ig["t"] == io["t"] == 0.3
        assert rel_maxnorm(qg, qo) <= FP64_TOL
    q32, i32 = gpu_evolve(spec, "fp32", 0.3)
    assert i32["t"] == 0.3 and rel_l1(q32, qo) <= FP32_SHOCK_L1_TOL


def test_vc_2d_fp32(orc):
    spec = wl.random_smooth_2d("acoustics_vc", 131, 70, capa_index=2)
    dt = 0.3 / 131
    qo, _ = oracle_fixed_steps(orc, spec, dt, 4)
    qg, _ = gpu_fixed_steps(spec, "fp32", dt, 4)
    assert rel_maxnorm(qg, qo) <= FP32_SMOOTH_TOL


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batches_on_the_per_face_path(orc, prec):
    """Uneven members of the varying-medium, capacity workload in one batch
    (the per-face kernels run member by member inside each captured
    attempt): the same bits as solving each alone; the first against the
    oracle."""
    import torch
    from paper_1111_6583_gb300 import claw
    specs = [wl.acoustics_vc_2d(n=n, t_end=t) for n, t in ((48, 0.2), (64, 0.15), (40, 0.25))]
    b = claw.Batch(specs, prec)
    infos = b.evolve()
    torch.cuda.synchronize()
    for k, sp in enumerate(specs):
        s = claw.Solver(sp, prec)
        ia = s.evolve(sp["t_end"])
        qa = s.q.double().cpu().numpy()
        s.close()
        assert infos[k]["status"] == 0 and infos[k]["t"] == sp["t_end"]
        assert infos[k]["steps"] == ia["steps"]
        assert np.array_equal(qa, b.q[k].double().cpu().numpy())
        if k == 0:
            qo, io = oracle_evolve(orc, sp, sp["t_end"])
            if prec == "fp64":
                assert io["steps"] == ia["steps"]
                assert rel_maxnorm(qa, qo) <= FP64_TOL
            else:
                assert rel_l1(qa, qo) <= FP32_SHOCK_L1_TOL
    b.close()


def test_batches_with_capacity_in_1d(orc):
    import torch
    from paper_1111_6583_gb300 import claw
    specs = []
    for n in (300, 457):
        sp = wl.random_1d("sw_roe", n, char_decomp=0)
        x = (np.arange(n) + 0.5) / n
        sp.update(num_aux=1, capa_index=0, t_end=0.05,
                  aux=np.ascontiguousarray((1.0 + 0.4 * np.sin(2 * np.pi * x))[None]))
        specs.append(sp)
    b = claw.Batch(specs, "fp64")
    infos = b.evolve()
    torch.cuda.synchronize()
    for k, sp in enumerate(specs):
        qo, io = oracle_evolve(orc, sp, sp["t_end"])
        assert infos[k]["steps"] == io["steps"]
        assert rel_maxnorm(b.q[k].double().cpu().numpy(), qo) <= FP64_TOL
    b.close()


@pytest.mark.parametrize("ndim,scheme", [(1, "classic"), (2, "classic"), (2, "sharpclaw")])
def test_conserved_totals_weight_the_capacity(ndim, scheme):
    """claw_conserved_totals returns (sum_i kappa_i Q_i) dV: equal to the sum
    formed here from the initial data, and unchanged by periodic steps
    (shallow water, a conservation law, with a varying capacity)."""
    import torch
    from paper_1111_6583_gb300 import claw
    if ndim == 1:
        spec = wl.random_1d("sw_roe", 150, scheme=scheme, char_decomp=0)
        x = (np.arange(150) + 0.5) / 150
        kap = (1.0 + 0.4 * np.sin(2 * np.pi * x))[None]
    else:
        spec = wl.random_smooth_2d("sw_roe", 48, 36, scheme=scheme, char_decomp=0)
        X, Y = np.meshgrid((np.arange(48) + 0.5) / 48, (np.arange(36) + 0.5) / 36, indexing="xy")
        kap = (1.0 + 0.4 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y))[None]
    spec.update(num_aux=1, capa_index=0, aux=np.ascontiguousarray(kap))
    dV = np.prod([(spec["upper"][d] - spec["lower"][d]) / spec["n"][d] for d in range(ndim)])
    q0 = spec["q0"]
    want = (q0 * spec["aux"][0]).reshape(q0.shape[0], -1).sum(axis=1) * dV
    s = claw.Solver(spec, "fp64")
    t0 = np.array(s.totals())
    assert np.allclose(t0, want, rtol=1e-14, atol=1e-14 * np.abs(want).max())
    for _ in range(6):
        s.step(0.3 / spec["n"][0])
    s.sync()
    torch.cuda.synchronize()
    t1 = np.array(s.totals())
    scale = (np.abs(q0) * spec["aux"][0]).reshape(q0.shape[0], -1).sum(axis=1).max() * dV
    assert np.abs(t1 - t0).max() <= 1e-12 * scale
    s.close()


@pytest.mark.parametrize("sched", [("all", 0), ("srw", 2000)])
def test_server_on_the_per_face_path(orc, sched):
    """Varying-medium, capacity requests through the continuous-batching
    server (a budget that admits one or two at a time): the same bits as
    solving each alone."""
    from paper_1111_6583_gb300 import claw
    specs = [wl.acoustics_vc_2d(n=n, t_end=t) for n, t in ((48, 0.2), (64, 0.15), (40, 0.25))]
    sv = claw.Server(specs[0], "fp64", budget_bytes=3 << 20, max_slots=4)
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
        s = claw.Solver(sp, "fp64")
        ia = s.evolve(sp["t_end"])
        qa = s.q.double().cpu().numpy()
        s.close()
        assert ia["steps"] == r["steps"]
        assert np.array_equal(qa, r["q"].astype(np.float64))


@pytest.mark.parametrize("case", ["sw_capacity", "vc_capacity", "vc"])
def test_dimensional_splitting_on_the_per_face_path(orc, case):
    """Godunov dimensional splitting on the per-face path (x sweeps over dt
    from Q^n, then y sweeps over dt from that state): a capacity field, and
    the varying-medium solver with or without one; fixed steps and a
    controller run against the oracle."""
    if case == "sw_capacity":
        spec = wl.random_smooth_2d("sw_roe", 70, 45, char_decomp=0, transverse=0)
        X, Y = np.meshgrid((np.arange(70) + 0.5) / 70, (np.arange(45) + 0.5) / 45, indexing="xy")
        kap = (1.0 + 0.4 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y))[None]
        spec.update(num_aux=1, capa_index=0, aux=np.ascontiguousarray(kap))
    else:
        spec = wl.acoustics_vc_2d(n=64, t_end=0.2, capacity=(case == "vc_capacity"))
        spec["transverse"] = 0
    spec["dim_split"] = 1
    dt = 0.3 / spec["n"][0]
    qo, co = oracle_fixed_steps(orc, spec, dt, 4)
    qg, cg = gpu_fixed_steps(spec, "fp64", dt, 4)
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    assert np.allclose(cg, co, rtol=1e-13, atol=0)
    t_end = 0.1
    qo, io = oracle_evolve(orc, spec, t_end)
    for graph in (True, False):
        qg, ig = gpu_evolve(spec, "fp64", t_end, use_graph=graph)
        assert ig["status"] == 0 and ig["steps"] == io["steps"] and ig["t"] == t_end
        assert rel_maxnorm(qg, qo) <= FP64_TOL


def _axisym_with_capacity(nx, ny, t, split):
    """The axisymmetric shock-bubble on a grid stretched in z (a capacity
    field), so that the source steps run with the per-face kernels."""
    sp = wl.shock_bubble_axisym(nx=nx, ny=ny, t_end=t, sub=2, source_split=split)
    xi = (np.arange(nx) + 0.5) / nx
    kap = np.broadcast_to(1.0 + 0.2 * np.cos(np.pi * xi), (ny, nx))
    sp.update(num_aux=1, capa_index=0, aux=np.ascontiguousarray(kap[None]))
    return sp


@pytest.mark.parametrize("split", ["godunov", "strang"])
def test_per_face_path_with_source_solver_batch_server(orc, split):
    import torch
    from paper_1111_6583_gb300 import claw
    specs = [_axisym_with_capacity(nx, ny, t, split) for nx, ny, t in ((64, 16, 0.06),
                                                                        (80, 20, 0.05))]
    alone = []
    for k, sp in enumerate(specs):
        s = claw.Solver(sp, "fp64")
        ia = s.evolve(sp["t_end"])
        alone.append((s.q.double().cpu().numpy(), ia))
        s.close()
        if k == 0:
            qo, io = oracle_evolve(orc, sp, sp["t_end"])
            assert io["status"] == "ok" and io["steps"] == ia["steps"]
            assert rel_maxnorm(alone[0][0], qo) <= FP64_TOL
    b = claw.Batch(specs, "fp64")
    infos = b.evolve()
    torch.cuda.synchronize()
    for k in range(len(specs)):
        assert infos[k]["steps"] == alone[k][1]["steps"]
        assert np.array_equal(alone[k][0], b.q[k].double().cpu().numpy())
    b.close()
    sv = claw.Server(specs[0], "fp64", budget_bytes=64 << 20, max_slots=4)
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
    for k, t in enumerate(tickets):
        assert results[t]["steps"] == alone[k][1]["steps"]
        assert np.array_equal(alone[k][0], results[t]["q"].astype(np.float64))
