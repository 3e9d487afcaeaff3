"""3D classic step (transverse + double-transverse terms) on the GPU against
the CPU oracle."""
import numpy as np
import pytest

from paper_1111_6583_gb300 import workloads as wl
from tests.gpu_util import (FP32_SMOOTH_TOL, FP64_TOL, gpu_evolve, gpu_fixed_steps,
                            oracle_evolve, oracle_fixed_steps, rel_maxnorm)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("rp", ["advection", "acoustics"])
@pytest.mark.parametrize("order,transverse", [(2, 2), (2, 1), (1, 1), (2, 0)])
def test_3d_fixed_dt_fp64(orc, rp, order, transverse):
    spec = wl.random_3d(rp, 13, 11, 9, order=order, transverse=transverse)
    dt = 0.25 / 13
    qo, co = oracle_fixed_steps(orc, spec, dt, 4)
    qg, cg = gpu_fixed_steps(spec, "fp64", dt, 4)
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    assert np.allclose(cg, co, rtol=1e-13, atol=0)


@pytest.mark.parametrize("bc", ["wall", "extrap"])
def test_3d_acoustics_boundaries(orc, bc):
    spec = wl.random_3d("acoustics", 12, 10, 14, bc=bc)
    spec["bc_lower"] = [bc, "periodic", "wall"]
    spec["bc_upper"] = ["extrap", "periodic", bc]
    dt = 0.2 / 14
    qo, _ = oracle_fixed_steps(orc, spec, dt, 5)
    qg, _ = gpu_fixed_steps(spec, "fp64", dt, 5)
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    q32, _ = gpu_fixed_steps(spec, "fp32", dt, 5)
    assert rel_maxnorm(q32, qo) <= FP32_SMOOTH_TOL


@pytest.mark.parametrize("rp", ["advection", "acoustics"])
def test_3d_several_patches_and_segments(orc, rp):
    """Grids that span several 14 x 14 patches of owner lines (ragged last
    patches) and several 32-cell segments along each sweep, with mixed
    boundaries; FP64 against the oracle, FP32 against it too."""
    spec = wl.random_3d(rp, 70, 33, 45, bc="wall")
    spec["bc_lower"] = ["periodic", "wall", "extrap"]
    spec["bc_upper"] = ["periodic", "extrap", "wall"]
    dt = 0.2 / 70
    qo, co = oracle_fixed_steps(orc, spec, dt, 3)
    qg, cg = gpu_fixed_steps(spec, "fp64", dt, 3)
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    assert np.allclose(cg, co, rtol=1e-13, atol=0)
    q32, _ = gpu_fixed_steps(spec, "fp32", dt, 3)
    assert rel_maxnorm(q32, qo) <= FP32_SMOOTH_TOL


@pytest.mark.parametrize("n3", [(56, 9, 31), (29, 10, 33), (5, 4, 4)])
def test_3d_x_sweep_chunks(orc, n3):
    """The x sweep's decomposition: 28 owned cells per warp (nx = 56 puts the
    last face in the halo lane of the second chunk), ten owner lines per
    block (lines -1 .. ny-1: ny = 9 fills one block exactly, ny = 10 leaves
    one line for a second block), 32 owner planes per segment (nz + 1 = 32
    exactly; nz = 33: a second segment), and a grid smaller than one chunk
    (four cells, the smallest a direction may have)."""
    spec = wl.random_3d("acoustics", *n3, bc="wall")
    spec["bc_lower"] = ["wall", "extrap", "periodic"]
    spec["bc_upper"] = ["extrap", "wall", "periodic"]
    dt = 0.2 / max(n3)
    qo, co = oracle_fixed_steps(orc, spec, dt, 3)
    qg, cg = gpu_fixed_steps(spec, "fp64", dt, 3)
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    assert np.allclose(cg, co, rtol=1e-13, atol=0)
    q32, _ = gpu_fixed_steps(spec, "fp32", dt, 3)
    assert rel_maxnorm(q32, qo) <= FP32_SMOOTH_TOL


@pytest.mark.parametrize("rp", ["acoustics", "advection"])
def test_3d_inflow_boundaries(orc, rp):
    """Inflow faces in each direction (the ghost cells take a given state)
    beside walls and extrapolation, over several x chunks, y blocks and z
    segments; FP64 and FP32 against the oracle."""
    spec = wl.random_3d(rp, 61, 12, 35, bc="extrap")
    spec["bc_lower"] = ["inflow", "inflow", "extrap"]
    spec["bc_upper"] = ["extrap", "wall" if rp == "acoustics" else "extrap", "inflow"]
    spec["inflow"] = list(np.asarray(spec["q0"])[:, 0, 0, 0] * 1.05)
    dt = 0.2 / 61
    qo, co = oracle_fixed_steps(orc, spec, dt, 3)
    qg, cg = gpu_fixed_steps(spec, "fp64", dt, 3)
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    assert np.allclose(cg, co, rtol=1e-13, atol=0)
    q32, _ = gpu_fixed_steps(spec, "fp32", dt, 3)
    assert rel_maxnorm(q32, qo) <= FP32_SMOOTH_TOL


def test_3d_diagonal_shift():
    n = 16
    spec = wl.random_3d("advection", n, n, n, params=[1.0, 1.0, 1.0], order=2, transverse=2)
    qg, cg = gpu_fixed_steps(spec, "fp64", 1.0 / n, 1)
    assert cg[0] == 1.0
    assert np.abs(qg - np.roll(spec["q0"], (1, 1, 1), axis=(1, 2, 3))).max() <= 1e-14


def test_3d_controller_run(orc):
    spec = wl.random_3d("acoustics", 16, 12, 10, bc="wall")
    qo, io = oracle_evolve(orc, spec, 0.15)
    qg, ig = gpu_evolve(spec, "fp64", 0.15)
    assert ig["steps"] == io["steps"] and ig["t"] == 0.15
    assert rel_maxnorm(qg, qo) <= FP64_TOL


def _batch_specs(rp, bc):
    specs = []
    for k, (n3, te) in enumerate([((16, 12, 10), 0.15), ((9, 13, 11), 0.08), ((20, 8, 6), 0.2)]):
        sp = wl.random_3d(rp, *n3, seed=wl.SEED + 31 * k, bc=bc)
        sp["t_end"] = te
        specs.append(sp)
    return specs


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("rp,bc", [("acoustics", "wall"), ("advection", "periodic")])
def test_3d_batch_members_match_oracle(orc, rp, bc, use_graph):
    """A batch of 3D grids of different shapes and end times: each member takes
    the oracle's CFL steps and ends at its own t_end with the oracle's state."""
    import torch
    from paper_1111_6583_gb300 import claw
    specs = _batch_specs(rp, bc)
    b = claw.Batch(specs, "fp64")
    infos = b.evolve(use_graph=use_graph)
    torch.cuda.synchronize()
    for k, sp in enumerate(specs):
        qo, io = oracle_evolve(orc, sp, sp["t_end"])
        assert infos[k]["steps"] == io["steps"] and infos[k]["t"] == sp["t_end"], k
        assert rel_maxnorm(b.q[k].double().cpu().numpy(), qo) <= FP64_TOL, k
    b.close()


def test_3d_batch_fp32_matches_solvers():
    """FP32 3D batch members against FP32 single-grid solvers of the same
    grids, bit for bit (every face value has one writer in a fixed order)."""
    import torch
    from paper_1111_6583_gb300 import claw
    specs = _batch_specs("acoustics", "wall")
    b = claw.Batch(specs, "fp32")
    infos = b.evolve()
    torch.cuda.synchronize()
    for k, sp in enumerate(specs):
        s = claw.Solver(sp, "fp32")
        ia = s.evolve(sp["t_end"])
        assert infos[k]["steps"] == ia["steps"] and infos[k]["t"] == ia["t"], k
        qa = s.q.double().cpu().numpy()
        assert np.array_equal(b.q[k].double().cpu().numpy(), qa), k
        s.close()
    b.close()


@pytest.mark.parametrize("sched", [("all", 0), ("srw", 1500)])
def test_3d_server_matches_solver_and_oracle(orc, sched):
    """3D requests of different shapes and end times through the continuous-
    batching server (a budget that admits one or two at a time): each takes
    the single-grid solver's CFL steps and ends at its state bit for bit, and
    at the FP64 oracle's within the parity bound."""
    from paper_1111_6583_gb300 import claw
    specs = _batch_specs("acoustics", "wall")
    sv = claw.Server(specs[0], "fp64", budget_bytes=1 << 20, max_slots=4)
    sv.schedule(*sched)
    tickets = [sv.submit(sp) for sp in specs]
    done = {}
    guard = 0
    while len(done) < len(tickets):
        sv.pump(3)
        for t in sv.take_done():
            done[t] = sv.poll(t)
        guard += 1
        assert guard < 100000
    sv.close()
    for t, sp in zip(tickets, specs):
        r = done[t]
        assert r["status"] == "ok" and r["t"] == sp["t_end"]
        s = claw.Solver(sp, "fp64")
        ia = s.evolve(sp["t_end"])
        qa = s.q.double().cpu().numpy()
        s.close()
        assert ia["steps"] == r["steps"]
        assert np.array_equal(r["q"], qa)
        qo, io = oracle_evolve(orc, sp, sp["t_end"])
        assert io["steps"] == r["steps"] and rel_maxnorm(r["q"], qo) <= FP64_TOL


def test_1d_advection_server_takes_its_dimension_from_the_grid():
    """A one-field method is ambiguous between dimensions; the server made
    from a 1D spec serves 1D grids and refuses others."""
    from paper_1111_6583_gb300 import claw
    sp = wl.random_1d("advection", 200)
    sp["t_end"] = 0.1
    sv = claw.Server(sp, "fp64", budget_bytes=1 << 24, max_slots=2)
    t = sv.submit(sp)
    with pytest.raises(RuntimeError):
        sv.submit(wl.random_3d("advection", 8, 8, 8))
    while not sv.take_done():
        sv.pump(4)
    r = sv.poll(t)
    sv.close()
    s = claw.Solver(sp, "fp64")
    ia = s.evolve(0.1)
    qa = s.q.double().cpu().numpy()
    s.close()
    assert r["status"] == "ok" and r["steps"] == ia["steps"]
    assert np.array_equal(qa, r["q"].astype(np.float64))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n3", [(37, 29, 23), (70, 15, 33)])
def test_3d_runs_are_bitwise_repeatable(prec, n3):
    """The same 3D run twice, on grids whose patches and segments have ragged
    edges, gives the same bits (no result depends on the order in which blocks
    run)."""
    from paper_1111_6583_gb300 import claw
    spec = wl.random_3d("acoustics", *n3, bc="wall")
    out = []
    for _ in range(2):
        s = claw.Solver(spec, prec)
        info = s.evolve(0.05)
        out.append(s.q.double().cpu().numpy())
        s.close()
        assert info["status"] == 0
    assert np.array_equal(out[0], out[1])
