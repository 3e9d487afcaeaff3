"""GPU parity at the workloads' full sizes, in the launch configuration the
bench times (autotuned tiles, CUDA graphs of step attempts, the fused batch
launch): a few steps each, compared with the oracle element by element (the
oracle finishes a few steps of these sizes in seconds).

- 2D shallow-water dam break, 1024 x 1024, classic FP64 (the headline) and FP32;
- 2D Euler shock-bubble, 2048 x 1024, SharpClaw WENO5-char + SSP-RK3, FP64 and FP32;
- axisymmetric shock-bubble, 1280 x 320, classic + source, FP64;
- the 4096-member FP32 elasticity ensemble (90.7 M cells, one batch), sampled
  members compared with the oracle run of that member alone;
- the Table 1 acoustics system: 2D at 1024^2, 3D at 64^3;
- the 2^26-cell 1D acoustics line of the roofline variant, FP64 and FP32.
FP32 runs are compared with the FP64 oracle (L1 where the data have jumps).
"""
import numpy as np
import pytest

from paper_1111_6583_gb300 import workloads as wl
from tests.gpu_util import (FP32_SHOCK_L1_TOL, FP32_SMOOTH_TOL, FP64_TOL, oracle_evolve, rel_l1,
                            rel_maxnorm)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _gpu_steps(spec, prec, t_end, steps):
    """The bench's path: autotuned tiles, graph-captured attempts."""
    import torch
    from paper_1111_6583_gb300 import claw
    s = claw.Solver(spec, prec)
    s.tune()
    info = s.evolve(t_end, max_steps=steps, use_graph=True)
    torch.cuda.synchronize()
    q = s.q.double().cpu().numpy()
    s.close()
    return q, info


def test_headline_dambreak_1024_fp64_and_fp32(orc):
    spec = wl.sw_dambreak_2d(n=1024)
    qo, io = oracle_evolve(orc, spec, 1.5, max_steps=8)
    qg, ig = _gpu_steps(spec, "fp64", 1.5, 8)
    assert ig["status"] == 0 and ig["steps"] == io["steps"] == 8
    assert ig["t"] == pytest.approx(io["t"], rel=1e-14)
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    q32, i32 = _gpu_steps(spec, "fp32", 1.5, 8)
    assert i32["status"] == 0 and rel_l1(q32, qo) <= FP32_SHOCK_L1_TOL


def test_shock_bubble_2048x1024_fp64_and_fp32(orc):
    spec = wl.shock_bubble_2d()
    qo, io = oracle_evolve(orc, spec, spec["t_end"], max_steps=1)
    qg, ig = _gpu_steps(spec, "fp64", spec["t_end"], 1)
    assert ig["status"] == 0 and ig["steps"] == io["steps"] == 1
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    q32, i32 = _gpu_steps(spec, "fp32", spec["t_end"], 1)
    assert i32["status"] == 0 and rel_l1(q32, qo) <= FP32_SHOCK_L1_TOL


def test_axisymmetric_1280x320_fp64(orc):
    spec = wl.shock_bubble_axisym()
    qo, io = oracle_evolve(orc, spec, spec["t_end"], max_steps=6)
    qg, ig = _gpu_steps(spec, "fp64", spec["t_end"], 6)
    assert ig["status"] == 0 and ig["steps"] == io["steps"] == 6
    assert rel_maxnorm(qg, qo) <= FP64_TOL


def test_elasticity_ensemble_4096_sampled(orc):
    """The whole ensemble in one FP32 batch (30 controller steps per member,
    enough for the velocity, zero at the start, to reach the scale of the
    stress wave); members of the smallest, a middle and the largest size
    against the FP64 oracle."""
    import torch
    from paper_1111_6583_gb300 import claw
    ens = wl.elasticity_ensemble(4096)
    specs = [wl.elasticity_member(e["n"], e["amp"], e["width"], t_end=e["t_end"]) for e in ens]
    b = claw.Batch(specs, "fp32")
    infos = b.evolve(max_steps=30)
    torch.cuda.synchronize()
    sizes = np.array([sp["q0"].shape[1] for sp in specs])
    picks = [int(np.argmin(sizes)), int(np.argsort(sizes)[len(sizes) // 2]), int(np.argmax(sizes))]
    q = b.sync()
    for k in picks:
        qo, io = oracle_evolve(orc, specs[k], specs[k]["t_end"], max_steps=30)
        assert infos[k]["steps"] == io["steps"] == 30
        assert rel_maxnorm(q[k].double().cpu().numpy(), qo) <= FP32_SMOOTH_TOL, k
    b.close()


@pytest.mark.parametrize("nd,n,steps", [(2, 1024, 6), (3, 64, 4)])
def test_table1_acoustics(orc, nd, n, steps):
    """The paper's Table 1 acoustics system in the bench's configuration: 2D at
    the bench size, 3D at 64^3 (the oracle's 3D step is slow at 256^3)."""
    spec = wl.acoustics_2d(n=n) if nd == 2 else wl.acoustics_3d(n=n)
    qo, io = oracle_evolve(orc, spec, spec["t_end"], max_steps=steps)
    run = _gpu_steps if nd == 2 else _gpu_steps_untuned
    qg, ig = run(spec, "fp64", spec["t_end"], steps)
    assert ig["status"] == 0 and ig["steps"] == io["steps"] == steps
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    q32, i32 = run(spec, "fp32", spec["t_end"], steps)
    assert i32["status"] == 0 and rel_l1(q32, qo) <= FP32_SHOCK_L1_TOL


def _gpu_steps_untuned(spec, prec, t_end, steps):
    import torch
    from paper_1111_6583_gb300 import claw
    s = claw.Solver(spec, prec)
    info = s.evolve(t_end, max_steps=steps, use_graph=True)
    torch.cuda.synchronize()
    q = s.q.double().cpu().numpy()
    s.close()
    return q, info


def test_acoustics_1d_2p26(orc):
    """The 2^26-cell 1D acoustics line the bench times (FP32 staged through
    the shared-memory ring, FP64 direct), two controller steps each, every
    cell against the oracle."""
    spec = wl.acoustics_1d(n=1 << 26, t_end=1e9)
    qo, io = oracle_evolve(orc, spec, 1e9, max_steps=2)
    qg, ig = _gpu_steps_untuned(spec, "fp64", 1e9, 2)
    assert ig["status"] == 0 and ig["steps"] == io["steps"] == 2
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    del qg
    q32, i32 = _gpu_steps_untuned(spec, "fp32", 1e9, 2)
    assert i32["status"] == 0 and i32["steps"] == 2
    assert rel_l1(q32, qo) <= FP32_SHOCK_L1_TOL
