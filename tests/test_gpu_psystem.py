"""GPU parity of the 2D p-system in a checkerboard medium (Sec. 7.3: f-wave
normal solves with per-cell (rho, K), SharpClaw WENO) against the oracle.
"""
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


@pytest.mark.parametrize("order,integrator", [(5, "ssp_rk3"), (5, "ssp104"), (7, "ssp_rk3"),
                                              (9, "ssp104")])
def test_psystem_fixed_dt_fp64(orc, order, integrator):
    spec = wl.random_smooth_2d("elasticity_fwave", 72, 40, weno_order=order,
                               time_integrator=integrator)
    dt = (0.3 if integrator == "ssp_rk3" else 0.8) / 72
    qo, co = oracle_fixed_steps(orc, spec, dt, 3)
    qg, cg = gpu_fixed_steps(spec, "fp64", dt, 3)
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    assert np.allclose(cg, co, rtol=1e-13, atol=0)


def test_psystem_fp32(orc):
    spec = wl.random_smooth_2d("elasticity_fwave", 72, 40)
    dt = 0.3 / 72
    qo, _ = oracle_fixed_steps(orc, spec, dt, 3)
    qg, _ = gpu_fixed_steps(spec, "fp32", dt, 3)
    assert rel_maxnorm(qg, qo) <= FP32_SMOOTH_TOL


@pytest.mark.parametrize("integrator", ["ssp_rk3", "ssp104"])
def test_checkerboard_quadrant_controller(orc, integrator):
    """The paper's setup at reduced size: 3 x 3 material periods of 16 cells,
    walls at x = 0 and y = 0, extrapolation at the far sides, the Gaussian
    stress pulse at the origin; evolved through the CFL controller."""
    cfl = (0.5, 0.6) if integrator == "ssp_rk3" else (1.0, 1.2)
    spec = wl.psystem_checkerboard_2d(periods=3, cells_per_period=16, t_end=0.6,
                                      integrator=integrator, cfl=cfl)
    qo, io = oracle_evolve(orc, spec, 0.6)
    qg, ig = gpu_evolve(spec, "fp64", 0.6)
    assert io["status"] == "ok" and ig["status"] == 0
    assert ig["steps"] == io["steps"] and ig["rejects"] == io["rejects"]
    assert ig["t"] == io["t"] == 0.6
    assert rel_maxnorm(qg, qo) <= FP64_TOL


def test_psystem_batch_equals_alone(orc):
    import torch
    from paper_1111_6583_gb300 import claw
    specs = [wl.psystem_checkerboard_2d(periods=p, cells_per_period=c, t_end=t)
             for p, c, t in ((2, 16, 0.3), (3, 12, 0.5), (2, 24, 0.4))]
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
    b.close()
