"""GPU parity of SharpClaw with the ten-stage fourth-order SSP(10,4) time
integrator (Sec. 2.1; Ketcheson 2008, low-storage form) against the oracle:
fixed steps in 1D and 2D, the CFL controller at Courant numbers above one
(the method's SSP coefficient is 6), and batched members equal to solves
alone.
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


@pytest.mark.parametrize("rp", ["advection", "acoustics", "sw_roe", "euler_roe",
                                "euler_hlle", "elasticity_fwave"])
def test_ssp104_1d_fixed_dt_fp64(orc, rp):
    char = 0 if rp == "elasticity_fwave" else 1
    spec = wl.random_1d(rp, 300, scheme="sharpclaw", char_decomp=char,
                        time_integrator="ssp104")
    dt = 0.5 / 300
    qo, co = oracle_fixed_steps(orc, spec, dt, 3)
    qg, cg = gpu_fixed_steps(spec, "fp64", dt, 3)
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    assert np.allclose(cg, co, rtol=1e-13, atol=0)


@pytest.mark.parametrize("rp", ["acoustics", "sw_roe", "euler_roe"])
def test_ssp104_2d_fixed_dt_fp64(orc, rp):
    spec = wl.random_smooth_2d(rp, 70, 37, scheme="sharpclaw", char_decomp=1,
                                time_integrator="ssp104")
    dt = 0.3 / 70
    qo, _ = oracle_fixed_steps(orc, spec, dt, 2)
    qg, _ = gpu_fixed_steps(spec, "fp64", dt, 2)
    assert rel_maxnorm(qg, qo) <= FP64_TOL


def test_ssp104_2d_fp32(orc):
    spec = wl.random_smooth_2d("euler_roe", 70, 37, scheme="sharpclaw", char_decomp=1,
                                time_integrator="ssp104")
    dt = 0.3 / 70
    qo, _ = oracle_fixed_steps(orc, spec, dt, 2)
    qg, _ = gpu_fixed_steps(spec, "fp32", dt, 2)
    assert rel_maxnorm(qg, qo) <= FP32_SMOOTH_TOL


@pytest.mark.parametrize("use_graph", [True, False])
def test_ssp104_controller_above_unit_cfl(orc, use_graph):
    """Acoustics pulse, WENO5 + SSP(10,4) at cfl_desired 2.0 / cfl_max 2.5:
    same accepted steps, rejections and final time as the oracle."""
    spec = wl.random_1d("acoustics", 500, scheme="sharpclaw", char_decomp=1,
                        time_integrator="ssp104", cfl_desired=2.0, cfl_max=2.5)
    qo, io = oracle_evolve(orc, spec, 0.6)
    qg, ig = gpu_evolve(spec, "fp64", 0.6, use_graph=use_graph)
    assert ig["steps"] == io["steps"] and ig["rejects"] == io["rejects"]
    assert ig["t"] == io["t"] == 0.6
    assert io["cfl_max_seen"] > 1.5
    assert rel_maxnorm(qg, qo) <= FP64_TOL


def test_ssp104_reject_and_retry(orc):
    """An initial dt far above the stable step is rejected and retried."""
    spec = wl.random_1d("sw_roe", 256, scheme="sharpclaw", char_decomp=1,
                        time_integrator="ssp104", cfl_desired=2.0, cfl_max=2.5,
                        dt_initial=0.01)
    qo, io = oracle_evolve(orc, spec, 0.1)
    qg, ig = gpu_evolve(spec, "fp64", 0.1)
    assert io["rejects"] >= 1 and ig["rejects"] == io["rejects"]
    assert ig["steps"] == io["steps"]
    assert rel_maxnorm(qg, qo) <= FP64_TOL


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ssp104_batch_equals_alone(orc, prec):
    import torch
    from paper_1111_6583_gb300 import claw
    specs = []
    for k, n in enumerate([64, 300, 1025]):
        sp = wl.elasticity_member(n, 0.2 + 0.1 * k, 2.0 + k, t_end=0.5 + 0.1 * k)
        sp.update(scheme="sharpclaw", char_decomp=0, time_integrator="ssp104",
                  cfl_desired=2.0, cfl_max=2.5)
        specs.append(sp)
    b = claw.Batch(specs, prec)
    infos = b.evolve()
    torch.cuda.synchronize()
    for k, sp in enumerate(specs):
        s = claw.Solver(sp, prec)
        ia = s.evolve(sp["t_end"])
        qa = s.q.double().cpu().numpy()
        s.close()
        assert infos[k]["steps"] == ia["steps"] and infos[k]["t"] == sp["t_end"]
        assert np.array_equal(qa, b.q[k].double().cpu().numpy())
        if prec == "fp64":
            qo, io = oracle_evolve(orc, sp, sp["t_end"])
            assert io["steps"] == ia["steps"]
            assert rel_maxnorm(qa, qo) <= FP64_TOL
    b.close()
