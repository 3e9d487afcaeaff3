"""GPU parity of SharpClaw with WENO of orders 7 to 17 (Sec. 2.1 and the
PyWENO subsection) against the oracle, whose coefficients come from an
independent exact derivation: every Riemann solver in 1D, the 2D systems,
component- and characteristic-wise, boundary conditions that reach the
wider ghost layers (4 to 9 cells), FP32, and the shock-bubble with WENO7 +
SSP(10,4) through the controller.  Orders 15 and 17 take the smoothness
indicators' full quadratic forms in the definitions' order on both sides.
"""
import numpy as np
import pytest

from paper_1111_6583_gb300 import workloads as wl
from tests.gpu_util import (FP32_SMOOTH_TOL, FP64_TOL, gpu_evolve, gpu_fixed_steps,
                            oracle_evolve, oracle_fixed_steps, rel_maxnorm)

pytestmark = pytest.mark.gpu

RPS_1D = ["advection", "acoustics", "sw_roe", "euler_roe", "euler_hlle", "elasticity_fwave"]
RPS_2D = ["advection", "acoustics", "sw_roe", "euler_roe", "euler_hlle"]
ORDERS = [7, 9, 11, 13, 15, 17]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("rp", RPS_1D)
@pytest.mark.parametrize("char", [0, 1])
def test_weno_order_1d_fp64(orc, order, rp, char):
    if rp == "elasticity_fwave" and char:
        pytest.skip("no characteristic projection for f-wave elasticity")
    spec = wl.random_1d(rp, 300, scheme="sharpclaw", char_decomp=char, weno_order=order)
    dt = 0.15 / 300
    qo, co = oracle_fixed_steps(orc, spec, dt, 3)
    qg, cg = gpu_fixed_steps(spec, "fp64", dt, 3)
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    assert np.allclose(cg, co, rtol=1e-13, atol=0)


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("rp", RPS_2D)
def test_weno_order_2d_fp64(orc, order, rp):
    spec = wl.random_smooth_2d(rp, 70, 37, scheme="sharpclaw", char_decomp=1, weno_order=order)
    dt = 0.1 / 70
    qo, _ = oracle_fixed_steps(orc, spec, dt, 2)
    qg, _ = gpu_fixed_steps(spec, "fp64", dt, 2)
    assert rel_maxnorm(qg, qo) <= FP64_TOL


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("bc", ["wall", "extrap"])
def test_weno_order_boundaries(orc, order, bc):
    """Ghost layers of width 4 to 9 filled by wall and extrapolation rules."""
    s1 = wl.random_1d("euler_roe", 64, bc=(bc, bc), scheme="sharpclaw", char_decomp=1,
                      weno_order=order)
    qo, _ = oracle_fixed_steps(orc, s1, 0.1 / 64, 3)
    qg, _ = gpu_fixed_steps(s1, "fp64", 0.1 / 64, 3)
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    s2 = wl.random_smooth_2d("sw_roe", 33, 21, bc=bc, scheme="sharpclaw", char_decomp=1,
                             weno_order=order)
    qo, _ = oracle_fixed_steps(orc, s2, 0.1 / 33, 2)
    qg, _ = gpu_fixed_steps(s2, "fp64", 0.1 / 33, 2)
    assert rel_maxnorm(qg, qo) <= FP64_TOL


@pytest.mark.parametrize("order", ORDERS)
def test_weno_order_2d_fp32(orc, order):
    spec = wl.random_smooth_2d("euler_roe", 70, 37, scheme="sharpclaw", char_decomp=1,
                               weno_order=order)
    dt = 0.1 / 70
    qo, _ = oracle_fixed_steps(orc, spec, dt, 2)
    qg, _ = gpu_fixed_steps(spec, "fp32", dt, 2)
    assert rel_maxnorm(qg, qo) <= FP32_SMOOTH_TOL


def test_shock_bubble_weno7_ssp104_controller(orc):
    """The paper's shock-bubble comparison runs WENO5 against WENO7; here the
    planar form at 64 x 32 with WENO7 + SSP(10,4) (inflow, extrapolation and
    wall ghosts) through the CFL controller, steps and state as the oracle."""
    spec = wl.shock_bubble_2d(nx=64, ny=32, t_end=0.1, sub=4)
    spec.update(weno_order=7, time_integrator="ssp104", cfl_desired=2.0, cfl_max=2.5)
    qo, io = oracle_evolve(orc, spec, 0.1)
    qg, ig = gpu_evolve(spec, "fp64", 0.1)
    assert io["status"] == "ok" and ig["status"] == 0
    assert ig["steps"] == io["steps"] and ig["t"] == io["t"] == 0.1
    assert rel_maxnorm(qg, qo) <= FP64_TOL
