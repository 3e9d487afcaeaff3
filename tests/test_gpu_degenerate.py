"""Degenerate cases of the step on the GPU.

- A uniform state (periodic boundaries) is a steady state: every jump is
  zero, so every wave, fluctuation, limiter ratio and transverse piece is
  zero, and the classic update returns the state bit for bit (HLLE forms its
  middle state by a division, and WENO normalises its weights, so those two
  hold it to rounding).  The zero-wave branch of every limiter form (the
  dot-product one, the wave-strength ratio, the FP64 division-free one) is
  what runs here.
- Evolving to the current time takes no step and leaves the state alone.
- A step limit stops the run after that many accepted steps, short of t_end.
"""
import numpy as np
import pytest

from paper_1111_6583_gb300 import workloads as wl
from tests.gpu_util import gpu_fixed_steps, rel_maxnorm

pytestmark = pytest.mark.gpu

RPS_1D = ["advection", "acoustics", "sw_roe", "euler_roe", "euler_hlle", "elasticity_fwave"]
RPS_2D = ["advection", "acoustics", "sw_roe", "euler_roe", "euler_hlle"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _uniform(spec, rp):
    """The spec with q0 replaced by its mean over the cells (a physical state:
    the admissible sets are convex); zero for elasticity, whose layered medium
    keeps only the state of zero strain and velocity at rest."""
    q0 = np.asarray(spec["q0"], dtype=np.float64)
    axes = tuple(range(1, q0.ndim))
    if rp == "elasticity_fwave":
        u = np.zeros_like(q0)
    else:
        u = np.broadcast_to(q0.mean(axis=axes, keepdims=True), q0.shape).copy()
    spec = dict(spec)
    spec["q0"] = u
    return spec


def _check_steady(spec, rp, prec, dt, nsteps, exact):
    q, _ = gpu_fixed_steps(spec, prec, dt, nsteps)
    ref = np.asarray(spec["q0"], dtype=np.float32 if prec == "fp32" else np.float64)
    ref = ref.astype(np.float64)
    if exact or not ref.any():
        # (the zero state stays zero in every form: each product has a zero)
        assert np.array_equal(q, ref), (rp, prec, np.abs(q - ref).max())
    else:
        assert rel_maxnorm(q, ref) <= (1e-14 if prec == "fp64" else 2e-6), rp


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("rp", RPS_1D)
def test_uniform_state_steady_1d(rp, prec):
    spec = _uniform(wl.random_1d(rp, 257, jump=False), rp)
    _check_steady(spec, rp, prec, 0.2 / 257, 5, exact=rp != "euler_hlle")
    spec["scheme"] = "sharpclaw"
    _check_steady(spec, rp, prec, 0.2 / 257, 2, exact=False)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("rp", RPS_2D)
def test_uniform_state_steady_2d(rp, prec):
    spec = _uniform(wl.random_smooth_2d(rp, 67, 45), rp)
    _check_steady(spec, rp, prec, 0.2 / 67, 4, exact=rp != "euler_hlle")
    spec["scheme"] = "sharpclaw"
    _check_steady(spec, rp, prec, 0.2 / 67, 2, exact=False)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("rp", ["advection", "acoustics"])
def test_uniform_state_steady_3d(rp, prec):
    spec = _uniform(wl.random_3d(rp, 33, 14, 11), rp)
    _check_steady(spec, rp, prec, 0.2 / 33, 3, exact=True)


def test_evolve_to_current_time_takes_no_step():
    import torch
    from paper_1111_6583_gb300 import claw
    spec = wl.sw_dambreak_2d(n=96)
    s = claw.Solver(spec, "fp64", t0=0.25)
    before = s.q.clone()
    info = s.evolve(0.25)
    torch.cuda.synchronize()
    assert info["status"] == claw.CLAW_OK
    assert info["steps"] == 0 and info["t"] == 0.25
    assert torch.equal(s.sync(), before)
    s.close()


def test_step_limit_stops_short_of_t_end():
    import torch
    from paper_1111_6583_gb300 import claw
    spec = wl.sw_dambreak_2d(n=96)
    s = claw.Solver(spec, "fp64")
    info = s.evolve(1.5, max_steps=3)
    torch.cuda.synchronize()
    assert info["steps"] == 3 and 0.0 < info["t"] < 1.5
    info2 = s.evolve(1.5)
    assert info2["t"] == 1.5 and info2["steps"] > 3
    s.close()
