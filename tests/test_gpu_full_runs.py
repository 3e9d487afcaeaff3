"""GPU against the oracle over whole runs (controller steps to the final time)
at the oracle's sizes of the paper-shaped workloads:

- 2D Euler shock-bubble at 256 x 128 (SharpClaw WENO5-char + SSP-RK3) to
  t = 0.2, FP64 (max-norm 1e-12) and FP32 (L1 1e-4; the data carry shocks);
- the FP32 elasticity ensemble: all 4096 members in one batched launch per
  step to t = 50, three of the smaller members against the oracle run of that
  member alone (L1 1e-4: the nonlinear stress waves steepen into shocks), and
  the smallest member in FP64 one-at-a-time (max-norm 1e-12);
- the axisymmetric shock-bubble (Euler + tracer + geometric source, classic
  full transverse) at 320 x 80 to its final time, FP64.
"""
import numpy as np
import pytest

from paper_1111_6583_gb300 import workloads as wl
from tests.gpu_util import (FP32_SHOCK_L1_TOL, FP64_TOL, gpu_evolve, oracle_evolve, rel_l1,
                            rel_maxnorm)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def test_shock_bubble_256x128_to_final_time(orc):
    spec = wl.shock_bubble_2d(nx=256, ny=128)
    t_end = spec["t_end"]
    qo, io = oracle_evolve(orc, spec, t_end)
    assert io["status"] == "ok" and io["t"] == t_end
    qg, ig = gpu_evolve(spec, "fp64", t_end)
    assert ig["status"] == 0 and ig["t"] == t_end and ig["steps"] == io["steps"]
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    q32, i32 = gpu_evolve(spec, "fp32", t_end)
    assert i32["status"] == 0 and i32["t"] == t_end
    assert rel_l1(q32, qo) <= FP32_SHOCK_L1_TOL


def test_elasticity_ensemble_to_t50(orc):
    import torch
    from paper_1111_6583_gb300 import claw
    ens = wl.elasticity_ensemble(4096)
    specs = [wl.elasticity_member(e["n"], e["amp"], e["width"], t_end=50.0) for e in ens]
    b = claw.Batch(specs, "fp32")
    infos = b.evolve()
    torch.cuda.synchronize()
    q = b.sync()
    assert all(i["status"] == 0 and i["t"] == 50.0 for i in infos)
    sizes = np.array([sp["q0"].shape[1] for sp in specs])
    small = [k for k in np.argsort(sizes) if sizes[k] <= (1 << 14)]
    picks = [int(small[0]), int(small[len(small) // 2]), int(small[-1])]
    for k in picks:
        qo, io = oracle_evolve(orc, specs[k], 50.0)
        assert io["t"] == 50.0
        assert rel_l1(q[k].double().cpu().numpy(), qo) <= FP32_SHOCK_L1_TOL, (k, sizes[k])
    b.close()
    # FP64, the smallest member alone, over the whole run
    k = picks[0]
    qo, io = oracle_evolve(orc, specs[k], 50.0)
    qg, ig = gpu_evolve(specs[k], "fp64", 50.0)
    assert ig["steps"] == io["steps"] and ig["t"] == 50.0
    assert rel_maxnorm(qg, qo) <= FP64_TOL


def test_axisymmetric_320x80_to_final_time(orc):
    spec = wl.shock_bubble_axisym(nx=320, ny=80)
    t_end = spec["t_end"]
    qo, io = oracle_evolve(orc, spec, t_end)
    qg, ig = gpu_evolve(spec, "fp64", t_end)
    assert ig["status"] == 0 and ig["t"] == t_end and ig["steps"] == io["steps"]
    assert rel_maxnorm(qg, qo) <= FP64_TOL
