"""GPU parity: the CUDA kernels (through the C ABI) against the CPU oracle on
the same seeded inputs, element by element.

Sizes span several tiles with ragged tails (1D tiles of 240 cells in FP64 and 480 in FP32; 2D
strips of 60/124 columns and row segments of 8..128 rows; SharpClaw tiles of
16x8 and 128 cells).  FP64 tolerance: max-norm relative 1e-12; FP32: 1e-5
relative on smooth data, L1 1e-4 where the data have jumps.
"""
import numpy as np
import pytest

from paper_1111_6583_gb300 import workloads as wl
from tests.gpu_util import (FP32_SHOCK_L1_TOL, FP32_SMOOTH_TOL, FP64_TOL, gpu_evolve,
                            gpu_fixed_steps, oracle_evolve, oracle_fixed_steps, rel_l1,
                            rel_maxnorm)

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


# --------------------------------------------------------------------------
# classic 1D, fixed dt
# --------------------------------------------------------------------------
@pytest.mark.parametrize("rp", RPS_1D)
@pytest.mark.parametrize("lim", ["mc", "minmod", "superbee", "vanleer", "none"])
def test_classic1d_fixed_dt_fp64(orc, rp, lim):
    spec = wl.random_1d(rp, 601, lim=lim)
    dt = 0.3 / 601
    qg, cg = gpu_fixed_steps(spec, "fp64", dt, 5)
    qo, co = oracle_fixed_steps(orc, spec, dt, 5)
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    assert np.allclose(cg, co, rtol=1e-13, atol=0)


@pytest.mark.parametrize("bc", [("wall", "wall"), ("extrap", "wall"), ("inflow", "extrap")])
@pytest.mark.parametrize("rp", ["sw_roe", "euler_roe", "acoustics"])
def test_classic1d_boundaries_fp64(orc, rp, bc):
    spec = wl.random_1d(rp, 257, bc=bc)
    if "inflow" in bc:
        spec["inflow"] = list(spec["q0"][:, 0] * 1.05)
    dt = 0.3 / 257
    qg, _ = gpu_fixed_steps(spec, "fp64", dt, 6)
    qo, _ = oracle_fixed_steps(orc, spec, dt, 6)
    assert rel_maxnorm(qg, qo) <= FP64_TOL


@pytest.mark.parametrize("rp", RPS_1D)
def test_classic1d_order1_and_fp32(orc, rp):
    spec = wl.random_1d(rp, 1100, order=1)
    dt = 0.3 / 1100
    qg, _ = gpu_fixed_steps(spec, "fp64", dt, 4)
    qo, _ = oracle_fixed_steps(orc, spec, dt, 4)
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    spec = wl.random_1d(rp, 1100, jump=False)
    qg, _ = gpu_fixed_steps(spec, "fp32", dt, 4)
    qo, _ = oracle_fixed_steps(orc, spec, dt, 4)
    assert rel_maxnorm(qg, qo) <= FP32_SMOOTH_TOL


# --------------------------------------------------------------------------
# classic 2D, fixed dt, several tile shapes
# --------------------------------------------------------------------------
def _spec2d(rp, nx, ny, **kw):
    spec = wl.random_smooth_2d(rp, nx, ny, **kw)
    return spec


@pytest.mark.parametrize("rp", RPS_2D)
@pytest.mark.parametrize("order,transverse", [(2, 2), (2, 1), (2, 0), (1, 1)])
def test_classic2d_fixed_dt_fp64(orc, rp, order, transverse):
    spec = _spec2d(rp, 131, 70, order=order, transverse=transverse)
    dt = 0.25 / 131
    qo, co = oracle_fixed_steps(orc, spec, dt, 4)
    for tune in ((128, 32), (64, 8), (64, 128)):
        import torch
        from paper_1111_6583_gb300 import claw
        s = claw.Solver(spec, "fp64")
        s.tune(*tune)
        for _ in range(4):
            info = s.step(dt)
        s.sync()
        qg = s.q.cpu().numpy()
        s.close()
        assert rel_maxnorm(qg, qo) <= FP64_TOL, tune
        assert info["cfl"] == pytest.approx(co[-1], rel=1e-13)


@pytest.mark.parametrize("rp", ["acoustics", "advection"])
@pytest.mark.parametrize("lim", ["minmod", "superbee", "vanleer", "none"])
def test_classic2d_wave_strength_limiters(orc, rp, lim):
    """The constant-coefficient solvers limit by wave strengths (FP64: the
    division-free forms of phi(u/a) a); every limiter in 2D and in 3D, FP64
    against the oracle's dot-product form, FP32 against it too."""
    spec = _spec2d(rp, 131, 70, lim=lim)
    dt = 0.25 / 131
    qo, co = oracle_fixed_steps(orc, spec, dt, 4)
    qg, cg = gpu_fixed_steps(spec, "fp64", dt, 4)
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    assert np.allclose(cg, co, rtol=1e-13, atol=0)
    q32, _ = gpu_fixed_steps(spec, "fp32", dt, 4)
    assert rel_maxnorm(q32, qo) <= FP32_SMOOTH_TOL
    spec = wl.random_3d(rp, 30, 17, 13, bc="wall", lim=lim)
    dt = 0.2 / 30
    qo, _ = oracle_fixed_steps(orc, spec, dt, 3)
    qg, _ = gpu_fixed_steps(spec, "fp64", dt, 3)
    assert rel_maxnorm(qg, qo) <= FP64_TOL


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("rp,nx,ny", [("sw_roe", 131, 70), ("euler_roe", 250, 61),
                                       ("sw_roe", 372, 33), ("acoustics", 113, 57),
                                       ("advection", 85, 40)])
def test_classic2d_tile_shapes_bitwise(rp, nx, ny, prec):
    """Every tile shape gives the same bits, in both precisions (strips of 60
    and 124 columns): narrow last strips whose upper
    warps sit idle (131 and 250 columns), a last strip exactly full (372 =
    3 x 124), chunk heights that do not divide the rows (29, 13, 7), one
    chunk for all rows, and the autotuned shape."""
    from paper_1111_6583_gb300 import claw
    spec = _spec2d(rp, nx, ny, order=2, transverse=2)
    dt = 0.25 / nx
    out = []
    for tune in ((128, 32), (128, 29), (64, 13), (128, 7), (64, 128), None):
        s = claw.Solver(spec, prec)
        if tune is None:
            s.tune()
        else:
            s.tune(*tune)
        for _ in range(3):
            s.step(dt)
        s.sync()
        out.append(s.q.cpu().numpy())
        s.close()
    for k in range(1, len(out)):
        assert np.array_equal(out[k], out[0]), k


@pytest.mark.parametrize("rp", ["sw_roe", "euler_roe", "acoustics", "advection"])
@pytest.mark.parametrize("bc", ["wall", "extrap"])
def test_classic2d_boundaries_fp64(orc, rp, bc):
    spec = _spec2d(rp, 67, 45, bc=bc)
    spec["bc_lower"] = [bc, "wall"]
    spec["bc_upper"] = ["extrap", bc]
    dt = 0.25 / 67
    qo, _ = oracle_fixed_steps(orc, spec, dt, 5)
    qg, _ = gpu_fixed_steps(spec, "fp64", dt, 5)
    assert rel_maxnorm(qg, qo) <= FP64_TOL


def test_classic2d_inflow_fp64(orc):
    spec = wl.shock_bubble_2d(nx=96, ny=48, scheme="classic")
    dt = 0.2 / 96 / 3.0
    qo, _ = oracle_fixed_steps(orc, spec, dt, 6)
    qg, _ = gpu_fixed_steps(spec, "fp64", dt, 6)
    assert rel_maxnorm(qg, qo) <= FP64_TOL


@pytest.mark.parametrize("rp", RPS_2D)
def test_classic2d_fp32(orc, rp):
    spec = _spec2d(rp, 131, 70)
    dt = 0.25 / 131
    qo, _ = oracle_fixed_steps(orc, spec, dt, 4)
    qg, _ = gpu_fixed_steps(spec, "fp32", dt, 4)
    assert rel_maxnorm(qg, qo) <= FP32_SMOOTH_TOL


# --------------------------------------------------------------------------
# SharpClaw, fixed dt
# --------------------------------------------------------------------------
@pytest.mark.parametrize("rp", RPS_1D)
@pytest.mark.parametrize("char", [0, 1])
def test_sharpclaw1d_fp64(orc, rp, char):
    if rp == "elasticity_fwave" and char:
        pytest.skip("no characteristic projection for f-wave elasticity")
    spec = wl.random_1d(rp, 300, scheme="sharpclaw", char_decomp=char)
    dt = 0.15 / 300
    qo, co = oracle_fixed_steps(orc, spec, dt, 3)
    qg, cg = gpu_fixed_steps(spec, "fp64", dt, 3)
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    assert np.allclose(cg, co, rtol=1e-13, atol=0)


@pytest.mark.parametrize("rp", RPS_2D)
@pytest.mark.parametrize("char", [0, 1])
def test_sharpclaw2d_fp64(orc, rp, char):
    spec = _spec2d(rp, 70, 37, scheme="sharpclaw", char_decomp=char)
    dt = 0.1 / 70
    qo, _ = oracle_fixed_steps(orc, spec, dt, 3)
    qg, _ = gpu_fixed_steps(spec, "fp64", dt, 3)
    assert rel_maxnorm(qg, qo) <= FP64_TOL


@pytest.mark.parametrize("rp", ["sw_roe", "euler_roe"])
def test_sharpclaw2d_fp32(orc, rp):
    spec = _spec2d(rp, 70, 37, scheme="sharpclaw", char_decomp=1)
    dt = 0.1 / 70
    qo, _ = oracle_fixed_steps(orc, spec, dt, 3)
    qg, _ = gpu_fixed_steps(spec, "fp32", dt, 3)
    assert rel_maxnorm(qg, qo) <= FP32_SMOOTH_TOL


# --------------------------------------------------------------------------
# controller runs (accept / reject / final-time clip) and the paper workloads
# --------------------------------------------------------------------------
@pytest.mark.parametrize("use_graph", [True, False])
def test_config_acoustics_1d_full_run(orc, use_graph):
    """1D acoustics, 2000 cells, MC, CFL 0.9, t = 2 (about 4445 steps)."""
    spec = wl.acoustics_1d(n=2000)
    qo, io = oracle_evolve(orc, spec, 2.0)
    qg, ig = gpu_evolve(spec, "fp64", 2.0, use_graph=use_graph)
    assert ig["steps"] == io["steps"] and ig["t"] == io["t"] == 2.0
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    q32, i32 = gpu_evolve(spec, "fp32", 2.0)
    assert i32["t"] == 2.0 and rel_l1(q32, qo) <= FP32_SHOCK_L1_TOL


def test_config_dambreak_256_full_run(orc):
    """2D shallow-water dam break at the oracle size 256^2 to t = 1.5."""
    spec = wl.sw_dambreak_2d(n=256)
    qo, io = oracle_evolve(orc, spec, 1.5)
    qg, ig = gpu_evolve(spec, "fp64", 1.5)
    assert ig["steps"] == io["steps"] and ig["t"] == 1.5
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    q32, i32 = gpu_evolve(spec, "fp32", 1.5)
    assert rel_l1(q32, qo) <= FP32_SHOCK_L1_TOL


def test_reject_and_retry_parity(orc):
    spec = wl.random_1d("sw_roe", 400, dt_initial=0.02)
    qo, io = oracle_evolve(orc, spec, 0.2)
    qg, ig = gpu_evolve(spec, "fp64", 0.2)
    assert io["rejects"] >= 1 and ig["rejects"] == io["rejects"]
    assert ig["steps"] == io["steps"]
    assert rel_maxnorm(qg, qo) <= FP64_TOL


def test_nonphysical_status():
    spec = wl.sw_dambreak_2d(n=64)
    spec["q0"][0, 10, 10] = -1.0
    qg, ig = gpu_evolve(spec, "fp64", 0.5)
    assert ig["status"] == 6  # CLAW_ENONPHYSICAL


def test_cfl_failure_status_keeps_qn():
    """A first dt far above the stable one and no retries allowed: the run
    stops with CLAW_ECFL and the state is still Q^n (the rejected attempt
    wrote only a work buffer)."""
    spec = wl.random_smooth_2d("sw_roe", 96, 64, dt_initial=0.5, max_retries=0)
    qg, ig = gpu_evolve(spec, "fp64", 0.3)
    assert ig["status"] == 5  # CLAW_ECFL
    assert ig["steps"] == 0 and ig["t"] == 0.0
    assert np.array_equal(qg, spec["q0"])


def test_conserved_totals_drift():
    import torch
    from paper_1111_6583_gb300 import claw
    spec = wl.random_smooth_2d("euler_roe", 200, 130)
    for prec, tol in (("fp64", 1e-13), ("fp32", 1e-6)):
        s = claw.Solver(spec, prec)
        t0 = s.totals()
        s.evolve(0.2)
        t1 = s.totals()
        ref = np.abs(spec["q0"]).reshape(4, -1).sum(axis=1) / (200 * 130)
        assert (np.abs(t1 - t0) / ref).max() <= tol, prec
        s.close()


def test_totals_match_oracle(orc):
    from paper_1111_6583_gb300 import claw
    spec = wl.random_smooth_2d("sw_roe", 333, 77)
    s = claw.Solver(spec, "fp64")
    P = orc.make_problem(spec)
    assert np.allclose(s.totals(), orc.totals(P, spec["q0"]), rtol=1e-15, atol=1e-15)
    s.close()


def test_checkpoint_restore_bitwise():
    import torch
    from paper_1111_6583_gb300 import claw
    spec = wl.sw_dambreak_2d(n=128)
    a = claw.Solver(spec, "fp64")
    a.evolve(0.5)
    blob = a.checkpoint()
    a.evolve(1.0)
    qa = a.q.cpu().numpy().copy()
    b = claw.Solver(spec, "fp64")
    b.restore(blob)
    b.evolve(1.0)
    assert np.array_equal(b.q.cpu().numpy(), qa)
    a.close()
    b.close()


# --------------------------------------------------------------------------
# transonic rarefactions: the entropy fix acts at the sonic point
# --------------------------------------------------------------------------
def _sonic_sod_spec(n, order):
    """Toro's sonic-rarefaction Sod variant (x0 = 0.3, t = 0.2)."""
    g = 1.4
    x = (np.arange(n) + 0.5) / n
    left = x < 0.3
    rho = np.where(left, 1.0, 0.125)
    u = np.where(left, 0.75, 0.0)
    p = np.where(left, 1.0, 0.1)
    spec = wl._base(1, [n], [0.0], [1.0], "euler_roe", params=[g], order=order,
                    bc_lower=["extrap"], bc_upper=["extrap"])
    spec.update(q0=np.ascontiguousarray(np.stack([rho, rho * u, p / (g - 1) + 0.5 * rho * u * u])),
                aux=None)
    return spec


def _dambreak10_spec(n, order, ndim=1, axis=0):
    """Dam break h = 10 | 1 (transonic rarefaction) on [-5, 5]; in 2D the data
    vary along `axis` only, with walls across it and periodic along the other."""
    if ndim == 1:
        x = -5.0 + (np.arange(n) + 0.5) * 10.0 / n
        spec = wl._base(1, [n], [-5.0], [5.0], "sw_roe", params=[1.0], order=order,
                        bc_lower=["extrap"], bc_upper=["extrap"])
        spec.update(q0=np.ascontiguousarray(np.stack([np.where(x < 0, 10.0, 1.0), np.zeros(n)])),
                    aux=None)
        return spec
    m = 19
    shape = (m, n) if axis == 0 else (n, m)  # (ny, nx)
    nn = [n, m] if axis == 0 else [m, n]
    lo = [-5.0, 0.0] if axis == 0 else [0.0, -5.0]
    hi = [5.0, 1.0] if axis == 0 else [1.0, 5.0]
    bcl = ["extrap", "periodic"] if axis == 0 else ["periodic", "extrap"]
    x = -5.0 + (np.arange(n) + 0.5) * 10.0 / n
    h1 = np.where(x < 0, 10.0, 1.0)
    h = np.broadcast_to(h1[None, :] if axis == 0 else h1[:, None], shape)
    spec = wl._base(2, nn, lo, hi, "sw_roe", params=[1.0], order=order, bc_lower=bcl,
                    bc_upper=list(bcl))
    spec.update(q0=np.ascontiguousarray(np.stack([h, np.zeros(shape), np.zeros(shape)])), aux=None)
    return spec


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("case", ["sonic_sod", "dambreak10"])
def test_entropy_fix_transonic_full_run(orc, case, order):
    """Controller runs to t_end on data whose rarefaction crosses the sonic
    point, so the Harten-Hyman split acts in every step."""
    spec = _sonic_sod_spec(437, order) if case == "sonic_sod" else _dambreak10_spec(437, order)
    t_end = 0.2 if case == "sonic_sod" else 0.5
    qo, io = oracle_evolve(orc, spec, t_end)
    qg, ig = gpu_evolve(spec, "fp64", t_end)
    assert ig["steps"] == io["steps"] and ig["t"] == t_end
    assert rel_maxnorm(qg, qo) <= FP64_TOL
    q32, _ = gpu_evolve(spec, "fp32", t_end)
    assert rel_l1(q32, qo) <= FP32_SHOCK_L1_TOL


@pytest.mark.parametrize("axis", [0, 1])
def test_entropy_fix_transonic_2d_both_directions(orc, axis):
    spec = _dambreak10_spec(211, 2, ndim=2, axis=axis)
    qo, io = oracle_evolve(orc, spec, 0.5)
    qg, ig = gpu_evolve(spec, "fp64", 0.5)
    assert ig["steps"] == io["steps"] and ig["t"] == 0.5
    assert rel_maxnorm(qg, qo) <= FP64_TOL
