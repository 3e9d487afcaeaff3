"""The allocation-free SharpClaw step (claw_sharp_step_noalloc) against the
CPU oracle and against the ordinary solver handle.

Callers that cannot let the library allocate device memory (their memory is
owned by their own allocator or arena, or allocation is not allowed where they
call) use claw_sharp_step_noalloc: it keeps its stage states and control block
in a static device array.  This file runs last so that a failure here comes
after every other test has run; it must pass alone and after the others.
"""
import ctypes

import numpy as np
import pytest

from paper_1111_6583_gb300 import workloads as wl
from tests.gpu_util import (FP64_TOL, FP32_SHOCK_L1_TOL, FP32_SMOOTH_TOL, oracle_fixed_steps,
                            rel_l1, rel_maxnorm)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _noalloc_two_steps(spec, prec, dt):
    import torch
    from paper_1111_6583_gb300 import claw
    lib = claw.load()
    m = claw.method_from_spec(spec, prec)
    g = claw.grid_from_spec(spec)
    tdt = torch.float64 if prec == "fp64" else torch.float32
    q0 = torch.as_tensor(spec["q0"], dtype=tdt).cuda().contiguous()
    q1 = torch.empty_like(q0)
    q2 = torch.empty_like(q0)
    aux = (torch.as_tensor(spec["aux"], dtype=tdt).cuda().contiguous()
           if spec.get("aux") is not None else None)
    stream = torch.cuda.current_stream().cuda_stream
    cfl = ctypes.c_double(0.0)
    cfls = []
    for src, dst in ((q0, q1), (q1, q2)):
        st = lib.claw_sharp_step_noalloc(ctypes.byref(m), ctypes.byref(g),
                                         ctypes.c_void_p(src.data_ptr()),
                                         ctypes.c_void_p(dst.data_ptr()),
                                         ctypes.c_void_p(aux.data_ptr()) if aux is not None
                                         else None, float(dt), ctypes.c_void_p(stream),
                                         ctypes.byref(cfl))
        assert st == claw.CLAW_OK, lib.claw_last_error(None)
        cfls.append(cfl.value)
    torch.cuda.synchronize()
    return q2.double().cpu().numpy(), cfls


def _handle_two_steps(spec, prec, dt):
    import torch
    from paper_1111_6583_gb300 import claw
    s = claw.Solver(spec, prec)
    cfls = [s.step(dt)["cfl"], s.step(dt)["cfl"]]
    s.sync()
    torch.cuda.synchronize()
    q = s.q.double().cpu().numpy()
    s.close()
    return q, cfls


def _case(case):
    if case == "euler2d":
        spec = wl.random_smooth_2d("euler_roe", 70, 37, scheme="sharpclaw", char_decomp=1)
        dt = 0.1 / 70
    elif case == "sw1d":
        spec = wl.random_1d("sw_roe", 300, scheme="sharpclaw", char_decomp=1)
        dt = 0.15 / 300
    else:  # f-wave elasticity in a layered medium: the aux fields are read
        spec = wl.random_1d("elasticity_fwave", 300, scheme="sharpclaw", char_decomp=0)
        dt = 0.15 / 300
    return spec, dt


@pytest.mark.parametrize("prec,tol", [("fp64", FP64_TOL), ("fp32", FP32_SMOOTH_TOL)])
@pytest.mark.parametrize("case", ["euler2d", "sw1d", "elasticity1d"])
def test_noalloc_step_matches_oracle_and_solver_handle(orc, case, prec, tol):
    spec, dt = _case(case)
    qa, ca = _noalloc_two_steps(spec, prec, dt)
    qo, co = oracle_fixed_steps(orc, spec, dt, 2)
    if prec == "fp64" or case == "euler2d":
        assert rel_maxnorm(qa, qo) <= tol
    else:  # the 1D cases carry a jump: the FP32 bound for shocked data
        assert rel_l1(qa, qo) <= FP32_SHOCK_L1_TOL
    assert np.allclose(ca, co, rtol=1e-5 if prec == "fp32" else 1e-13, atol=0)
    qb, cb = _handle_two_steps(spec, prec, dt)
    assert rel_maxnorm(qa, qb) <= tol
    assert np.allclose(ca, cb, rtol=1e-6 if prec == "fp32" else 1e-13, atol=0)


def _call(lib, m, g, q_in, q_out, aux=None, dt=1e-3):
    return lib.claw_sharp_step_noalloc(ctypes.byref(m), ctypes.byref(g), q_in, q_out, aux,
                                       float(dt), None, None)


def test_noalloc_rejects_bad_methods_before_any_launch():
    """Methods the step cannot take return CLAW_EINVAL from the host-side checks
    (the pointers below are never dereferenced)."""
    import torch
    from paper_1111_6583_gb300 import claw
    lib = claw.load()
    x = torch.zeros(4096, dtype=torch.float64, device="cuda")
    y = torch.zeros(4096, dtype=torch.float64, device="cuda")
    px, py = ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr())
    spec, _ = _case("elasticity1d")
    spec["n"] = [300]
    g = claw.grid_from_spec(spec)
    # the f-wave solver reads two aux fields: a missing aux pointer is refused
    m = claw.method_from_spec(spec, "fp64")
    assert _call(lib, m, g, px, py, None) == claw.CLAW_EINVAL
    # and so is a num_aux that does not match the solver
    m = claw.method_from_spec(spec, "fp64")
    m.num_aux = 0
    assert _call(lib, m, g, px, py, None) == claw.CLAW_EINVAL
    # SSP(10,4) is not taken by this step (it would need more stage states)
    spec2, _ = _case("sw1d")
    g2 = claw.grid_from_spec(spec2)
    m = claw.method_from_spec(spec2, "fp64")
    m.time_integrator = 1
    assert _call(lib, m, g2, px, py) == claw.CLAW_EINVAL
    assert b"SSP-RK3" in lib.claw_last_error(None)
    # an unknown limiter or precision is refused by the handle API's checks
    m = claw.method_from_spec(spec2, "fp64")
    m.prec = 7
    assert _call(lib, m, g2, px, py) == claw.CLAW_EINVAL
    # extents beyond int range are refused, not truncated
    m = claw.method_from_spec(spec2, "fp64")
    g3 = claw.grid_from_spec(spec2)
    g3.n[0] = 2 ** 32 + 16
    assert _call(lib, m, g3, px, py) == claw.CLAW_EINVAL
    # in place is refused
    assert _call(lib, m, g2, px, px) == claw.CLAW_EINVAL


def test_noalloc_rejects_grid_beyond_scratch():
    import torch
    from paper_1111_6583_gb300 import claw
    lib = claw.load()
    spec = wl.random_smooth_2d("euler_roe", 70, 37, scheme="sharpclaw", char_decomp=1)
    spec["n"] = [1024, 1024]  # two FP64 stage states need 64 MiB > 8 MiB
    m = claw.method_from_spec(spec, "fp64")
    g = claw.grid_from_spec(spec)
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    y = torch.zeros(16, dtype=torch.float64, device="cuda")
    st = lib.claw_sharp_step_noalloc(ctypes.byref(m), ctypes.byref(g),
                                     ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                     None, 1e-3, None, None)
    assert st == claw.CLAW_EINVAL
    assert b"too large" in lib.claw_last_error(None)
