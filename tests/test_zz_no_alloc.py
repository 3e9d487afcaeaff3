"""The allocation-free SharpClaw step (claw_sharp_step_noalloc) against the
ordinary solver handle.

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
from tests.gpu_util import FP64_TOL, FP32_SMOOTH_TOL, rel_maxnorm

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


@pytest.mark.parametrize("prec,tol", [("fp64", FP64_TOL), ("fp32", FP32_SMOOTH_TOL)])
@pytest.mark.parametrize("case", ["euler2d", "sw1d"])
def test_noalloc_step_matches_solver_handle(case, prec, tol):
    if case == "euler2d":
        spec = wl.random_smooth_2d("euler_roe", 70, 37, scheme="sharpclaw", char_decomp=1)
        dt = 0.1 / 70
    else:
        spec = wl.random_1d("sw_roe", 300, scheme="sharpclaw", char_decomp=1)
        dt = 0.15 / 300
    qa, ca = _noalloc_two_steps(spec, prec, dt)
    qb, cb = _handle_two_steps(spec, prec, dt)
    assert rel_maxnorm(qa, qb) <= tol
    assert np.allclose(ca, cb, rtol=1e-6 if prec == "fp32" else 1e-13, atol=0)


def test_noalloc_rejects_grid_beyond_scratch():
    import torch
    from paper_1111_6583_gb300 import claw
    lib = claw.load()
    spec = wl.random_smooth_2d("euler_roe", 70, 37, scheme="sharpclaw", char_decomp=1)
    spec["n"] = [1024, 1024]  # two FP64 stage states need 64 MiB > 8 MiB
    m = claw.method_from_spec(spec, "fp64")
    g = claw.grid_from_spec(spec)
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    st = lib.claw_sharp_step_noalloc(ctypes.byref(m), ctypes.byref(g),
                                     ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                     None, 1e-3, None, None)
    assert st == claw.CLAW_EINVAL
    assert b"too large" in lib.claw_last_error(None)
