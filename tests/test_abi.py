"""The C-ABI library builds, loads and exports every entry point that
include/clawgpu.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "clawgpu.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(claw_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1111_6583_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("claw_solver_create", "claw_bind_state", "claw_step", "claw_evolve_to_time",
                 "claw_conserved_totals", "claw_checkpoint", "claw_restore", "claw_batch_create",
                 "claw_batch_evolve", "claw_server_create", "claw_server_submit",
                 "claw_server_poll", "claw_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header(lib_path):
    from paper_1111_6583_gb300 import claw
    assert set(declared_functions()) <= set(claw.exported_symbols())


def test_method_init_and_validation_without_gpu(lib_path):
    """Host-side validation runs without touching the GPU."""
    from paper_1111_6583_gb300 import claw
    lib = claw.load()
    m = claw.claw_method()
    assert lib.claw_method_init(ctypes.byref(m), claw.RP["sw_roe"], 2) == claw.CLAW_OK
    assert m.num_eqn == 3 and m.transverse == 2 and m.lim == claw.LIM["mc"]
    assert lib.claw_method_init(ctypes.byref(m), claw.RP["elasticity_fwave"], 3) == claw.CLAW_EINVAL
    # the 2D p-system defaults to SharpClaw (normal solves only)
    assert lib.claw_method_init(ctypes.byref(m), claw.RP["elasticity_fwave"], 2) == claw.CLAW_OK
    assert m.scheme == claw.SHARPCLAW and m.num_eqn == 3 and m.num_aux == 2
    assert lib.claw_method_init(ctypes.byref(m), 99, 1) == claw.CLAW_EINVAL
    g = claw.claw_grid()
    g.ndim = 2
    g.n[0] = 2  # too few cells
    g.n[1] = 64
    g.upper[0] = g.upper[1] = 1.0
    lib.claw_method_init(ctypes.byref(m), claw.RP["sw_roe"], 2)
    h = ctypes.c_void_p()
    assert lib.claw_solver_create(ctypes.byref(m), ctypes.byref(g), None,
                                  ctypes.byref(h)) == claw.CLAW_EINVAL
    assert b"too few cells" in lib.claw_last_error(None)
    g.n[0] = 64
    m.bc_lower[0] = claw.BC["periodic"]
    m.bc_upper[0] = claw.BC["wall"]
    assert lib.claw_solver_create(ctypes.byref(m), ctypes.byref(g), None,
                                  ctypes.byref(h)) == claw.CLAW_EINVAL
    assert b"paired" in lib.claw_last_error(None)
    lib.claw_method_init(ctypes.byref(m), claw.RP["elasticity_fwave"], 2)
    m.scheme = claw.CLASSIC
    m.bc_upper[0] = claw.BC["periodic"]
    assert lib.claw_solver_create(ctypes.byref(m), ctypes.byref(g), None,
                                  ctypes.byref(h)) == claw.CLAW_EINVAL
    assert b"SharpClaw" in lib.claw_last_error(None)
    lib.claw_method_init(ctypes.byref(m), claw.RP["elasticity_fwave"], 1)
    m.scheme = claw.SHARPCLAW
    m.char_decomp = 1
    g.ndim = 1
    assert lib.claw_solver_create(ctypes.byref(m), ctypes.byref(g), None,
                                  ctypes.byref(h)) == claw.CLAW_EINVAL
    # SharpClaw options: odd WENO orders 5..17, the two SSP integrators, and
    # a grid at least as wide as the WENO ghost layer
    lib.claw_method_init(ctypes.byref(m), claw.RP["euler_roe"], 1)
    m.scheme = claw.SHARPCLAW
    g.n[0] = 64
    for bad in (19, 6, 3):
        m.weno_order = bad
        assert lib.claw_solver_create(ctypes.byref(m), ctypes.byref(g), None,
                                      ctypes.byref(h)) == claw.CLAW_EINVAL
        assert b"weno_order" in lib.claw_last_error(None)
    m.weno_order = 9
    m.time_integrator = 2
    assert lib.claw_solver_create(ctypes.byref(m), ctypes.byref(g), None,
                                  ctypes.byref(h)) == claw.CLAW_EINVAL
    assert b"time integrator" in lib.claw_last_error(None)
    m.time_integrator = 1
    g.n[0] = 4
    assert lib.claw_solver_create(ctypes.byref(m), ctypes.byref(g), None,
                                  ctypes.byref(h)) == claw.CLAW_EINVAL
    assert b"too few cells" in lib.claw_last_error(None)
    # source splitting: Godunov by default, Strang on request, nothing else
    lib.claw_method_init(ctypes.byref(m), claw.RP["euler_tracer"], 2)
    assert m.source_split == claw.SOURCE_SPLIT["godunov"]
    m.source = claw.SOURCE["axisymmetric"]
    m.source_split = 3
    g.ndim = 2
    g.n[0] = g.n[1] = 64
    assert lib.claw_solver_create(ctypes.byref(m), ctypes.byref(g), None,
                                  ctypes.byref(h)) == claw.CLAW_EINVAL
    assert b"source_split" in lib.claw_last_error(None)
    assert lib.claw_version().startswith(b"clawgpu")


def test_server_entry_points_validate_without_gpu(lib_path):
    """The server's argument checks return before any CUDA call: the
    dimension of claw_server_create_nd, a method the dimension cannot take,
    and null handles for the schedule and completion calls."""
    from paper_1111_6583_gb300 import claw
    lib = claw.load()
    m = claw.claw_method()
    h = ctypes.c_void_p()
    lib.claw_method_init(ctypes.byref(m), claw.RP["acoustics"], 3)
    for nd in (0, 4):
        assert lib.claw_server_create_nd(ctypes.byref(m), nd, 1 << 20, 4, None,
                                         ctypes.byref(h)) == claw.CLAW_EINVAL
    assert lib.claw_server_create_nd(ctypes.byref(m), 3, 1 << 20, 0, None,
                                     ctypes.byref(h)) == claw.CLAW_EINVAL
    # SharpClaw has no 3D form
    m.scheme = claw.SHARPCLAW
    assert lib.claw_server_create_nd(ctypes.byref(m), 3, 1 << 20, 4, None,
                                     ctypes.byref(h)) == claw.CLAW_EINVAL
    assert b"3D" in lib.claw_last_error(None)
    assert lib.claw_server_schedule(None, claw.SCHED["srw"], 1) == claw.CLAW_EINVAL
    n = ctypes.c_int()
    buf = (ctypes.c_uint64 * 4)()
    assert lib.claw_server_take_done(None, buf, 4, ctypes.byref(n)) == claw.CLAW_EINVAL
