"""Plain FP64 CPU oracle for the finite-volume step of Clawpack-classic and
SharpClaw (PyClaw, Ketcheson et al.).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the CUDA library: the C source ``oracle.c`` is an independent restatement of
the method (Sec. 2, Eq. (fluxdiff) and Eq. (lwflux); Sec. 2.1 on transverse
solvers and SharpClaw; Sec. 4 on ghost cells and the CFL check).

Every function here marshals numpy arrays into the C oracle; no arithmetic of
the method is done in Python.

Parity status: every function is pinned by ``tests/test_oracle_pins.py``
(closed forms, conservation, exact Riemann solutions, convergence orders);
the paper prints no worked example, so no pin uses a printed value.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess

import numpy as np

from .weno_coeffs import weno_tables

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")

RP = {"advection": 0, "acoustics": 1, "sw_roe": 2, "euler_roe": 3, "euler_hlle": 4,
      "elasticity_fwave": 5, "euler_tracer": 6, "acoustics_vc": 7}
LIM = {"none": 0, "minmod": 1, "superbee": 2, "vanleer": 3, "mc": 4}
BC = {"periodic": 0, "wall": 1, "extrap": 2, "inflow": 3}
SCHEME = {"classic": 0, "sharpclaw": 1}
STATUS = {0: "ok", 1: "einval", 5: "ecfl", 6: "enonphysical"}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, no FMA contraction, OpenMP)."""
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Prob(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double),
        ("rp", ctypes.c_int), ("scheme", ctypes.c_int), ("lim", ctypes.c_int),
        ("order", ctypes.c_int), ("transverse", ctypes.c_int), ("char_decomp", ctypes.c_int),
        ("entropy_fix", ctypes.c_int),
        ("num_eqn", ctypes.c_int), ("num_aux", ctypes.c_int), ("num_waves", ctypes.c_int),
        ("bc_lo", ctypes.c_int * 3), ("bc_hi", ctypes.c_int * 3),
        ("inflow", ctypes.c_double * 8), ("params", ctypes.c_double * 8),
        ("cfl_desired", ctypes.c_double), ("cfl_max", ctypes.c_double),
        ("dt_initial", ctypes.c_double), ("dt_max", ctypes.c_double),
        ("max_retries", ctypes.c_int), ("weno_eps", ctypes.c_double),
        ("nz", ctypes.c_int), ("dz", ctypes.c_double),
        ("time_integrator", ctypes.c_int),
        ("weno_r", ctypes.c_int),
        ("weno_c", ctypes.c_double * 81),
        ("weno_d", ctypes.c_double * 9),
        ("weno_b", ctypes.c_double * 729),
        ("source", ctypes.c_int),
        ("dim_split", ctypes.c_int),
        ("lower", ctypes.c_double * 2),
        ("capa_index", ctypes.c_int),
        ("source_split", ctypes.c_int),
    ]


class _RunInfo(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("dt_next", ctypes.c_double),
                ("cfl_last", ctypes.c_double), ("cfl_max_seen", ctypes.c_double),
                ("steps", ctypes.c_int), ("rejects", ctypes.c_int), ("status", ctypes.c_int)]


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _bind(ctypes.CDLL(_SO))
    return _lib


def build_variant(source_text: str, path: str) -> str:
    """Compile a modified copy of oracle.c into the shared library ``path``
    (same flags as build()).  Tests use it to plant a mistake in the oracle
    and check that the pins catch it; the oracle itself is never changed."""
    src = path + ".c"
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
                    "-shared", "-std=c11", "-I" + _HERE, src, "-o", path, "-lm"], check=True)
    return path


@contextlib.contextmanager
def variant(path: str):
    """Run the functions of this module on the library ``path`` (a variant from
    build_variant) inside the with-block."""
    global _lib
    saved = _load()
    _lib = _bind(ctypes.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


def _bind(lib):
    P = ctypes.POINTER(_Prob)
    lib.orc_num_eqn.restype = ctypes.c_int
    lib.orc_num_waves.restype = ctypes.c_int
    lib.orc_riemann.argtypes = [P, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    lib.orc_transverse.argtypes = [P, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    lib.orc_phi.restype = ctypes.c_double
    lib.orc_phi.argtypes = [ctypes.c_int, ctypes.c_double]
    lib.orc_weno5.restype = ctypes.c_double
    lib.orc_weno5.argtypes = [_dp, ctypes.c_double]
    lib.orc_weno_r.restype = ctypes.c_double
    lib.orc_weno_r.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp, ctypes.c_double]
    lib.orc_char_matrices.argtypes = [P, ctypes.c_int, _dp, _dp, _dp, _dp]
    lib.orc_fill_ghost.argtypes = [P, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
    lib.orc_classic_step.argtypes = [P, _dp, _dp, ctypes.c_double, _dp]
    lib.orc_sharp_L.argtypes = [P, _dp, _dp, _dp, _dp]
    lib.orc_sharp_step.argtypes = [P, _dp, _dp, ctypes.c_double, _dp]
    lib.orc_ssp_rk3_linear.restype = ctypes.c_double
    lib.orc_ssp_rk3_linear.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
    lib.orc_ssp104_linear.restype = ctypes.c_double
    lib.orc_ssp104_linear.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
    lib.orc_max_speeds.argtypes = [P, _dp, _dp, _dp]
    lib.orc_transverse_vc.restype = None
    lib.orc_transverse_vc.argtypes = [P, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
    lib.orc_source_step.restype = None
    lib.orc_source_step.argtypes = [P, _dp, ctypes.c_double]
    lib.orc_evolve.argtypes = [P, _dp, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                               ctypes.POINTER(_RunInfo)]
    lib.orc_totals.argtypes = [P, _dp, _dp]
    lib.orc_threads.restype = ctypes.c_int
    return lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def num_eqn(rp: str, ndim: int) -> int:
    return _load().orc_num_eqn(RP[rp], ndim)


def num_waves(rp: str, ndim: int) -> int:
    return _load().orc_num_waves(RP[rp], ndim)


def threads() -> int:
    return _load().orc_threads()


def make_problem(spec: dict):
    """Build the C problem record from a workload spec dict (see the package's
    workloads module for the keys)."""
    lib = _load()
    p = _Prob()
    ndim = int(spec["ndim"])
    n = list(spec["n"]) + [1, 1]
    lo = list(spec["lower"]) + [0.0, 0.0]
    hi = list(spec["upper"]) + [1.0, 1.0]
    p.ndim = ndim
    p.nx, p.ny = int(n[0]), (int(n[1]) if ndim >= 2 else 1)
    p.nz = int(n[2]) if ndim == 3 else 1
    p.dx = (hi[0] - lo[0]) / n[0]
    p.dy = (hi[1] - lo[1]) / n[1] if ndim >= 2 else 1.0
    p.dz = (hi[2] - lo[2]) / n[2] if ndim == 3 else 1.0
    p.rp = RP[spec["rp"]]
    p.scheme = SCHEME[spec.get("scheme", "classic")]
    p.lim = LIM[spec.get("lim", "mc")]
    p.order = int(spec.get("order", 2))
    p.transverse = int(spec.get("transverse", 2)) if ndim >= 2 else 0
    p.char_decomp = int(spec.get("char_decomp", 0))
    p.entropy_fix = int(spec.get("entropy_fix", 1))
    p.num_eqn = lib.orc_num_eqn(p.rp, ndim)
    p.num_aux = int(spec.get("num_aux", 2 if spec["rp"] in ("elasticity_fwave", "acoustics_vc")
                                 else 0))
    p.num_waves = lib.orc_num_waves(p.rp, ndim)
    bl = list(spec.get("bc_lower", ["periodic"] * ndim)) + ["periodic"] * 2
    bh = list(spec.get("bc_upper", ["periodic"] * ndim)) + ["periodic"] * 2
    for d in range(3):
        p.bc_lo[d] = BC[bl[d]]
        p.bc_hi[d] = BC[bh[d]]
    inflow = list(spec.get("inflow", [])) + [0.0] * 8
    params = list(spec.get("params", [])) + [0.0] * 8
    for k in range(8):
        p.inflow[k] = float(inflow[k])
        p.params[k] = float(params[k])
    p.cfl_desired = float(spec.get("cfl_desired", 0.9))
    p.cfl_max = float(spec.get("cfl_max", 1.0))
    p.dt_initial = float(spec.get("dt_initial", 0.0))
    p.dt_max = float(spec.get("dt_max", 1e30))
    p.max_retries = int(spec.get("max_retries", 8))
    p.weno_eps = float(spec.get("weno_eps", 1e-6))
    p.time_integrator = {"ssp_rk3": 0, "ssp104": 1}[spec.get("time_integrator", "ssp_rk3")]
    order = int(spec.get("weno_order", 5))
    if order % 2 == 0 or not 5 <= order <= 17:
        raise ValueError("weno_order must be odd, 5..17")
    p.weno_r = (order + 1) // 2
    if p.weno_r > 3:
        cf, df, bf = weno_tables(p.weno_r)
        p.weno_c[:len(cf)] = cf
        p.weno_d[:len(df)] = df
        p.weno_b[:len(bf)] = bf
    p.source = {"none": 0, "axisymmetric": 1}[spec.get("source", "none")]
    p.dim_split = int(spec.get("dim_split", 0))
    p.lower[0] = float(lo[0])
    p.lower[1] = float(lo[1])
    p.capa_index = int(spec.get("capa_index", -1))
    p.source_split = {"godunov": 1, "strang": 2}[spec.get("source_split", "godunov")]
    return p


def _shape(p):
    if p.ndim == 3:
        return (p.num_eqn, p.nz, p.ny, p.nx)
    return (p.num_eqn, p.ny, p.nx) if p.ndim == 2 else (p.num_eqn, p.nx)


def _arr(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def riemann(p, direction, ql, qr, auxl=None, auxr=None):
    """One Riemann solve: returns (waves[nw, m], speeds[nw], amdq[m], apdq[m])."""
    m, nw = p.num_eqn, p.num_waves
    ql, qr = _arr(ql), _arr(qr)
    al = _arr(auxl if auxl is not None else np.zeros(8))
    ar = _arr(auxr if auxr is not None else np.zeros(8))
    W = np.zeros((nw, m)); s = np.zeros(nw); am = np.zeros(m); ap = np.zeros(m)
    _load().orc_riemann(ctypes.byref(p), direction, _ptr(ql), _ptr(qr), _ptr(al), _ptr(ar),
                        _ptr(W), _ptr(s), _ptr(am), _ptr(ap))
    return W, s, am, ap


def transverse(p, direction, ql, qr, asdq, auxl=None, auxr=None):
    """Transverse split of asdq: returns (bmasdq, bpasdq)."""
    m = p.num_eqn
    ql, qr, asdq = _arr(ql), _arr(qr), _arr(asdq)
    al = _arr(auxl if auxl is not None else np.zeros(8))
    ar = _arr(auxr if auxr is not None else np.zeros(8))
    bm = np.zeros(m); bp = np.zeros(m)
    _load().orc_transverse(ctypes.byref(p), direction, _ptr(ql), _ptr(qr), _ptr(al), _ptr(ar),
                           _ptr(asdq), _ptr(bm), _ptr(bp))
    return bm, bp


def transverse_vc(p, direction, a_m, a_c, a_p, asdq):
    """Varying-medium acoustics transverse split: (bm, bp)."""
    m = p.num_eqn
    bm, bp = np.zeros(m), np.zeros(m)
    _load().orc_transverse_vc(ctypes.byref(p), direction, _ptr(_arr(a_m)), _ptr(_arr(a_c)),
                              _ptr(_arr(a_p)), _ptr(_arr(asdq)), _ptr(bm), _ptr(bp))
    return bm, bp


def phi(lim: str, theta: float) -> float:
    return _load().orc_phi(LIM[lim], float(theta))


def weno_r(r, v, eps=1e-6) -> float:
    """WENO of order 2r-1: left-biased value at the right edge of the centre
    cell of v[0..2r-2], coefficients from oracle.weno_coeffs."""
    cf, df, bf = weno_tables(r)
    v = np.ascontiguousarray(v, dtype=np.float64)
    assert v.shape == (2 * r - 1,)
    c = np.array(cf)
    d = np.array(df)
    b = np.array(bf)
    return _load().orc_weno_r(int(r), _ptr(c), _ptr(d), _ptr(b), _ptr(v), float(eps))


def weno5(v, eps=1e-6) -> float:
    v = _arr(v)
    return _load().orc_weno5(_ptr(v), float(eps))


def char_matrices(p, direction, ql, qr):
    m = p.num_eqn
    L = np.zeros((m, m)); R = np.zeros((m, m))
    st = _load().orc_char_matrices(ctypes.byref(p), direction, _ptr(_arr(ql)), _ptr(_arr(qr)),
                                   _ptr(L), _ptr(R))
    if st != 0:
        raise ValueError("no characteristic decomposition for this solver")
    return L, R


def fill_ghost(p, q, g, is_aux=False):
    q = _arr(q)
    nc = q.shape[0]
    if p.ndim == 2:
        out = np.zeros((nc, p.ny + 2 * g, p.nx + 2 * g))
    else:
        out = np.zeros((nc, p.nx + 2 * g))
    _load().orc_fill_ghost(ctypes.byref(p), _ptr(q), nc, g, int(is_aux), _ptr(out))
    return out


def step(p, q, aux=None, dt=None):
    """One step (classic or SharpClaw by p.scheme) with the given dt; returns (q_new, cfl)."""
    q = _arr(q, _shape(p)).copy()
    aux = _arr(aux) if aux is not None else None
    cfl = ctypes.c_double(0.0)
    fn = _load().orc_sharp_step if p.scheme == 1 else _load().orc_classic_step
    st = fn(ctypes.byref(p), _ptr(q), _ptr(aux), float(dt), ctypes.byref(cfl))
    if st != 0:
        raise ValueError("oracle step failed: %s" % STATUS.get(st, st))
    return q, cfl.value


def sharp_L(p, q, aux=None):
    q = _arr(q, _shape(p))
    L = np.zeros_like(q)
    smax = np.zeros(2)
    st = _load().orc_sharp_L(ctypes.byref(p), _ptr(q), _ptr(_arr(aux) if aux is not None else None),
                             _ptr(L), _ptr(smax))
    if st != 0:
        raise ValueError("oracle L failed: %s" % STATUS.get(st, st))
    return L, smax


def source_step(p, q, dt):
    """One source step (the problem's source term over dt), returns a copy."""
    q = _arr(q, _shape(p)).copy()
    _load().orc_source_step(ctypes.byref(p), _ptr(q), float(dt))
    return q


def ssp_rk3_linear(lam, dt, q0) -> float:
    return _load().orc_ssp_rk3_linear(float(lam), float(dt), float(q0))


def ssp104_linear(lam, dt, q0) -> float:
    return _load().orc_ssp104_linear(float(lam), float(dt), float(q0))


def max_speeds(p, q, aux=None):
    smax = np.zeros(3)
    _load().orc_max_speeds(ctypes.byref(p), _ptr(_arr(q, _shape(p))),
                           _ptr(_arr(aux) if aux is not None else None), _ptr(smax))
    return smax


def evolve(p, q, aux=None, t0=0.0, t_end=1.0, max_steps=10 ** 9):
    """Evolve with the CFL controller; returns (q, info dict)."""
    q = _arr(q, _shape(p)).copy()
    info = _RunInfo()
    _load().orc_evolve(ctypes.byref(p), _ptr(q), _ptr(_arr(aux) if aux is not None else None),
                       float(t0), float(t_end), int(max_steps), ctypes.byref(info))
    return q, {"t": info.t, "dt_next": info.dt_next, "cfl_last": info.cfl_last,
               "cfl_max_seen": info.cfl_max_seen, "steps": info.steps,
               "rejects": info.rejects, "status": STATUS.get(info.status, info.status)}


def totals(p, q):
    out = np.zeros(p.num_eqn)
    _load().orc_totals(ctypes.byref(p), _ptr(_arr(q, _shape(p))), _ptr(out))
    return out
