"""Thin ctypes binding of libclawgpu (include/clawgpu.h).

Functions named ``claw_*`` mirror the C ABI one to one (argument marshalling
only).  ``Solver``, ``Batch`` and ``Server`` are small conveniences that take
torch tensors for device memory and the current torch stream; every numerical
step still runs in the library's CUDA kernels.  There is no CPU fallback:
importing this module on a machine without the built library raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libclawgpu.so")

CLAW_OK, CLAW_EINVAL, CLAW_ENOMEM, CLAW_EBUDGET, CLAW_ECUDA = 0, 1, 2, 3, 4
CLAW_ECFL, CLAW_ENONPHYSICAL, CLAW_ETIMEOUT, CLAW_EBUSY = 5, 6, 7, 8
STATUS_NAMES = {0: "ok", 1: "einval", 2: "enomem", 3: "ebudget", 4: "ecuda", 5: "ecfl",
                6: "enonphysical", 7: "etimeout", 8: "ebusy"}
FP64, FP32 = 0, 1
CLASSIC, SHARPCLAW = 0, 1
RP = {"advection": 0, "acoustics": 1, "sw_roe": 2, "euler_roe": 3, "euler_hlle": 4,
      "elasticity_fwave": 5, "euler_tracer": 6, "acoustics_vc": 7}
SOURCE = {"none": 0, "axisymmetric": 1}
SOURCE_SPLIT = {"godunov": 1, "strang": 2}
SCHED = {"all": 0, "srw": 1}
LIM = {"none": 0, "minmod": 1, "superbee": 2, "vanleer": 3, "mc": 4}
BC = {"periodic": 0, "wall": 1, "extrap": 2, "inflow": 3}
TIME_INTEGRATOR = {"ssp_rk3": 0, "ssp104": 1}


class ClawError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class claw_grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int64 * 3),
                ("lower", ctypes.c_double * 3), ("upper", ctypes.c_double * 3)]


class claw_method(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int), ("rp", ctypes.c_int), ("lim", ctypes.c_int),
                ("prec", ctypes.c_int), ("order", ctypes.c_int), ("transverse", ctypes.c_int),
                ("weno_order", ctypes.c_int), ("char_decomp", ctypes.c_int),
                ("entropy_fix", ctypes.c_int), ("max_retries", ctypes.c_int),
                ("cfl_desired", ctypes.c_double), ("cfl_max", ctypes.c_double),
                ("dt_initial", ctypes.c_double), ("dt_max", ctypes.c_double),
                ("weno_eps", ctypes.c_double), ("bc_lower", ctypes.c_int * 3),
                ("bc_upper", ctypes.c_int * 3), ("inflow", ctypes.c_double * 8),
                ("params", ctypes.c_double * 8), ("num_eqn", ctypes.c_int),
                ("num_aux", ctypes.c_int), ("time_integrator", ctypes.c_int),
                ("source", ctypes.c_int), ("dim_split", ctypes.c_int),
                ("capa_index", ctypes.c_int), ("source_split", ctypes.c_int)]


class claw_step_info(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("dt_used", ctypes.c_double),
                ("dt_next", ctypes.c_double), ("cfl", ctypes.c_double),
                ("cfl_max_seen", ctypes.c_double), ("steps", ctypes.c_int64),
                ("rejects", ctypes.c_int64), ("accepted", ctypes.c_int), ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class claw_req_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("steps", ctypes.c_int64), ("t", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double)]


_VP = ctypes.c_void_p
_P = ctypes.POINTER
_SIGS = {
    "claw_method_init": (ctypes.c_int, [_P(claw_method), ctypes.c_int, ctypes.c_int]),
    "claw_solver_create": (ctypes.c_int, [_P(claw_method), _P(claw_grid), _VP, _P(_VP)]),
    "claw_bind_state": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_double]),
    "claw_solver_tune": (ctypes.c_int, [_VP, ctypes.c_int, _P(ctypes.c_int), _P(ctypes.c_int)]),
    "claw_step": (ctypes.c_int, [_VP, ctypes.c_double, _P(claw_step_info)]),
    "claw_advance": (ctypes.c_int, [_VP, ctypes.c_int]),
    "claw_set_t_end": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_int64]),
    "claw_evolve_to_time": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_int64, ctypes.c_int,
                                           _P(claw_step_info)]),
    "claw_get_info": (ctypes.c_int, [_VP, _P(claw_step_info)]),
    "claw_current_state": (ctypes.c_int, [_VP, _P(_VP)]),
    "claw_sync_state": (ctypes.c_int, [_VP]),
    "claw_conserved_totals": (ctypes.c_int, [_VP, _P(ctypes.c_double)]),
    "claw_checkpoint": (ctypes.c_int, [_VP, _VP, _P(ctypes.c_size_t)]),
    "claw_restore": (ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    "claw_step_host": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int]),
    "claw_solver_destroy": (ctypes.c_int, [_VP]),
    "claw_batch_create": (ctypes.c_int, [_P(claw_method), _P(claw_grid), ctypes.c_int, _VP,
                                         _P(_VP)]),
    "claw_batch_bind": (ctypes.c_int, [_VP, _P(_VP), _P(_VP), _P(ctypes.c_double)]),
    "claw_batch_evolve": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int64, _P(claw_step_info)]),
    "claw_batch_advance": (ctypes.c_int, [_VP, ctypes.c_int]),
    "claw_batch_info": (ctypes.c_int, [_VP, _P(claw_step_info)]),
    "claw_batch_sync_state": (ctypes.c_int, [_VP]),
    "claw_batch_destroy": (ctypes.c_int, [_VP]),
    "claw_server_create": (ctypes.c_int, [_P(claw_method), ctypes.c_size_t, ctypes.c_int, _VP,
                                          _P(_VP)]),
    "claw_server_submit": (ctypes.c_int, [_VP, _P(claw_grid), _VP, _VP, ctypes.c_double,
                                          _P(ctypes.c_uint64)]),
    "claw_server_pump": (ctypes.c_int, [_VP, ctypes.c_int, _P(ctypes.c_int), _P(ctypes.c_int)]),
    "claw_server_poll": (ctypes.c_int, [_VP, ctypes.c_uint64, _VP, _P(claw_req_info)]),
    "claw_server_create_nd": (ctypes.c_int, [_P(claw_method), ctypes.c_int, ctypes.c_size_t,
                                             ctypes.c_int, _VP, _P(_VP)]),
    "claw_server_schedule": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int64]),
    "claw_server_take_done": (ctypes.c_int, [_VP, _P(ctypes.c_uint64), ctypes.c_int,
                                             _P(ctypes.c_int)]),
    "claw_server_destroy": (ctypes.c_int, [_VP]),
    "claw_sharp_step_noalloc": (ctypes.c_int, [_P(claw_method), _P(claw_grid), _VP, _VP, _VP,
                                               ctypes.c_double, _VP, _P(ctypes.c_double)]),
    "claw_fma_peak": (ctypes.c_int, [ctypes.c_int, _VP, _P(ctypes.c_double),
                                     _P(ctypes.c_double)]),
    "claw_async_wait_probe": (ctypes.c_int, [ctypes.c_int, _VP, _P(ctypes.c_int),
                                             _P(ctypes.c_int), _P(ctypes.c_double)]),
    "claw_batch_tune": (ctypes.c_int, [_VP, ctypes.c_int, _P(ctypes.c_int), _P(ctypes.c_int)]),
    "claw_server_tune": (ctypes.c_int, [_VP, ctypes.c_int, _P(ctypes.c_int), _P(ctypes.c_int)]),
    "claw_clock": (ctypes.c_double, []),
    "claw_last_error": (ctypes.c_char_p, [_VP]),
    "claw_version": (ctypes.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libclawgpu.so (built by paper_1111_6583_gb300.build); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("libclawgpu.so is not built (run __graft_entry__.build()); "
                               "there is no CPU fallback")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(st, handle=None):
    if st != CLAW_OK:
        raise ClawError(st, load().claw_last_error(handle).decode())
    return st


# ---- one-to-one wrappers (same names as the C ABI) ------------------------
def _mk(name):
    def f(*args):
        return getattr(load(), name)(*args)
    f.__name__ = name
    f.__doc__ = "C ABI call %s (see include/clawgpu.h)." % name
    return f


for _name in _SIGS:
    globals()[_name] = _mk(_name)


# ---- conveniences -----------------------------------------------------------
def _torch():
    import torch
    return torch


def current_stream_handle():
    torch = _torch()
    return torch.cuda.current_stream().cuda_stream


def grid_from_spec(spec) -> claw_grid:
    g = claw_grid()
    g.ndim = int(spec["ndim"])
    n = list(spec["n"]) + [1, 1]
    lo = list(spec["lower"]) + [0.0, 0.0]
    hi = list(spec["upper"]) + [1.0, 1.0]
    for d in range(3):
        g.n[d] = int(n[d]) if d < g.ndim else 1
        g.lower[d] = float(lo[d])
        g.upper[d] = float(hi[d])
    return g


def method_from_spec(spec, prec="fp64") -> claw_method:
    m = claw_method()
    ndim = int(spec["ndim"])
    _check(load().claw_method_init(ctypes.byref(m), RP[spec["rp"]], ndim))
    m.scheme = SHARPCLAW if spec.get("scheme", "classic") == "sharpclaw" else CLASSIC
    m.lim = LIM[spec.get("lim", "mc")]
    m.prec = FP32 if prec in ("fp32", FP32) else FP64
    m.order = int(spec.get("order", 2))
    m.transverse = int(spec.get("transverse", 2)) if ndim >= 2 else 0
    m.char_decomp = int(spec.get("char_decomp", 0))
    m.entropy_fix = int(spec.get("entropy_fix", 1))
    m.max_retries = int(spec.get("max_retries", 8))
    m.cfl_desired = float(spec.get("cfl_desired", 0.9))
    m.cfl_max = float(spec.get("cfl_max", 1.0))
    m.dt_initial = float(spec.get("dt_initial", 0.0))
    m.dt_max = float(spec.get("dt_max", 1e30))
    m.weno_eps = float(spec.get("weno_eps", 1e-6))
    m.weno_order = int(spec.get("weno_order", 5))
    m.time_integrator = TIME_INTEGRATOR[spec.get("time_integrator", "ssp_rk3")]
    m.source = SOURCE[spec.get("source", "none")]
    m.dim_split = int(spec.get("dim_split", 0))
    m.capa_index = int(spec.get("capa_index", -1))
    m.source_split = SOURCE_SPLIT[spec.get("source_split", "godunov")]
    m.num_aux = int(spec.get("num_aux", m.num_aux))
    bl = list(spec.get("bc_lower", ["periodic"] * ndim)) + ["periodic"] * 2
    bh = list(spec.get("bc_upper", ["periodic"] * ndim)) + ["periodic"] * 2
    for d in range(3):
        m.bc_lower[d] = BC[bl[d]]
        m.bc_upper[d] = BC[bh[d]]
    inflow = list(spec.get("inflow", [])) + [0.0] * 8
    params = list(spec.get("params", [])) + [0.0] * 8
    for k in range(8):
        m.inflow[k] = float(inflow[k])
        m.params[k] = float(params[k])
    return m


def _dtype(prec):
    torch = _torch()
    return torch.float32 if prec in ("fp32", FP32) else torch.float64


class Solver:
    """One grid: owns nothing but the handle; q (and aux) are torch tensors."""

    def __init__(self, spec, prec="fp64", q=None, aux=None, t0=0.0, stream=None):
        torch = _torch()
        self.spec = spec
        self.prec = prec
        self.method = method_from_spec(spec, prec)
        self.grid = grid_from_spec(spec)
        dt = _dtype(prec)
        self.q = q if q is not None else torch.as_tensor(spec["q0"], dtype=dt).cuda().contiguous()
        aux_src = aux if aux is not None else spec.get("aux")
        self.aux = (torch.as_tensor(aux_src, dtype=dt).cuda().contiguous()
                    if aux_src is not None else None)
        self.stream = stream if stream is not None else current_stream_handle()
        h = ctypes.c_void_p()
        _check(load().claw_solver_create(ctypes.byref(self.method), ctypes.byref(self.grid),
                                         ctypes.c_void_p(self.stream), ctypes.byref(h)))
        self.h = h
        _check(load().claw_bind_state(self.h, ctypes.c_void_p(self.q.data_ptr()),
                                      ctypes.c_void_p(self.aux.data_ptr()) if self.aux is not None
                                      else None, float(t0)), self.h)

    def tune(self, bw=None, h=None):
        b, hh = ctypes.c_int(bw or 0), ctypes.c_int(h or 0)
        _check(load().claw_solver_tune(self.h, 0 if bw is None else 1, ctypes.byref(b),
                                       ctypes.byref(hh)), self.h)
        return b.value, hh.value

    def step(self, dt=0.0):
        info = claw_step_info()
        st = load().claw_step(self.h, float(dt), ctypes.byref(info))
        if st not in (CLAW_OK, CLAW_ECFL, CLAW_ENONPHYSICAL):
            _check(st, self.h)
        return info.as_dict()

    def advance(self, n=1):
        _check(load().claw_advance(self.h, int(n)), self.h)

    def set_t_end(self, t_end, max_steps=0):
        _check(load().claw_set_t_end(self.h, float(t_end), int(max_steps)), self.h)

    def evolve(self, t_end, max_steps=0, use_graph=True):
        info = claw_step_info()
        st = load().claw_evolve_to_time(self.h, float(t_end), int(max_steps), int(use_graph),
                                        ctypes.byref(info))
        if st not in (CLAW_OK, CLAW_ECFL, CLAW_ENONPHYSICAL):
            _check(st, self.h)
        return info.as_dict()

    def info(self):
        info = claw_step_info()
        _check(load().claw_get_info(self.h, ctypes.byref(info)), self.h)
        return info.as_dict()

    def sync(self):
        _check(load().claw_sync_state(self.h), self.h)
        return self.q

    def current(self):
        p = ctypes.c_void_p()
        _check(load().claw_current_state(self.h, ctypes.byref(p)), self.h)
        return p.value

    def totals(self):
        out = (ctypes.c_double * int(self.method.num_eqn))()
        _check(load().claw_conserved_totals(self.h, out), self.h)
        return np.array(out[:])

    def checkpoint(self):
        n = ctypes.c_size_t(0)
        _check(load().claw_checkpoint(self.h, None, ctypes.byref(n)), self.h)
        buf = ctypes.create_string_buffer(n.value)
        _check(load().claw_checkpoint(self.h, buf, ctypes.byref(n)), self.h)
        return buf.raw

    def restore(self, blob):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(load().claw_restore(self.h, buf, len(blob)), self.h)

    def step_host(self, q_in, q_out, n=1):
        return load().claw_step_host(self.h, ctypes.c_void_p(q_in.data_ptr()),
                                     ctypes.c_void_p(q_out.data_ptr()), int(n))

    def close(self):
        if getattr(self, "h", None):
            load().claw_solver_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many grids of one method, advanced by fused launches over a tile table."""

    def __init__(self, specs, prec="fp32", stream=None):
        torch = _torch()
        dt = _dtype(prec)
        self.specs = specs
        self.method = method_from_spec(specs[0], prec)
        self.n = len(specs)
        grids = (claw_grid * self.n)(*[grid_from_spec(s) for s in specs])
        self.q = [torch.as_tensor(s["q0"], dtype=dt).cuda().contiguous() for s in specs]
        self.aux = [torch.as_tensor(s["aux"], dtype=dt).cuda().contiguous()
                    if s.get("aux") is not None else None for s in specs]
        self.stream = stream if stream is not None else current_stream_handle()
        h = ctypes.c_void_p()
        _check(load().claw_batch_create(ctypes.byref(self.method), grids, self.n,
                                        ctypes.c_void_p(self.stream), ctypes.byref(h)))
        self.h = h
        qp = (ctypes.c_void_p * self.n)(*[t.data_ptr() for t in self.q])
        ap = (ctypes.c_void_p * self.n)(*[(t.data_ptr() if t is not None else 0) for t in self.aux])
        te = (ctypes.c_double * self.n)(*[float(s["t_end"]) for s in specs])
        _check(load().claw_batch_bind(self.h, qp, ap if self.aux[0] is not None else None, te),
               self.h)

    def evolve(self, use_graph=True, max_steps=0):
        infos = (claw_step_info * self.n)()
        st = load().claw_batch_evolve(self.h, int(use_graph), int(max_steps), infos)
        if st not in (CLAW_OK, CLAW_ECFL, CLAW_ENONPHYSICAL):
            _check(st, self.h)
        return [i.as_dict() for i in infos]

    def advance(self, n=1):
        _check(load().claw_batch_advance(self.h, int(n)), self.h)

    def tune(self, bw=None, h=None):
        """Autotune the fused launch (no arguments) or set it; returns (bw, h)."""
        b, hh = ctypes.c_int(bw or 0), ctypes.c_int(h or 0)
        _check(load().claw_batch_tune(self.h, 0 if h is None else 1, ctypes.byref(b),
                                      ctypes.byref(hh)), self.h)
        return b.value, hh.value

    def info(self):
        infos = (claw_step_info * self.n)()
        _check(load().claw_batch_info(self.h, infos), self.h)
        return [i.as_dict() for i in infos]

    def sync(self):
        _check(load().claw_batch_sync_state(self.h), self.h)
        return self.q

    def close(self):
        if getattr(self, "h", None):
            load().claw_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server of independent solves of one method."""

    def __init__(self, spec, prec="fp32", budget_bytes=120 << 30, max_slots=256, stream=None):
        self.method = method_from_spec(spec, prec)
        self.prec = prec
        self.np_dtype = np.float32 if prec in ("fp32", FP32) else np.float64
        self.stream = stream if stream is not None else current_stream_handle()
        h = ctypes.c_void_p()
        _check(load().claw_server_create_nd(ctypes.byref(self.method), int(spec["ndim"]),
                                            int(budget_bytes), int(max_slots),
                                            ctypes.c_void_p(self.stream), ctypes.byref(h)))
        self.h = h
        self.shapes = {}

    def submit(self, spec):
        q0 = np.ascontiguousarray(spec["q0"], dtype=self.np_dtype)
        aux = spec.get("aux")
        aux = np.ascontiguousarray(aux, dtype=self.np_dtype) if aux is not None else None
        g = grid_from_spec(spec)
        t = ctypes.c_uint64()
        st = load().claw_server_submit(self.h, ctypes.byref(g), q0.ctypes.data_as(ctypes.c_void_p),
                                       aux.ctypes.data_as(ctypes.c_void_p) if aux is not None
                                       else None, float(spec["t_end"]), ctypes.byref(t))
        _check(st, self.h)
        self.shapes[t.value] = q0.shape
        return t.value

    def schedule(self, policy="srw", min_cells=1 << 23):
        """'all': every running request steps in every attempt; 'srw':
        shortest remaining work first, min_cells cells per attempt."""
        _check(load().claw_server_schedule(self.h, SCHED[policy], int(min_cells)), self.h)

    def tune(self, bw=None, h=None):
        """Autotune the fused launch on the running requests (no arguments) or
        set it; returns (bw, h)."""
        b, hh = ctypes.c_int(bw or 0), ctypes.c_int(h or 0)
        _check(load().claw_server_tune(self.h, 0 if h is None else 1, ctypes.byref(b),
                                       ctypes.byref(hh)), self.h)
        return b.value, hh.value

    def take_done(self, cap=1024):
        """Tickets finished since the last call (oldest first)."""
        buf = (ctypes.c_uint64 * cap)()
        n = ctypes.c_int()
        _check(load().claw_server_take_done(self.h, buf, int(cap), ctypes.byref(n)), self.h)
        return [int(buf[i]) for i in range(n.value)]

    def pump(self, steps=8):
        r, qd = ctypes.c_int(), ctypes.c_int()
        _check(load().claw_server_pump(self.h, int(steps), ctypes.byref(r), ctypes.byref(qd)),
               self.h)
        return r.value, qd.value

    def poll(self, ticket, want_state=True):
        info = claw_req_info()
        out = np.empty(self.shapes[ticket], dtype=self.np_dtype) if want_state else None
        st = load().claw_server_poll(self.h, ticket,
                                     out.ctypes.data_as(ctypes.c_void_p) if out is not None
                                     else None, ctypes.byref(info))
        if st == CLAW_EBUSY:
            return None
        d = {k: getattr(info, k) for k, _ in claw_req_info._fields_}
        d["status"] = STATUS_NAMES.get(st, st)
        d["q"] = out
        del self.shapes[ticket]
        return d

    def close(self):
        if getattr(self, "h", None):
            load().claw_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def clock():
    return load().claw_clock()


def async_wait_probe(limit_us=20000, stream=None):
    """Self-test of the bounded barrier wait (claw_async_wait_probe): returns
    (gave_up, copied, waited_us)."""
    g, c, w = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
    st = load().claw_async_wait_probe(int(limit_us), stream, ctypes.byref(g), ctypes.byref(c),
                                      ctypes.byref(w))
    if st != CLAW_OK:
        raise RuntimeError(load().claw_last_error(None).decode())
    return bool(g.value), bool(c.value), w.value


def fma_peak(prec="fp64", stream=None, with_clock=False):
    """Measured FMA throughput of the current device in TFLOP/s (claw_fma_peak);
    with_clock: (TFLOP/s, SM MHz the probe ran at)."""
    out, mhz = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = load().claw_fma_peak(FP64 if prec == "fp64" else FP32, stream,
                              ctypes.byref(out), ctypes.byref(mhz))
    if st != CLAW_OK:
        raise RuntimeError(load().claw_last_error(None).decode())
    return (out.value, mhz.value) if with_clock else out.value
