"""Pins for the oracle's pieces of the axisymmetric shock-bubble setup
(Sec. 7.2): the Euler Roe solver with a passive tracer, the geometric source
by Godunov splitting, and dimensionally split classic steps.

Pinned against closed forms and reductions that do not use the oracle's own
formulas: the source ODE's exact solution (both velocities stay constant,
kinetic energy decays like the density, internal energy like its gamma-th
power), the Euler solver without tracer, scalar advection for the tracer in
a uniform flow, the corner-transport-upwind formula and exact translation
for the split step, and the 1D step for data that vary in one direction.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1111_6583_gb300 import workloads as wl


def _euler_spec(rp, nx, ny, **kw):
    return wl.random_smooth_2d(rp, nx, ny, **kw)


@pytest.mark.parametrize("d", [0, 1])
def test_tracer_solver_reduces_to_euler(d):
    st = _euler_spec("euler_tracer", 8, 8)
    se = _euler_spec("euler_roe", 8, 8)
    Pt, Pe = oracle.make_problem(st), oracle.make_problem(se)
    rng = np.random.default_rng(3 + d)
    for trial in range(40):
        def state():
            rho = rng.uniform(0.5, 2.0)
            u, v = rng.normal(0, 1.5, 2)
            p = rng.uniform(0.3, 2.0)
            return np.array([rho, rho * u, rho * v, p / 0.4 + 0.5 * rho * (u * u + v * v),
                             rng.uniform(0, 1)])
        ql, qr = state(), state()
        W, s, am, ap = oracle.riemann(Pt, d, ql, qr)
        We, se_, ame, ape = oracle.riemann(Pe, d, ql[:4], qr[:4])
        # waves: Euler waves (u-c, entropy, shear) then tracer then u+c
        for pt, pe in zip([0, 1, 2, 4], [0, 1, 2, 3]):
            assert np.allclose(W[pt][:4], We[pe], rtol=1e-14, atol=1e-14)
            assert W[pt][4] == 0.0 and s[pt] == se_[pe]
        assert np.allclose(am[:4], ame, rtol=1e-13, atol=1e-13)
        assert np.allclose(ap[:4], ape, rtol=1e-13, atol=1e-13)
        # tracer wave: the jump of phi alone, moving with the normal Roe velocity
        dphi = qr[4] - ql[4]
        assert np.all(W[3][:4] == 0.0) and W[3][4] == dphi
        assert s[3] == se_[1]
        un = s[3]
        assert am[4] == pytest.approx(min(un, 0.0) * dphi, abs=1e-15)
        assert ap[4] == pytest.approx(max(un, 0.0) * dphi, abs=1e-15)
        assert np.allclose(W.sum(axis=0), qr - ql, rtol=1e-13, atol=1e-13)


def test_tracer_in_uniform_flow_is_scalar_advection():
    """Uniform (rho, u, v, p) with a tracer blob: the Euler part stays
    uniform and the tracer follows the scalar advection solver with speeds
    (u, v) (classic, MC, full transverse)."""
    nx, ny = 40, 30
    u, v = 0.7, 0.4
    spec = wl.random_smooth_2d("euler_tracer", nx, ny)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y, indexing="xy")
    phi = np.exp(-60 * ((X - 0.4) ** 2 + (Y - 0.5) ** 2))
    rho, p = 1.3, 0.9
    E = p / 0.4 + 0.5 * rho * (u * u + v * v)
    q = np.stack([np.full_like(X, rho), np.full_like(X, rho * u), np.full_like(X, rho * v),
                  np.full_like(X, E), phi])
    spec["q0"] = q
    sa = wl.random_smooth_2d("advection", nx, ny, params=[u, v])
    sa["q0"] = phi[None].copy()
    Pt, Pa = oracle.make_problem(spec), oracle.make_problem(sa)
    qa = sa["q0"]
    dt = 0.5 / nx
    for _ in range(6):
        q, _ = oracle.step(Pt, q, None, dt)
        qa, _ = oracle.step(Pa, qa, None, dt)
    assert np.abs(q[4] - qa[0]).max() <= 1e-13
    for k, val in enumerate([rho, rho * u, rho * v, E]):
        assert np.abs(q[k] - val).max() <= 1e-13 * abs(val) + 1e-15


def _source_exact(q0, r, t, gamma=1.4):
    rho0, mu, mv, E0 = q0[:4]
    u, v = mu / rho0, mv / rho0
    a = v / r
    ke0 = 0.5 * rho0 * (u * u + v * v)
    rho = rho0 * math.exp(-a * t)
    E = (E0 - ke0) * math.exp(-a * gamma * t) + ke0 * math.exp(-a * t)
    return np.array([rho, rho * u, rho * v, E, q0[4]])


def test_source_step_second_order_to_closed_form():
    """The geometric source ODE has an exact solution (u and v constant,
    rho ~ exp(-v t/r), internal energy ~ exp(-gamma v t/r)); the two-stage
    step's local error falls by 8 when dt halves and vanishes with v = 0."""
    spec = wl.shock_bubble_axisym(nx=4, ny=4, t_end=0.1, sub=2)
    P = oracle.make_problem(spec)
    rng = np.random.default_rng(9)
    q = np.zeros((5, 4, 4))
    for j in range(4):
        for i in range(4):
            rho = rng.uniform(0.5, 2)
            u, v = rng.normal(0, 1, 2)
            p = rng.uniform(0.5, 2)
            q[:, j, i] = [rho, rho * u, rho * v, p / 0.4 + 0.5 * rho * (u * u + v * v),
                          rng.uniform()]
    r = 0.0 + (np.arange(4) + 0.5) * (0.5 / 4)
    for dt in (0.02,):
        e1 = e2 = 0.0
        q1 = oracle.source_step(P, q, dt)
        q2 = oracle.source_step(P, q, dt / 2)
        for j in range(4):
            for i in range(4):
                ex1 = _source_exact(q[:, j, i], r[j], dt)
                ex2 = _source_exact(q[:, j, i], r[j], dt / 2)
                e1 = max(e1, np.abs(q1[:, j, i] - ex1).max() / np.abs(ex1).max())
                e2 = max(e2, np.abs(q2[:, j, i] - ex2).max() / np.abs(ex2).max())
        assert 6.5 < e1 / e2 < 9.5, (e1, e2)
    # integrated to t = 0.1 the error is second order (ratio 4 per halving)
    errs = []
    for nsteps in (200, 400):
        qs = q.copy()
        for _ in range(nsteps):
            qs = oracle.source_step(P, qs, 0.1 / nsteps)
        e = 0.0
        for j in range(4):
            for i in range(4):
                ex = _source_exact(q[:, j, i], r[j], 0.1)
                e = max(e, np.abs(qs[:, j, i] - ex).max() / np.abs(ex).max())
        errs.append(e)
    assert 3.5 < errs[0] / errs[1] < 4.5 and errs[1] < 1e-4, errs
    # no radial velocity: no source
    q0 = q.copy()
    q0[2] = 0.0
    q0[3] = 1.0 / 0.4 + 0.5 * q0[1] ** 2 / q0[0]
    assert np.array_equal(oracle.source_step(P, q0, 0.05), q0)


def test_uniform_state_step_is_the_source_step():
    """Godunov splitting: on a uniform state the hyperbolic step changes
    nothing (periodic), so the step equals one source step."""
    spec = wl.shock_bubble_axisym(nx=12, ny=8, t_end=0.1, sub=2)
    spec.update(bc_lower=["periodic", "periodic"], bc_upper=["periodic", "periodic"])
    rho, u, v, p = 1.2, 0.3, -0.2, 1.1
    E = p / 0.4 + 0.5 * rho * (u * u + v * v)
    q = np.stack([np.full((8, 12), x) for x in (rho, rho * u, rho * v, E, 0.5)])
    P = oracle.make_problem(spec)
    got, _ = oracle.step(P, q, None, 0.01)
    want = oracle.source_step(P, q, 0.01)
    assert np.abs(got - want).max() <= 1e-14 * np.abs(want).max()


def test_tracer_is_passive_in_the_axisymmetric_run():
    """The Euler components of the shock-bubble run do not depend on the
    tracer: the same run without it (Euler Roe, 4 components) agrees."""
    st = wl.shock_bubble_axisym(nx=80, ny=20, t_end=0.05, sub=4)
    se = dict(st, rp="euler_roe", q0=st["q0"][:4].copy(), inflow=st["inflow"][:4])
    qt, it = oracle.evolve(oracle.make_problem(st), st["q0"], None, t_end=0.05)
    qe, ie = oracle.evolve(oracle.make_problem(se), se["q0"], None, t_end=0.05)
    assert it["steps"] == ie["steps"] and it["status"] == ie["status"] == "ok"
    assert np.abs(qt[:4] - qe).max() <= 1e-12 * np.abs(qe).max()


def test_split_order1_advection_is_ctu():
    """First-order upwind sweeps, x then y, compose to the corner-transport
    upwind formula for u, v > 0."""
    nx, ny = 24, 20
    u, v = 1.0, 0.6
    spec = wl.random_smooth_2d("advection", nx, ny, params=[u, v], order=1, dim_split=1)
    q = spec["q0"]
    dt = 0.7 / nx
    nux, nuy = u * dt * nx, v * dt * ny
    got, _ = oracle.step(oracle.make_problem(spec), q, None, dt)
    Q = q[0]
    want = ((1 - nux) * (1 - nuy) * Q + nux * (1 - nuy) * np.roll(Q, 1, axis=1) +
            (1 - nux) * nuy * np.roll(Q, 1, axis=0) + nux * nuy * np.roll(np.roll(Q, 1, 0), 1, 1))
    assert np.abs(got[0] - want).max() <= 1e-14


@pytest.mark.parametrize("lim", ["mc", "superbee", "none"])
def test_split_translates_exactly_at_unit_courant(lim):
    nx = ny = 32
    spec = wl.random_smooth_2d("advection", nx, ny, params=[1.0, 1.0], lim=lim, dim_split=1)
    q = spec["q0"]
    got, cfl = oracle.step(oracle.make_problem(spec), q, None, 1.0 / nx)
    assert abs(cfl - 1.0) < 1e-14
    assert np.abs(got[0] - np.roll(np.roll(q[0], 1, 0), 1, 1)).max() <= 1e-14


def test_split_step_on_x_data_is_the_1d_step():
    """Data varying in x only: the y sweeps change nothing and the split step
    is the 1D step (Euler with the 2D solver's x direction)."""
    n1 = 64
    s1 = wl.random_1d("euler_roe", n1, jump=True)
    q1 = s1["q0"]
    q2 = np.zeros((4, 6, n1))
    q2[0] = q1[0][None]
    q2[1] = q1[1][None]
    q2[3] = q1[2][None]
    s2 = wl.random_smooth_2d("euler_roe", n1, 6, dim_split=1, transverse=0)
    s2["q0"] = q2
    P1, P2 = oracle.make_problem(s1), oracle.make_problem(s2)
    dt = 0.3 / n1
    a, c1 = oracle.step(P1, q1, None, dt)
    b, c2 = oracle.step(P2, q2, None, dt)
    assert abs(c1 - c2) <= 1e-15 * c1
    for k2, k1 in ((0, 0), (1, 1), (3, 2)):
        assert np.abs(b[k2] - a[k1][None]).max() <= 1e-13 * np.abs(a[k1]).max()
    assert np.abs(b[2]).max() <= 1e-15


def test_split_conserves_periodic():
    spec = wl.random_smooth_2d("euler_tracer", 30, 20, dim_split=1, transverse=0)
    P = oracle.make_problem(spec)
    q = spec["q0"]
    t0 = q[:4].sum(axis=(1, 2))
    for _ in range(5):
        q, _ = oracle.step(P, q, None, 0.3 / 30)
    assert np.abs(q[:4].sum(axis=(1, 2)) - t0).max() <= 1e-12 * np.abs(t0).max()
