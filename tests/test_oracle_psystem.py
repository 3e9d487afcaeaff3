"""Pins for the oracle's 2D p-system (Sec. 7.3: strain and momenta in a
spatially varying medium, f-wave normal solves, SharpClaw WENO).

Pinned against facts that do not come from the oracle's own formulas: the
f-waves sum to the normal flux jump and are eigenvectors of the normal
Jacobian on each side; data that vary in one direction only reduce to the
1D elasticity solver (itself pinned); the x <-> y transpose and the mirror
image across a reflecting wall; telescoping of the fluctuations (periodic
conservation).
"""
import numpy as np
import pytest

import oracle
from paper_1111_6583_gb300 import workloads as wl


def _flux(q, a, n):
    """normal flux of the p-system, written out here: (-m_n/rho, -sigma) in
    the (eps, m_n) components, sigma = exp(K eps) - 1"""
    f = np.zeros(3)
    f[0] = -q[n] / a[0]
    f[n] = -(np.exp(a[1] * q[0]) - 1.0)
    return f


@pytest.mark.parametrize("d", [0, 1])
def test_fwaves_sum_to_flux_jump_and_are_eigenvectors(d):
    spec = wl.random_smooth_2d("elasticity_fwave", 16, 16)
    P = oracle.make_problem(spec)
    rng = np.random.default_rng(7 + d)
    n, t = 1 + d, 2 - d
    for _ in range(30):
        ql = np.array([rng.uniform(-0.2, 0.4), rng.normal(), rng.normal()])
        qr = np.array([rng.uniform(-0.2, 0.4), rng.normal(), rng.normal()])
        al = np.array([rng.uniform(0.5, 5), rng.uniform(0.5, 5)])
        ar = np.array([rng.uniform(0.5, 5), rng.uniform(0.5, 5)])
        W, s, am, ap = oracle.riemann(P, d, ql, qr, al, ar)
        df = _flux(qr, ar, n) - _flux(ql, al, n)
        assert np.allclose(W.sum(axis=0), df, rtol=0, atol=1e-13 * (1 + np.abs(df).max()))
        assert np.allclose(am + ap, df, rtol=0, atol=1e-13 * (1 + np.abs(df).max()))
        assert np.all(W[:, t] == 0.0)
        # eigenvectors (1, +Z_l) (speed -c_l) and (1, -Z_r) (speed +c_r) of
        # the normal Jacobian [[0, -1/rho], [-sigma', 0]] on each side
        for (w, sp, a, q, sgn) in ((W[0], s[0], al, ql, 1.0), (W[1], s[1], ar, qr, -1.0)):
            c = np.sqrt(a[1] * np.exp(a[1] * q[0]) / a[0])
            Z = a[0] * c
            assert abs(sp - (-sgn) * c) <= 1e-14 * c
            assert abs(w[n] - sgn * Z * w[0]) <= 1e-13 * (abs(w[n]) + 1e-300)
        assert np.allclose(am, W[0]) and np.allclose(ap, W[1])


@pytest.mark.parametrize("d", [0, 1])
def test_one_dimensional_data_reduce_to_1d_elasticity(d):
    """Data and medium varying along direction d only: the 2D SharpClaw step
    equals the 1D elasticity step in (eps, m_d), and the other momentum
    stays zero."""
    n1, n2 = 48, 8
    sp1 = wl.random_1d("elasticity_fwave", n1, scheme="sharpclaw", char_decomp=0)
    q1, a1 = sp1["q0"], sp1["aux"]
    shape = (n2, n1) if d == 0 else (n1, n2)
    sp2 = wl.random_smooth_2d("elasticity_fwave", shape[1], shape[0])
    q2 = np.zeros((3,) + shape)
    a2 = np.zeros((2,) + shape)
    for k in range(2):
        a2[k] = a1[k][None, :] if d == 0 else a1[k][:, None]
    q2[0] = q1[0][None, :] if d == 0 else q1[0][:, None]
    q2[1 + d] = q1[1][None, :] if d == 0 else q1[1][:, None]
    sp2.update(q0=np.ascontiguousarray(q2), aux=np.ascontiguousarray(a2), bc_lower=["periodic"] * 2,
               bc_upper=["periodic"] * 2)
    sp2["n"] = [shape[1], shape[0]]
    P1, P2 = oracle.make_problem(sp1), oracle.make_problem(sp2)
    dt = 0.2 / n1
    for _ in range(3):
        q1, _ = oracle.step(P1, q1, a1, dt)
        q2, _ = oracle.step(P2, q2, sp2["aux"], dt)
    got_e = q2[0][0, :] if d == 0 else q2[0][:, 0]
    got_m = q2[1 + d][0, :] if d == 0 else q2[1 + d][:, 0]
    assert np.abs(got_e - q1[0]).max() <= 1e-13 * np.abs(q1[0]).max()
    assert np.abs(got_m - q1[1]).max() <= 1e-13 * np.abs(q1[1]).max()
    assert np.all(q2[2 - d] == 0.0)


def test_transpose_symmetry():
    sp = wl.random_smooth_2d("elasticity_fwave", 32, 24)
    spt = dict(sp)
    q = sp["q0"]
    spt["q0"] = np.ascontiguousarray(np.stack([q[0].T, q[2].T, q[1].T]))
    spt["aux"] = np.ascontiguousarray(np.stack([sp["aux"][0].T, sp["aux"][1].T]))
    spt["n"] = [24, 32]
    P, Pt = oracle.make_problem(sp), oracle.make_problem(spt)
    L, sm = oracle.sharp_L(P, sp["q0"], sp["aux"])
    Lt, smt = oracle.sharp_L(Pt, spt["q0"], spt["aux"])
    scale = np.abs(L).max()
    assert np.abs(Lt[0].T - L[0]).max() <= 1e-13 * scale
    assert np.abs(Lt[1].T - L[2]).max() <= 1e-13 * scale
    assert np.abs(Lt[2].T - L[1]).max() <= 1e-13 * scale
    assert abs(sm[0] - smt[1]) <= 1e-15 * sm[0] and abs(sm[1] - smt[0]) <= 1e-15 * sm[1]


def test_periodic_fluctuations_telescope():
    """f-waves sum to the jump of the flux with each cell's own medium, so
    the interface and in-cell fluctuations telescope: sum_i L_i = 0."""
    for order in (5, 7):
        sp = wl.random_smooth_2d("elasticity_fwave", 32, 24, weno_order=order)
        L, _ = oracle.sharp_L(oracle.make_problem(sp), sp["q0"], sp["aux"])
        for k in range(3):
            assert abs(L[k].sum()) <= 1e-13 * np.abs(L[k]).max() * L[k].size


def test_wall_is_the_mirror_image():
    """The quadrant problem (walls at x = 0 and y = 0, extrapolation at the
    far sides) equals the positive quadrant of the full problem whose data
    and medium are the mirror extension (strain even, each momentum odd in
    its own direction)."""
    sp = wl.psystem_checkerboard_2d(periods=2, cells_per_period=12, t_end=0.1,
                                    integrator="ssp_rk3")
    n = sp["n"][0]
    q, a = sp["q0"], sp["aux"]

    def ext(f, sx, sy):
        top = np.concatenate([sx * f[:, ::-1], f], axis=1)
        return np.concatenate([sy * top[::-1, :], top], axis=0)

    qf = np.stack([ext(q[0], 1, 1), ext(q[1], -1, 1), ext(q[2], 1, -1)])
    af = np.stack([ext(a[0], 1, 1), ext(a[1], 1, 1)])
    full = dict(sp, n=[2 * n, 2 * n], lower=[-2.0, -2.0], upper=[2.0, 2.0],
                bc_lower=["extrap", "extrap"], bc_upper=["extrap", "extrap"],
                q0=np.ascontiguousarray(qf), aux=np.ascontiguousarray(af))
    # a moving state: let the pulse run a little first
    Pq, Pf = oracle.make_problem(sp), oracle.make_problem(full)
    dt = 0.2 * sp["upper"][0] / n / 2.5
    for _ in range(4):
        q, _ = oracle.step(Pq, q, a, dt)
        qf, _ = oracle.step(Pf, qf, af, dt)
    sub = qf[:, n:, n:]
    for k in range(3):
        assert np.abs(sub[k] - q[k]).max() <= 1e-13 * np.abs(q).max()
