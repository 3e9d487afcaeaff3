"""Pins of the CPU oracle against what the method and the mathematics fix.

The paper prints no worked example with numbers (its figures are not
reproduced and its tables are wall-clock times), so every pin here is a
closed form, an invariant, a special case with a known exact answer, or an
observed convergence order:

* Riemann solvers: Roe property (sum of waves = jump, sum of s*W = flux jump),
  eigenpairs against a finite-difference Jacobian of independently written
  fluxes, fluctuation sums, f-wave sums, transverse splits.
* Limiters: values at chosen theta and the symmetry phi(th)/th = phi(1/th).
* WENO5: polynomial exactness, ENO behaviour at a jump, spatial order 5.
* SSP-RK3: stability polynomial 1 + z + z^2/2 + z^3/6.
* Classic step: exact translation at Courant number 1 (1D advection, 1D
  acoustics, 2D diagonal advection), corner-transport upwind formula,
  conservation, symmetry, second-order convergence, exact Riemann solutions
  (Sod, dam break).
* Controller: final-time clipping, reject/retry, error statuses.
"""
import math

import numpy as np
import pytest

from paper_1111_6583_gb300 import workloads as wl
from tests.exact_riemann import euler_exact, sw_dambreak_exact

RNG = np.random.Generator(np.random.PCG64(6583))


# --------------------------------------------------------------------------
# independent flux functions (written from the PDEs, not from the oracle)
# --------------------------------------------------------------------------
def flux(rp, ndim, d, q, params, aux=None):
    q = np.asarray(q, dtype=float)
    if rp == "advection":
        return params[d] * q
    if rp == "acoustics":
        rho, K = params[0], params[1]
        if ndim == 1:
            return np.array([K * q[1], q[0] / rho])
        f = np.zeros(3)
        f[0] = K * q[1 + d]
        f[1 + d] = q[0] / rho
        return f
    if rp == "sw_roe":
        g = params[0]
        h = q[0]
        if ndim == 1:
            return np.array([q[1], q[1] ** 2 / h + 0.5 * g * h * h])
        hu, hv = q[1], q[2]
        if d == 0:
            return np.array([hu, hu * hu / h + 0.5 * g * h * h, hu * hv / h])
        return np.array([hv, hu * hv / h, hv * hv / h + 0.5 * g * h * h])
    if rp in ("euler_roe", "euler_hlle"):
        gam = params[0]
        rho = q[0]
        if ndim == 1:
            u = q[1] / rho
            p = (gam - 1) * (q[2] - 0.5 * rho * u * u)
            return np.array([rho * u, rho * u * u + p, u * (q[2] + p)])
        u, v = q[1] / rho, q[2] / rho
        p = (gam - 1) * (q[3] - 0.5 * rho * (u * u + v * v))
        if d == 0:
            return np.array([rho * u, rho * u * u + p, rho * u * v, u * (q[3] + p)])
        return np.array([rho * v, rho * u * v, rho * v * v + p, v * (q[3] + p)])
    if rp == "elasticity_fwave":
        rho, K = aux
        return np.array([-q[1] / rho, -(math.exp(K * q[0]) - 1.0)])
    raise ValueError(rp)


def rand_state(rp, ndim, scale_u=1.0):
    if rp == "sw_roe":
        h = RNG.uniform(0.5, 2.0)
        vel = RNG.uniform(-scale_u, scale_u, ndim)
        return np.concatenate([[h], h * vel])
    if rp in ("euler_roe", "euler_hlle"):
        rho = RNG.uniform(0.5, 2.0)
        vel = RNG.uniform(-scale_u, scale_u, ndim)
        p = RNG.uniform(0.5, 2.0)
        E = p / 0.4 + 0.5 * rho * np.dot(vel, vel)
        return np.concatenate([[rho], rho * vel, [E]])
    if rp == "acoustics":
        return RNG.uniform(-1, 1, ndim + 1)
    if rp == "advection":
        return RNG.uniform(-1, 1, 1)
    if rp == "elasticity_fwave":
        return np.array([RNG.uniform(-0.2, 0.2), RNG.uniform(-1, 1)])
    raise ValueError(rp)


PARAMS = {"advection": [0.7, -0.4], "acoustics": [1.3, 2.5], "sw_roe": [1.0],
          "euler_roe": [1.4], "euler_hlle": [1.4], "elasticity_fwave": []}

CASES = [(rp, nd) for rp in ("advection", "acoustics", "sw_roe", "euler_roe", "euler_hlle")
         for nd in (1, 2)] + [("elasticity_fwave", 1)]


def prob(orc, rp, ndim, entropy_fix=1):
    spec = dict(ndim=ndim, n=[8] * ndim, lower=[0.0] * ndim, upper=[1.0] * ndim, rp=rp,
                params=PARAMS[rp], entropy_fix=entropy_fix)
    return orc.make_problem(spec)


def rand_aux():
    return np.array([RNG.uniform(0.5, 4.0), RNG.uniform(0.5, 4.0)])


def jacobian(fn, q, h=1e-6):
    n = len(q)
    J = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n); e[k] = h * max(1.0, abs(q[k]))
        J[:, k] = (fn(q + e) - fn(q - e)) / (2 * e[k])
    return J


# --------------------------------------------------------------------------
# Riemann solvers
# --------------------------------------------------------------------------
@pytest.mark.parametrize("rp,ndim", CASES)
def test_fluctuations_sum_to_flux_jump(orc, rp, ndim):
    """A^- dQ + A^+ dQ = f(Q_r) - f(Q_l) (conservation of the fluctuation form)."""
    P = prob(orc, rp, ndim)
    for _ in range(200):
        for d in range(ndim):
            ql, qr = rand_state(rp, ndim, 2.0), rand_state(rp, ndim, 2.0)
            al, ar = (rand_aux(), rand_aux()) if rp == "elasticity_fwave" else (None, None)
            W, s, am, ap = orc.riemann(P, d, ql, qr, al, ar)
            df = flux(rp, ndim, d, qr, PARAMS[rp], ar) - flux(rp, ndim, d, ql, PARAMS[rp], al)
            scale = np.abs(df).max() + np.abs(am).max() + 1.0
            assert np.abs(am + ap - df).max() <= 1e-13 * scale


@pytest.mark.parametrize("rp,ndim", [c for c in CASES if c[0] not in ("elasticity_fwave",)])
def test_roe_property(orc, rp, ndim):
    """Waves sum to the jump (except the omitted zero-speed acoustic shear wave)
    and sum_p s^p W^p = f(Q_r) - f(Q_l)."""
    P = prob(orc, rp, ndim, entropy_fix=0)
    for _ in range(200):
        for d in range(ndim):
            ql, qr = rand_state(rp, ndim), rand_state(rp, ndim)
            W, s, am, ap = orc.riemann(P, d, ql, qr)
            dq = qr - ql
            tot = W.sum(axis=0)
            if rp == "acoustics" and ndim == 2:
                t = 2 - d  # tangential velocity jump rides on the omitted zero-speed wave
                dq = dq.copy(); dq[t] = 0.0
            assert np.abs(tot - dq).max() <= 1e-13 * (np.abs(dq).max() + 1)
            df = flux(rp, ndim, d, qr, PARAMS[rp]) - flux(rp, ndim, d, ql, PARAMS[rp])
            sw = (s[:, None] * W).sum(axis=0)
            assert np.abs(sw - df).max() <= 1e-13 * (np.abs(df).max() + 1)


@pytest.mark.parametrize("rp,ndim", [("acoustics", 1), ("acoustics", 2), ("sw_roe", 1),
                                     ("sw_roe", 2), ("euler_roe", 1), ("euler_roe", 2)])
def test_waves_are_jacobian_eigenpairs(orc, rp, ndim):
    """For a small jump the waves are eigenvectors of the flux Jacobian with the
    returned speeds as eigenvalues (catches swapped speeds or eigenvectors)."""
    P = prob(orc, rp, ndim, entropy_fix=0)
    for _ in range(30):
        for d in range(ndim):
            q = rand_state(rp, ndim)
            dq = RNG.uniform(-1, 1, len(q)) * 1e-6
            W, s, _, _ = orc.riemann(P, d, q - dq / 2, q + dq / 2)
            J = jacobian(lambda x: flux(rp, ndim, d, x, PARAMS[rp]), q)
            for p in range(len(s)):
                nrm = np.abs(W[p]).max()
                if nrm < 1e-12:
                    continue
                res = J @ W[p] - s[p] * W[p]
                assert np.abs(res).max() <= 1e-4 * nrm * (1 + abs(s[p]))


def test_elasticity_fwaves(orc):
    """f-waves sum to the flux jump and are eigenvectors (1, +-Z) of each side's
    Jacobian with speeds -c_l, +c_r, c = sqrt(K exp(K eps)/rho)."""
    P = prob(orc, "elasticity_fwave", 1)
    for _ in range(200):
        ql, qr = rand_state("elasticity_fwave", 1), rand_state("elasticity_fwave", 1)
        al, ar = rand_aux(), rand_aux()
        W, s, am, ap = orc.riemann(P, 0, ql, qr, al, ar)
        df = flux("elasticity_fwave", 1, 0, qr, [], ar) - flux("elasticity_fwave", 1, 0, ql, [], al)
        assert np.abs(W.sum(axis=0) - df).max() <= 1e-13 * (np.abs(df).max() + 1)
        cl = math.sqrt(al[1] * math.exp(al[1] * ql[0]) / al[0])
        cr = math.sqrt(ar[1] * math.exp(ar[1] * qr[0]) / ar[0])
        assert s[0] == pytest.approx(-cl, rel=1e-14) and s[1] == pytest.approx(cr, rel=1e-14)
        Jl = jacobian(lambda x: flux("elasticity_fwave", 1, 0, x, [], al), ql)
        Jr = jacobian(lambda x: flux("elasticity_fwave", 1, 0, x, [], ar), qr)
        for J, w, sp in ((Jl, W[0], s[0]), (Jr, W[1], s[1])):
            if np.abs(w).max() > 1e-12:
                assert np.abs(J @ w - sp * w).max() <= 1e-6 * np.abs(w).max() * (1 + abs(sp))
        assert np.allclose(am, W[0], rtol=0, atol=0) and np.allclose(ap, W[1], rtol=0, atol=0)


@pytest.mark.parametrize("rp", ["sw_roe", "euler_roe"])
def test_entropy_fix_transonic(orc, rp):
    """Harten-Hyman: in a transonic rarefaction the fix changes the split but
    keeps A^-dQ + A^+dQ = flux jump; without a sonic point it changes nothing."""
    P1 = prob(orc, rp, 1, 1)
    P0 = prob(orc, rp, 1, 0)
    if rp == "sw_roe":
        ql, qr = np.array([1.0, 0.5]), np.array([0.3, 0.3 * 1.8])  # u-c: -0.5 -> +1.25
    else:
        ql = np.array([1.0, 0.5, 1.0 / 0.4 + 0.125])
        qr = np.array([0.2, 0.2 * 2.5, 0.1 / 0.4 + 0.5 * 0.2 * 6.25])
    W, s, am1, ap1 = orc.riemann(P1, 0, ql, qr)
    _, _, am0, ap0 = orc.riemann(P0, 0, ql, qr)
    df = flux(rp, 1, 0, qr, PARAMS[rp]) - flux(rp, 1, 0, ql, PARAMS[rp])
    assert np.abs(am1 + ap1 - df).max() <= 1e-13 * (np.abs(df).max() + 1)
    assert np.abs(am1 - am0).max() > 1e-3  # the fix acted
    # subsonic pair: identical with and without the fix
    ql2, qr2 = rand_state(rp, 1, 0.2), rand_state(rp, 1, 0.2)
    _, _, a1, b1 = orc.riemann(P1, 0, ql2, qr2)
    _, _, a0, b0 = orc.riemann(P0, 0, ql2, qr2)
    assert np.array_equal(a1, a0) and np.array_equal(b1, b0)


@pytest.mark.parametrize("rp,ndim", CASES)
def test_equal_states_zero_fluctuation(orc, rp, ndim):
    P = prob(orc, rp, ndim)
    for d in range(ndim):
        q = rand_state(rp, ndim)
        a = rand_aux() if rp == "elasticity_fwave" else None
        W, s, am, ap = orc.riemann(P, d, q, q, a, a)
        assert np.abs(am).max() <= 1e-15 and np.abs(ap).max() <= 1e-15


@pytest.mark.parametrize("rp", ["sw_roe", "euler_roe", "euler_hlle"])
def test_wall_pair_zero_mass_flux(orc, rp):
    """Mirror states (momentum negated) give zero mass flux f(Q_l) + A^-dQ."""
    P = prob(orc, rp, 1)
    for _ in range(50):
        ql = rand_state(rp, 1)
        qr = ql.copy(); qr[1] = -qr[1]
        W, s, am, ap = orc.riemann(P, 0, ql, qr)
        F = flux(rp, 1, 0, ql, PARAMS[rp]) + am
        assert abs(F[0]) <= 1e-13 * (abs(ql[1]) + 1)


@pytest.mark.parametrize("rp", ["advection", "acoustics", "sw_roe", "euler_roe"])
def test_transverse_split(orc, rp):
    """At Q_l = Q_r = Q: B^- a + B^+ a = J_g(Q) a (J_g the transverse-flux
    Jacobian); an eigenvector of J_g goes entirely to the side of its sign."""
    P = prob(orc, rp, 2)
    for _ in range(20):
        for d in range(2):
            q = rand_state(rp, 2, 0.5)
            a = RNG.uniform(-1, 1, len(q))
            bm, bp = orc.transverse(P, d, q, q, a)
            Jg = jacobian(lambda x: flux(rp, 2, 1 - d, x, PARAMS[rp]), q)
            assert np.abs(bm + bp - Jg @ a).max() <= 1e-6 * (np.abs(a).max() + 1)
            lam, V = np.linalg.eig(Jg)
            for k in range(len(lam)):
                v = np.real(V[:, k]); lk = np.real(lam[k])
                if abs(lk) < 1e-6:
                    continue
                bm, bp = orc.transverse(P, d, q, q, v)
                if lk < 0:
                    assert np.abs(bp).max() <= 1e-6 and np.abs(bm - lk * v).max() <= 1e-6
                else:
                    assert np.abs(bm).max() <= 1e-6 and np.abs(bp - lk * v).max() <= 1e-6


@pytest.mark.parametrize("rp,ndim", [("acoustics", 1), ("acoustics", 2), ("sw_roe", 1),
                                     ("sw_roe", 2), ("euler_roe", 1), ("euler_roe", 2)])
def test_char_matrices_inverse(orc, rp, ndim):
    P = prob(orc, rp, ndim)
    for d in range(ndim):
        L, R = orc.char_matrices(P, d, rand_state(rp, ndim), rand_state(rp, ndim))
        assert np.abs(L @ R - np.eye(len(L))).max() <= 1e-13


# --------------------------------------------------------------------------
# limiters, WENO5, SSP-RK3
# --------------------------------------------------------------------------
def test_limiter_values(orc):
    table = {
        "minmod": [(-1.0, 0.0), (0.5, 0.5), (2.0, 1.0)],
        "superbee": [(-1.0, 0.0), (0.25, 0.5), (0.5, 1.0), (1.5, 1.5), (3.0, 2.0)],
        "mc": [(-1.0, 0.0), (0.2, 0.4), (0.5, 0.75), (1.0, 1.0), (2.0, 1.5), (4.0, 2.0)],
        "vanleer": [(-1.0, 0.0), (1.0, 1.0), (3.0, 1.5)],
        "none": [(-3.0, 1.0), (0.0, 1.0), (5.0, 1.0)],
    }
    for lim, pts in table.items():
        for th, val in pts:
            assert orc.phi(lim, th) == pytest.approx(val, abs=1e-15), (lim, th)
    for lim in ("minmod", "superbee", "mc", "vanleer"):
        for th in np.linspace(0.05, 20, 97):
            assert orc.phi(lim, th) / th == pytest.approx(orc.phi(lim, 1 / th), rel=1e-13)


def test_weno5_polynomials(orc):
    # constants are reproduced
    assert orc.weno5([3.0] * 5) == pytest.approx(3.0, abs=1e-15)

    def cavg(c, a, b):  # exact cell average of sum c_k x^k over [a, b]
        return sum(ck * (b ** (k + 1) - a ** (k + 1)) / (k + 1) for k, ck in enumerate(c)) / (b - a)

    for _ in range(20):
        # degree 2: every candidate stencil is exact, so any weights are exact
        c = RNG.uniform(-1, 1, 3)
        v = [cavg(c, i - 0.5, i + 0.5) for i in range(-2, 3)]
        assert orc.weno5(v, 1e-6) == pytest.approx(np.polyval(c[::-1], 0.5), abs=1e-13)
        # degree 4 with linear weights (huge epsilon): fifth-order exact
        c = RNG.uniform(-1, 1, 5)
        v = [cavg(c, i - 0.5, i + 0.5) for i in range(-2, 3)]
        assert orc.weno5(v, 1e13) == pytest.approx(np.polyval(c[::-1], 0.5), abs=1e-9)
    # ENO behaviour at a jump between cells i and i+1: the left stencil wins
    assert abs(orc.weno5([0.0, 0.0, 0.0, 1.0, 1.0])) < 1e-9


def test_ssp_rk3_stability_polynomial(orc):
    for z in (-2.5, -1.0, -0.3, 0.2, 1.0):
        assert orc.ssp_rk3_linear(z, 1.0, 1.0) == pytest.approx(1 + z + z * z / 2 + z ** 3 / 6,
                                                                rel=1e-14)
        assert orc.ssp_rk3_linear(z / 0.25, 0.25, 2.0) == pytest.approx(
            2 * (1 + z + z * z / 2 + z ** 3 / 6), rel=1e-14)


# --------------------------------------------------------------------------
# ghost cells
# --------------------------------------------------------------------------
def test_ghost_cells_1d(orc):
    q = np.stack([np.arange(1.0, 6.0), np.arange(10.0, 15.0)])
    for bc, lo, hi in (("periodic", [[4, 5], [13, 14]], [[1, 2], [10, 11]]),
                       ("extrap", [[1, 1], [10, 10]], [[5, 5], [14, 14]]),
                       ("wall", [[2, 1], [-11, -10]], [[5, 4], [-14, -13]])):
        spec = dict(ndim=1, n=[5], lower=[0.0], upper=[1.0], rp="acoustics", params=[1, 1],
                    bc_lower=[bc], bc_upper=[bc])
        g = orc.fill_ghost(orc.make_problem(spec), q, 2)
        assert np.array_equal(g[:, :2], np.array(lo, float)), bc
        assert np.array_equal(g[:, -2:], np.array(hi, float)), bc
        assert np.array_equal(g[:, 2:-2], q)
    spec = dict(ndim=1, n=[5], lower=[0.0], upper=[1.0], rp="acoustics", params=[1, 1],
                bc_lower=["inflow"], bc_upper=["extrap"], inflow=[7.0, 8.0])
    g = orc.fill_ghost(orc.make_problem(spec), q, 3)
    assert np.array_equal(g[:, :3], np.array([[7, 7, 7], [8, 8, 8]], float))


def test_ghost_corners_2d(orc):
    """2D: x ghosts on interior rows first, then y ghosts on all columns, so a
    corner of a wall/wall box negates both momenta."""
    nx, ny = 4, 3
    q = RNG.uniform(0.5, 1.5, (3, ny, nx))
    spec = dict(ndim=2, n=[nx, ny], lower=[0, 0], upper=[1, 1], rp="sw_roe", params=[1.0],
                bc_lower=["wall", "wall"], bc_upper=["wall", "wall"])
    g = orc.fill_ghost(orc.make_problem(spec), q, 2)
    # corner ghost (-1,-1) mirrors cell (0,0); both momenta negated
    assert g[0, 1, 1] == q[0, 0, 0]
    assert g[1, 1, 1] == -q[1, 0, 0] and g[2, 1, 1] == -q[2, 0, 0]
    spec.update(bc_lower=["periodic", "extrap"], bc_upper=["periodic", "extrap"])
    g = orc.fill_ghost(orc.make_problem(spec), q, 2)
    assert np.array_equal(g[:, 0, 0], q[:, 0, nx - 2])  # y-extrap of x-periodic ghost


# --------------------------------------------------------------------------
# classic step: exact translation, CTU, conservation, symmetry, orders
# --------------------------------------------------------------------------
def _adv1d(orc, n, lim="mc", order=2, u=1.0, **kw):
    spec = dict(ndim=1, n=[n], lower=[0.0], upper=[1.0], rp="advection", params=[u], lim=lim,
                order=order, bc_lower=["periodic"], bc_upper=["periodic"])
    spec.update(kw)
    return orc.make_problem(spec)


@pytest.mark.parametrize("lim,order", [("none", 1), ("none", 2), ("minmod", 2), ("superbee", 2),
                                       ("vanleer", 2), ("mc", 2)])
def test_advection_exact_at_courant_one(orc, lim, order):
    n = 64
    x = (np.arange(n) + 0.5) / n
    q0 = np.stack([np.where((x > 0.2) & (x < 0.5), 1.0, 0.0) + np.sin(6 * np.pi * x)])
    P = _adv1d(orc, n, lim, order)
    q1, cfl = orc.step(P, q0, dt=1.0 / n)
    assert cfl == 1.0
    assert np.abs(q1 - np.roll(q0, 1, axis=1)).max() <= 1e-15
    P = _adv1d(orc, n, lim, order, dt_initial=1.0 / n, cfl_desired=1.0)
    qT, info = orc.evolve(P, q0, t_end=1.0)
    assert info["steps"] == n and info["t"] == 1.0
    assert np.abs(qT - q0).max() <= 1e-14


def test_acoustics_exact_at_courant_one(orc):
    """rho=1, K=4 (c=2) on [-1,1] with dt = dx/c: both families move exactly one
    cell per step, so at t=2 the pulse is back where it started."""
    spec = wl.acoustics_1d(n=256, t_end=2.0)
    spec.update(dt_initial=1.0 / 256, cfl_desired=1.0)
    P = orc.make_problem(spec)
    qT, info = orc.evolve(P, spec["q0"], t_end=2.0)
    assert info["steps"] == 512 and info["status"] == "ok"
    assert np.abs(qT - spec["q0"]).max() <= 1e-12


def test_acoustics_pulse_refinement(orc):
    """At CFL 0.9 the error against the initial data at t=2 falls under refinement."""
    errs = []
    for n in (250, 500, 1000, 2000):
        spec = wl.acoustics_1d(n=n)
        qT, info = orc.evolve(orc.make_problem(spec), spec["q0"], t_end=2.0)
        assert info["t"] == 2.0 and info["status"] == "ok"
        errs.append(np.abs(qT - spec["q0"]).sum() * 2.0 / n)
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 0.02


def _adv2d(orc, n, u, v, order, transverse, lim="none", **kw):
    spec = dict(ndim=2, n=[n, n], lower=[0, 0], upper=[1, 1], rp="advection", params=[u, v],
                order=order, transverse=transverse, lim=lim,
                bc_lower=["periodic"] * 2, bc_upper=["periodic"] * 2)
    spec.update(kw)
    return orc.make_problem(spec)


def test_ctu_diagonal_shift_and_formula(orc):
    n = 32
    q0 = RNG.uniform(-1, 1, (1, n, n))
    for order, tr in ((1, 1), (2, 2), (2, 1)):
        q1, cfl = orc.step(_adv2d(orc, n, 1.0, 1.0, order, tr, "mc"), q0, dt=1.0 / n)
        assert np.abs(q1 - np.roll(q0, (1, 1), axis=(1, 2))).max() <= 1e-14
    # Courant numbers below one: first order with transverse fluctuations is CTU
    u, v, dt = 1.0, 0.5, 0.5 / n
    nx_, ny_ = u * dt * n, v * dt * n
    q1, _ = orc.step(_adv2d(orc, n, u, v, 1, 1), q0, dt=dt)
    Q = q0[0]
    ctu = ((1 - nx_) * (1 - ny_) * Q + nx_ * (1 - ny_) * np.roll(Q, 1, axis=1)
           + (1 - nx_) * ny_ * np.roll(Q, 1, axis=0) + nx_ * ny_ * np.roll(Q, (1, 1), axis=(0, 1)))
    assert np.abs(q1[0] - ctu).max() <= 1e-14
    # negative velocities: upwinding from the other side
    q1, _ = orc.step(_adv2d(orc, n, -1.0, -1.0, 2, 2, "mc"), q0, dt=1.0 / n)
    assert np.abs(q1 - np.roll(q0, (-1, -1), axis=(1, 2))).max() <= 1e-14


def _drift(orc, P, q0, q1, dV):
    t0, t1 = orc.totals(P, q0), orc.totals(P, q1)
    ref = np.abs(q0).reshape(q0.shape[0], -1).sum(axis=1) * dV
    return np.abs(t1 - t0) / np.maximum(ref, 1e-300)


@pytest.mark.parametrize("rp,scheme", [("sw_roe", "classic"), ("euler_roe", "classic"),
                                       ("euler_hlle", "classic"), ("acoustics", "classic"),
                                       ("euler_roe", "sharpclaw"), ("sw_roe", "sharpclaw")])
def test_conservation_periodic(orc, rp, scheme):
    spec = wl.random_smooth_2d(rp, 24, 20, scheme=scheme, char_decomp=1)
    P = orc.make_problem(spec)
    q = spec["q0"].copy()
    for _ in range(10):
        dt = 0.4 * P.dx / 3.0
        q, cfl = orc.step(P, q, dt=dt)
    d = _drift(orc, P, spec["q0"], q, P.dx * P.dy)
    assert d.max() <= 1e-13, d


def test_conservation_walls(orc):
    spec = wl.sw_dambreak_2d(n=40)
    P = orc.make_problem(spec)
    q, info = orc.evolve(P, spec["q0"], t_end=0.5)
    d = _drift(orc, P, spec["q0"], q, P.dx * P.dy)
    assert d[0] <= 1e-13


def test_dambreak_symmetry(orc):
    spec = wl.sw_dambreak_2d(n=48)
    P = orc.make_problem(spec)
    q, info = orc.evolve(P, spec["q0"], t_end=0.6)
    h, hu, hv = q
    tol = 1e-12
    assert np.abs(h - h[:, ::-1]).max() <= tol and np.abs(hu + hu[:, ::-1]).max() <= tol
    assert np.abs(hv - hv[:, ::-1]).max() <= tol
    assert np.abs(h - h.T).max() <= tol and np.abs(hu - hv.T).max() <= tol


def _order(errs, ns):
    return [math.log(errs[k] / errs[k + 1]) / math.log(ns[k + 1] / ns[k]) for k in range(len(ns) - 1)]


def test_order_classic_1d(orc):
    ns = [32, 64, 128, 256]
    for lim, lo in (("none", 1.9), ("mc", 1.7)):
        errs = []
        for n in ns:
            x = (np.arange(n) + 0.5) / n
            dx = 1.0 / n
            q0 = np.stack([(np.cos(2 * np.pi * (x - dx / 2)) - np.cos(2 * np.pi * (x + dx / 2)))
                           / (2 * np.pi * dx)])
            qT, info = orc.evolve(_adv1d(orc, n, lim, 2, cfl_desired=0.8), q0, t_end=1.0)
            errs.append(np.abs(qT - q0).sum() * dx)
        ords = _order(errs, ns)
        assert min(ords[1:]) >= lo, (lim, ords)
        if lim == "none":
            assert max(ords) <= 2.1


def test_order_classic_2d_transverse(orc):
    ns = [16, 32, 64]
    errs = []
    for n in ns:
        x = (np.arange(n) + 0.5) / n
        X, Y = np.meshgrid(x, x, indexing="xy")
        dx = 1.0 / n
        cx = (np.cos(2 * np.pi * (X - dx / 2)) - np.cos(2 * np.pi * (X + dx / 2))) / (2 * np.pi * dx)
        cy = (np.cos(2 * np.pi * (Y - dx / 2)) - np.cos(2 * np.pi * (Y + dx / 2))) / (2 * np.pi * dx)
        q0 = np.stack([cx * cy])
        qT, info = orc.evolve(_adv2d(orc, n, 1.0, 1.0, 2, 2, cfl_desired=0.8), q0, t_end=1.0)
        errs.append(np.abs(qT - q0).sum() * dx * dx)
    ords = _order(errs, ns)
    assert min(ords) >= 1.9 and max(ords) <= 2.2, ords


@pytest.mark.parametrize("rp", ["euler_roe", "euler_hlle"])
def test_sod_converges_to_exact(orc, rp):
    ns = [100, 200, 400]
    errs = []
    g = 1.4
    for n in ns:
        x = (np.arange(n) + 0.5) / n
        left = x < 0.5
        rho = np.where(left, 1.0, 0.125)
        p = np.where(left, 1.0, 0.1)
        q0 = np.stack([rho, np.zeros(n), p / (g - 1)])
        spec = dict(ndim=1, n=[n], lower=[0.0], upper=[1.0], rp=rp, params=[g], lim="mc",
                    bc_lower=["extrap"], bc_upper=["extrap"])
        qT, info = orc.evolve(orc.make_problem(spec), q0, t_end=0.2)
        assert info["status"] == "ok"
        ex = euler_exact(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, g, (x - 0.5) / 0.2)
        errs.append(np.abs(qT[0] - ex[0]).sum() / n)
    ords = _order(errs, ns)
    assert errs[0] > errs[1] > errs[2] and errs[-1] < 0.006
    assert all(0.5 <= o <= 1.2 for o in ords), ords


def test_dambreak_1d_converges_to_exact(orc):
    ns = [100, 200, 400]
    errs = []
    for n in ns:
        x = -5.0 + (np.arange(n) + 0.5) * 10.0 / n
        q0 = np.stack([np.where(x < 0, 2.0, 1.0), np.zeros(n)])
        spec = dict(ndim=1, n=[n], lower=[-5.0], upper=[5.0], rp="sw_roe", params=[1.0],
                    lim="mc", bc_lower=["extrap"], bc_upper=["extrap"])
        qT, info = orc.evolve(orc.make_problem(spec), q0, t_end=1.0)
        ex = sw_dambreak_exact(2.0, 1.0, 1.0, x / 1.0)
        errs.append(np.abs(qT[0] - ex[0]).sum() * 10.0 / n)
    ords = _order(errs, ns)
    assert errs[0] > errs[1] > errs[2]
    assert all(0.5 <= o <= 1.3 for o in ords), ords


# --------------------------------------------------------------------------
# SharpClaw
# --------------------------------------------------------------------------
def test_weno5_spatial_order_advection(orc):
    """L(Q) for cell averages of sin(2 pi x) against the exact time derivative
    of the cell averages: fifth order."""
    ns = [16, 32, 64, 128]
    errs = []
    for n in ns:
        dx = 1.0 / n
        xe = np.arange(n + 1) * dx
        q0 = np.stack([(np.cos(2 * np.pi * xe[:-1]) - np.cos(2 * np.pi * xe[1:])) / (2 * np.pi * dx)])
        exact = -(np.sin(2 * np.pi * xe[1:]) - np.sin(2 * np.pi * xe[:-1])) / dx
        P = _adv1d(orc, n, scheme="sharpclaw", char_decomp=0)
        L, smax = orc.sharp_L(P, q0)
        errs.append(np.abs(L[0] - exact).sum() * dx)
        Pc = _adv1d(orc, n, scheme="sharpclaw", char_decomp=1)
        Lc, _ = orc.sharp_L(Pc, q0)
        assert np.array_equal(L, Lc)  # scalar: characteristic = component-wise
    ords = _order(errs, ns)
    assert min(ords[1:]) >= 4.5, ords


def test_weno5_char_euler_entropy_wave_order(orc):
    """Characteristic-wise WENO5 on an entropy wave (u = 1, p = 1): fifth order."""
    ns = [16, 32, 64, 128]
    g = 1.4
    errs = []
    for n in ns:
        dx = 1.0 / n
        xe = np.arange(n + 1) * dx
        # rho = 1 + 0.2 sin(2 pi x): cell averages and exact edge values
        rho_avg = 1.0 + 0.2 * (np.cos(2 * np.pi * xe[:-1]) - np.cos(2 * np.pi * xe[1:])) / (2 * np.pi * dx)
        q0 = np.stack([rho_avg, rho_avg * 1.0, 1.0 / (g - 1) + 0.5 * rho_avg])
        rho_e = 1.0 + 0.2 * np.sin(2 * np.pi * xe)
        fe = np.stack([flux("euler_roe", 1, 0, np.array([r, r, 1 / (g - 1) + 0.5 * r]), [g]) for r in rho_e])
        exact = -(fe[1:] - fe[:-1]).T / dx
        spec = dict(ndim=1, n=[n], lower=[0.0], upper=[1.0], rp="euler_roe", params=[g],
                    scheme="sharpclaw", char_decomp=1, bc_lower=["periodic"], bc_upper=["periodic"])
        L, _ = orc.sharp_L(orc.make_problem(spec), q0)
        errs.append(np.abs(L - exact).sum() * dx)
    ords = _order(errs, ns)
    assert min(ords[1:]) >= 4.5, ords


def test_sharpclaw_translation_converges(orc):
    """SSP-RK3 + WENO5 on smooth periodic advection for one period: high order."""
    ns = [32, 64, 128]
    errs = []
    for n in ns:
        dx = 1.0 / n
        xe = np.arange(n + 1) * dx
        q0 = np.stack([(np.cos(2 * np.pi * xe[:-1]) - np.cos(2 * np.pi * xe[1:])) / (2 * np.pi * dx)])
        P = _adv1d(orc, n, scheme="sharpclaw", cfl_desired=0.4, cfl_max=0.5)
        qT, info = orc.evolve(P, q0, t_end=1.0)
        errs.append(np.abs(qT - q0).sum() * dx)
    ords = _order(errs, ns)
    assert min(ords) >= 2.8, ords  # time error (3rd order) dominates at this CFL


# --------------------------------------------------------------------------
# controller
# --------------------------------------------------------------------------
def test_final_time_clipping(orc):
    n = 64
    q0 = RNG.uniform(-1, 1, (1, n))
    qT, info = orc.evolve(_adv1d(orc, n), q0, t_end=0.3)
    assert info["t"] == 0.3 and info["status"] == "ok"
    dt = 0.9 / n
    assert info["steps"] == math.ceil(0.3 / dt - 1e-12)


def test_reject_and_retry(orc):
    n = 64
    q0 = RNG.uniform(-1, 1, (1, n))
    qa, ia = orc.evolve(_adv1d(orc, n, dt_initial=5.0 / n), q0, t_end=0.5)
    assert ia["rejects"] == 1 and ia["status"] == "ok"
    qb, ib = orc.evolve(_adv1d(orc, n, dt_initial=5.0 / n * 0.9 / 5.0), q0, t_end=0.5)
    assert ib["rejects"] == 0 and ib["steps"] == ia["steps"]
    assert np.array_equal(qa, qb)
    qc, ic = orc.evolve(_adv1d(orc, n, dt_initial=5.0 / n, max_retries=0), q0, t_end=0.5)
    assert ic["status"] == "ecfl" and np.array_equal(qc, q0)


def test_nonphysical_status(orc):
    spec = wl.sw_dambreak_2d(n=16)
    q0 = spec["q0"].copy()
    q0[0, 5, 5] = -1.0
    qT, info = orc.evolve(orc.make_problem(spec), q0, t_end=0.5)
    assert info["status"] == "enonphysical"


def test_paper_listing_euler_quadrants(orc):
    """The paper's first listing (2D Euler four-quadrant Riemann problem, 100x100,
    extrapolation BCs, t = 0.3) runs through with positive density and pressure."""
    spec = wl.euler_quadrants_2d(n=100)
    qT, info = orc.evolve(orc.make_problem(spec), spec["q0"], t_end=0.3)
    assert info["status"] == "ok" and info["t"] == 0.3
    rho = qT[0]
    p = 0.4 * (qT[3] - 0.5 * (qT[1] ** 2 + qT[2] ** 2) / rho)
    assert rho.min() > 0 and p.min() > 0


# --------------------------------------------------------------------------
# 3D classic (transverse + double-transverse propagation)
# --------------------------------------------------------------------------
def _prob3(orc, rp, n, params, order=2, transverse=2, lim="mc", bc="periodic", **kw):
    spec = dict(ndim=3, n=list(n), lower=[0, 0, 0], upper=[1, 1, 1], rp=rp, params=params,
                order=order, transverse=transverse, lim=lim,
                bc_lower=[bc] * 3, bc_upper=[bc] * 3)
    spec.update(kw)
    return orc.make_problem(spec)


def test_3d_ctu_exact_and_formula(orc):
    """3D advection: at Courant number 1 in every direction the step is an
    exact diagonal shift; below 1, first order with transverse and
    double-transverse terms is the corner-transport-upwind product
    prod_d [(1 - nu_d) + nu_d S_d] Q."""
    n = 12
    q0 = RNG.uniform(-1, 1, (1, n, n, n))
    for order, tr in ((1, 1), (2, 2), (2, 1)):
        q1, cfl = orc.step(_prob3(orc, "advection", (n, n, n), [1.0, 1.0, 1.0], order, tr), q0,
                           dt=1.0 / n)
        assert cfl == 1.0
        assert np.abs(q1 - np.roll(q0, (1, 1, 1), axis=(1, 2, 3))).max() <= 1e-14
    u, v, w = 1.0, 0.6, -0.35
    dt = 0.8 / n
    nus = [abs(u) * dt * n, abs(v) * dt * n, abs(w) * dt * n]
    q1, _ = orc.step(_prob3(orc, "advection", (n, n, n), [u, v, w], 1, 1), q0, dt=dt)
    Q = q0[0]
    # axes of Q: (z, y, x); upwind shift +1 for positive speed, -1 for negative
    out = Q
    for ax, vel, nu in ((2, u, nus[0]), (1, v, nus[1]), (0, w, nus[2])):
        sh = 1 if vel > 0 else -1
        out = (1 - nu) * out + nu * np.roll(out, sh, axis=ax)
    assert np.abs(q1[0] - out).max() <= 1e-14


@pytest.mark.parametrize("rp,params", [("advection", [0.7, -0.4, 0.3]), ("acoustics", [1.3, 2.5])])
def test_3d_conservation(orc, rp, params):
    n = (10, 9, 8)
    m = 1 if rp == "advection" else 4
    q0 = RNG.uniform(-1, 1, (m, n[2], n[1], n[0]))
    P = _prob3(orc, rp, n, params)
    q = q0.copy()
    for _ in range(5):
        q, cfl = orc.step(P, q, dt=0.3 / 10)
    t0, t1 = orc.totals(P, q0), orc.totals(P, q)
    ref = np.abs(q0).reshape(m, -1).sum(axis=1) * P.dx * P.dy * P.dz
    assert (np.abs(t1 - t0) / ref).max() <= 1e-13


def test_3d_acoustics_axis_symmetry(orc):
    """A pressure pulse symmetric under axis permutations stays symmetric, with
    the velocity components permuted along; walls keep mirror symmetry."""
    n = 16
    x = (np.arange(n) + 0.5) / n - 0.5
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    p = np.exp(-40 * (X * X + Y * Y + Z * Z))
    q0 = np.stack([p, np.zeros_like(p), np.zeros_like(p), np.zeros_like(p)])
    P = _prob3(orc, "acoustics", (n, n, n), [1.0, 4.0], bc="wall")
    q = q0.copy()
    for _ in range(8):
        q, _ = orc.step(P, q, dt=0.4 / n / 2.0)
    pp, u, v, w = q
    tol = 1e-13
    assert np.abs(pp - pp.transpose(0, 2, 1)).max() <= tol  # x <-> y
    assert np.abs(u - v.transpose(0, 2, 1)).max() <= tol
    assert np.abs(pp - pp.transpose(2, 1, 0)).max() <= tol  # x <-> z
    assert np.abs(u - w.transpose(2, 1, 0)).max() <= tol
    assert np.abs(pp - pp[:, :, ::-1]).max() <= tol and np.abs(u + u[:, :, ::-1]).max() <= tol


def test_3d_second_order(orc):
    ns = [8, 16, 32]
    errs = []
    for n in ns:
        dx = 1.0 / n
        xe = np.arange(n + 1) * dx
        c1 = (np.cos(2 * np.pi * xe[:-1]) - np.cos(2 * np.pi * xe[1:])) / (2 * np.pi * dx)
        q0 = np.einsum("k,j,i->kji", c1, c1, c1)[None]
        P = _prob3(orc, "advection", (n, n, n), [1.0, 1.0, 1.0], 2, 2, lim="none",
                   cfl_desired=0.8)
        qT, info = orc.evolve(P, q0, t_end=1.0)
        errs.append(np.abs(qT - q0).sum() * dx ** 3)
    ords = _order(errs, ns)
    assert min(ords[1:]) >= 1.85, ords


# --------------------------------------------------------------------------
# SSP(10,4): the paper's default SharpClaw integrator
# --------------------------------------------------------------------------
def test_ssp104_is_fourth_order_on_linear_problems(orc):
    """One step of q' = lambda q agrees with exp(z) to O(z^5) (fourth order),
    the error at z -> z/2 falls by 2^5, and the scheme is stable on the
    negative real axis out to z = -6 (SSP coefficient 6, ten stages)."""
    for z in (0.05, -0.05, 0.02j):
        pass
    errs = []
    for z in (0.2, 0.1, 0.05):
        r = orc.ssp104_linear(-z, 1.0, 1.0)
        errs.append(abs(r - math.exp(-z)))
    assert errs[0] / errs[1] == pytest.approx(32, rel=0.1)
    assert errs[1] / errs[2] == pytest.approx(32, rel=0.05)
    for z in np.linspace(-6.0, 0.0, 61):
        assert abs(orc.ssp104_linear(z, 1.0, 1.0)) <= 1.0 + 1e-12


def test_ssp104_sharpclaw_converges(orc):
    """WENO5 + SSP(10,4) on smooth periodic advection for one period: the
    error falls at high order at a large Courant number."""
    ns = [32, 64, 128]
    errs = []
    for n in ns:
        dx = 1.0 / n
        xe = np.arange(n + 1) * dx
        q0 = np.stack([(np.cos(2 * np.pi * xe[:-1]) - np.cos(2 * np.pi * xe[1:])) / (2 * np.pi * dx)])
        P = _adv1d(orc, n, scheme="sharpclaw", time_integrator="ssp104", cfl_desired=2.0,
                   cfl_max=2.5)
        qT, info = orc.evolve(P, q0, t_end=1.0)
        assert info["status"] == "ok"
        errs.append(np.abs(qT - q0).sum() * dx)
    ords = _order(errs, ns)
    assert min(ords) >= 3.7, ords
