"""Pins of the Harten-Hyman entropy fix in the oracle's Roe solvers (shallow
water and Euler).  The paper's shallow-water workload uses "a Roe solver with
an entropy fix" (Sec. 5.1, Table 1); the split follows LeVeque's FVM book
(transonic rarefactions).

The fix replaces the Roe wave of a transonic family (speed u - c below zero on
its left state and above zero on its right state) by a left-going and a
right-going part.  Three properties fix it without restating its formula:

* Continuity.  At either edge of the transonic range (one of the two
  characteristic speeds reaching zero) the fixed split must meet the plain Roe
  split that applies beyond the edge, so the fluctuations are continuous
  along any path of states that crosses an edge: their jump over a step of
  size eta in the path parameter shrinks in proportion to eta.  A weight beta
  taken from the wrong end of the fan, or the two speeds exchanged, leaves a
  jump of the size of the wave at one or both edges (planted below).
* Convergence to exact solutions that contain a sonic point: Toro's
  sonic-rarefaction variant of Sod's problem (Euler) and a 10:1 dam break
  whose rarefaction is transonic (shallow water), first and second order.
* No expansion shock.  Without the fix, the first-order Roe scheme keeps a
  stationary jump at the sonic point whose size does not shrink under
  refinement; with it, the largest jump between neighbouring cells around the
  sonic point halves with the cell size.
"""
import math
import os

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
from tests.exact_riemann import euler_exact, sw_dambreak_exact

G_SW = 1.0
GAMMA = 1.4


# --------------------------------------------------------------------------
# states and characteristic speeds, written from the PDEs
# --------------------------------------------------------------------------
def _state(rp, ndim, d, rho, un, ut=0.0):
    """Conserved state with normal velocity un along direction d and tangential
    velocity ut.  Euler states are isentropic: p = rho^gamma / gamma, so the
    sound speed is rho^((gamma - 1) / 2)."""
    vel = np.zeros(ndim)
    vel[d] = un
    if ndim == 2:
        vel[1 - d] = ut
    if rp == "sw_roe":
        return np.concatenate([[rho], rho * vel])
    p = rho ** GAMMA / GAMMA
    return np.concatenate([[rho], rho * vel, [p / (GAMMA - 1) + 0.5 * rho * vel @ vel]])


def _speed(rp, ndim, d, q, last):
    """u_n - c (first family) or u_n + c (last family) of state q."""
    rho = q[0]
    un = q[1 + d] / rho
    if rp == "sw_roe":
        c = math.sqrt(G_SW * rho)
    else:
        ke = 0.5 * sum(q[1 + k] ** 2 for k in range(ndim)) / rho
        c = math.sqrt(GAMMA * (GAMMA - 1) * (q[-1] - ke) / rho)
    return un + c if last else un - c


def _invariant(rp, rho):
    """The part of the Riemann invariant u + 2c/(gamma - 1) (Euler) or u + 2c
    (shallow water) that depends on the state: states on a 1-rarefaction from
    (rho_l, u_l) have u = u_l + inv(rho_l) - inv(rho)."""
    if rp == "sw_roe":
        return 2.0 * math.sqrt(G_SW * rho)
    return 2.0 / (GAMMA - 1) * rho ** ((GAMMA - 1) / 2)


def _mirror(q, d):
    q = q.copy()
    q[1 + d] = -q[1 + d]
    return q


def _path(rp, ndim, d, edge):
    """A path t in [0, 1] of state pairs (ql, qr) along which one speed of the
    transonic test crosses zero.  edge '1r': the first family's right speed
    (u - c of Q_l + W^1) crosses zero with u_l - c_l = -0.5 held below it;
    '1l': u_l - c_l crosses zero with the right speed near +0.8.  The last
    family's edges ('3l', '3r') are the mirror images (x -> -x, left and right
    exchanged).  A tangential velocity rides along in 2D."""
    ut = 0.3 if ndim == 2 else 0.0

    def first(t):
        if edge in ("1r", "3l"):
            rr = 0.9 - 0.6 * t
            ql = _state(rp, ndim, d, 1.0, 0.5, ut)
            qr = _state(rp, ndim, d, rr, 0.5 + _invariant(rp, 1.0) - _invariant(rp, rr), -ut)
        else:
            ul = 1.0 - 0.3 + 0.6 * t  # the left sound speed is 1 for rho = 1
            ql = _state(rp, ndim, d, 1.0, ul, ut)
            qr = _state(rp, ndim, d, 0.5, ul + _invariant(rp, 1.0) - _invariant(rp, 0.5), -ut)
        return ql, qr

    if edge[0] == "1":
        return first
    return lambda t: (_mirror(first(t)[1], d), _mirror(first(t)[0], d))


def _edge_jumps(rp, ndim, d, edge, etas=(1e-3, 1e-4, 1e-5)):
    """Largest change of A^-dQ or A^+dQ over a step of each size eta across the
    edge, and the other speed of the pair at the edge."""
    spec = dict(ndim=ndim, n=[8] * ndim, lower=[0.0] * ndim, upper=[1.0] * ndim, rp=rp,
                params=[G_SW if rp == "sw_roe" else GAMMA], entropy_fix=1)
    P = oracle.make_problem(spec)
    path = _path(rp, ndim, d, edge)

    def speeds(t):
        ql, qr = path(t)
        W = oracle.riemann(P, d, ql, qr)[0]
        if edge[0] == "1":
            return _speed(rp, ndim, d, ql, False), _speed(rp, ndim, d, ql + W[0], False)
        return _speed(rp, ndim, d, qr - W[-1], True), _speed(rp, ndim, d, qr, True)

    k = 1 if edge in ("1r", "3r") else 0  # which speed crosses zero
    t0 = brentq(lambda t: speeds(t)[k], 0.0, 1.0, xtol=1e-15)
    other = speeds(t0)[1 - k]
    jumps = []
    for eta in etas:
        _, _, am_a, ap_a = oracle.riemann(P, d, *path(t0 - eta))
        _, _, am_b, ap_b = oracle.riemann(P, d, *path(t0 + eta))
        jumps.append(max(np.abs(am_a - am_b).max(), np.abs(ap_a - ap_b).max()))
    return jumps, other


EDGE_CASES = [(rp, nd, d, e) for rp in ("sw_roe", "euler_roe") for nd, d in ((1, 0), (2, 0), (2, 1))
              for e in ("1r", "1l", "3r", "3l")]


def _continuous(jumps):
    """Jumps that shrink in proportion to the step: the split is continuous."""
    return jumps[-1] <= 1e-4 and jumps[0] / jumps[-1] >= 50.0


@pytest.mark.parametrize("rp,ndim,d,edge", EDGE_CASES)
def test_entropy_fix_continuous_at_transonic_edges(orc, rp, ndim, d, edge):
    jumps, other = _edge_jumps(rp, ndim, d, edge)
    # the edge is one of the transonic range: the other speed lies on the
    # transonic side (left speed below zero, right speed above)
    assert (other < -0.1) if edge in ("1r", "3r") else (other > 0.1)
    assert _continuous(jumps), jumps


# --------------------------------------------------------------------------
# exact solutions with a sonic point
# --------------------------------------------------------------------------
def _sonic_sod(n, order, entropy_fix=1):
    """Toro's sonic-rarefaction Sod variant: (rho, u, p) = (1, 0.75, 1) left of
    x = 0.3, (0.125, 0, 0.1) right of it, t = 0.2; the left rarefaction
    contains its sonic point (at x = 0.3).  Returns the L1 density error and
    the largest density jump between neighbouring cells around x = 0.3."""
    g = GAMMA
    x = (np.arange(n) + 0.5) / n
    left = x < 0.3
    rho = np.where(left, 1.0, 0.125)
    u = np.where(left, 0.75, 0.0)
    p = np.where(left, 1.0, 0.1)
    q0 = np.stack([rho, rho * u, p / (g - 1) + 0.5 * rho * u * u])
    spec = dict(ndim=1, n=[n], lower=[0.0], upper=[1.0], rp="euler_roe", params=[g], lim="mc",
                order=order, entropy_fix=entropy_fix, bc_lower=["extrap"], bc_upper=["extrap"])
    qT, info = oracle.evolve(oracle.make_problem(spec), q0, t_end=0.2)
    assert info["status"] == "ok"
    ex = euler_exact(1.0, 0.75, 1.0, 0.125, 0.0, 0.1, g, (x - 0.3) / 0.2)
    i0 = int(round(0.3 * n))
    return np.abs(qT[0] - ex[0]).sum() / n, np.abs(np.diff(qT[0][i0 - 3:i0 + 3])).max()


def _dambreak_10(n, order, entropy_fix=1):
    """Dam break h = 10 | 1 at x = 0 on [-5, 5], g = 1, t = 0.5: the middle
    depth is below 4/9 of the left depth, so the rarefaction's tail moves
    right and its sonic point sits at x = 0."""
    x = -5.0 + (np.arange(n) + 0.5) * 10.0 / n
    q0 = np.stack([np.where(x < 0, 10.0, 1.0), np.zeros(n)])
    spec = dict(ndim=1, n=[n], lower=[-5.0], upper=[5.0], rp="sw_roe", params=[G_SW], lim="mc",
                order=order, entropy_fix=entropy_fix, bc_lower=["extrap"], bc_upper=["extrap"])
    qT, info = oracle.evolve(oracle.make_problem(spec), q0, t_end=0.5)
    assert info["status"] == "ok"
    ex = sw_dambreak_exact(10.0, 1.0, G_SW, x / 0.5)
    i0 = n // 2
    return np.abs(qT[0] - ex[0]).sum() * 10.0 / n, np.abs(np.diff(qT[0][i0 - 3:i0 + 3])).max()


def test_dambreak_10_is_transonic():
    """The exact solution of the 10:1 dam break has u - c > 0 in its middle
    state (h_m < 4 h_l / 9), so the fan crosses the sonic point."""
    xi = np.array([0.0, 0.05])
    h, u = sw_dambreak_exact(10.0, 1.0, G_SW, xi)
    assert u[0] - math.sqrt(G_SW * h[0]) == pytest.approx(0.0, abs=1e-12)  # sonic at xi = 0
    ex = sw_dambreak_exact(10.0, 1.0, G_SW, np.linspace(-4, 4, 801))
    hm = ex[0][np.argmin(np.abs(np.linspace(-4, 4, 801) - 1.0))]  # inside the middle state
    assert hm < 4.0 * 10.0 / 9.0


def _order(errs, ns):
    return [math.log(errs[i] / errs[i + 1]) / math.log(ns[i + 1] / ns[i])
            for i in range(len(ns) - 1)]


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("case", ["sonic_sod", "dambreak_10"])
def test_sonic_rarefaction_converges_to_exact(orc, case, order):
    ns = [100, 200, 400, 800]
    run = _sonic_sod if case == "sonic_sod" else _dambreak_10
    errs = [run(n, order)[0] for n in ns]
    ords = _order(errs, ns)
    assert all(errs[i] > errs[i + 1] for i in range(len(ns) - 1)), errs
    assert all(0.5 <= o <= 1.3 for o in ords), ords


@pytest.mark.parametrize("case", ["sonic_sod", "dambreak_10"])
def test_no_expansion_shock_at_sonic_point(orc, case):
    """First order: with the fix the jump at the sonic point halves per
    refinement; without it a stationary expansion shock stays."""
    ns = [100, 200, 400, 800]
    run = _sonic_sod if case == "sonic_sod" else _dambreak_10
    fixed = [run(n, 1, 1)[1] for n in ns]
    plain = [run(n, 1, 0)[1] for n in ns]
    assert all(fixed[i] / fixed[i + 1] >= 1.6 for i in range(len(ns) - 1)), fixed
    assert plain[-1] > 3.0 * fixed[-1] and plain[-2] / plain[-1] < 1.3, plain


# --------------------------------------------------------------------------
# planted mistakes: each must fail the pins above
# --------------------------------------------------------------------------
_BETA_FIRST = "double beta = (lamR - s[0]) / (lamR - lamL);"
_BETA_LAST = "double beta = (lamR - s[last]) / (lamR - lamL);"
_AM_FIRST = "amdq[k] = beta * lamL * W[0 * m + k];"
_AP_LAST = "apdq[k] = (1.0 - beta) * lamR * W[last * m + k];"

PLANTS = {
    # the weight of the left-going part taken from the other end of the fan
    "mirrored_beta": ((_BETA_FIRST, "double beta = (s[0] - lamL) / (lamR - lamL);"),
                      (_BETA_LAST, "double beta = (s[last] - lamL) / (lamR - lamL);")),
    # each part moved at the other edge's speed
    "exchanged_speeds": ((_AM_FIRST, "amdq[k] = beta * lamR * W[0 * m + k];"),
                         (_AP_LAST, "apdq[k] = (1.0 - beta) * lamL * W[last * m + k];")),
}


@pytest.mark.parametrize("plant", sorted(PLANTS))
def test_planted_entropy_fix_mistakes_fail_the_pins(orc, plant, tmp_path):
    src_path = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")
    text = open(src_path).read()
    for old, new in PLANTS[plant]:
        assert text.count(old) == 1, old
        text = text.replace(old, new)
    so = oracle.build_variant(text, str(tmp_path / ("oracle_%s.so" % plant)))
    failed = []
    with oracle.variant(so):
        for rp, ndim, d, edge in EDGE_CASES:
            jumps, _ = _edge_jumps(rp, ndim, d, edge)
            if not _continuous(jumps):
                failed.append((rp, ndim, d, edge))
    # both solvers, both families and both normal directions are caught
    assert {f[0] for f in failed} == {"sw_roe", "euler_roe"}, failed
    assert {f[3][0] for f in failed} == {"1", "3"}, failed
    assert {(f[1], f[2]) for f in failed} == {(1, 0), (2, 0), (2, 1)}, failed
    # the unplanted oracle passes the same checks (the test above), so the
    # variant's failures come from the planted lines alone
