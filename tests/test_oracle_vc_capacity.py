"""Pins for the oracle's acoustics in a varying medium and the capacity
function kappa of Eq. (conslaw) (capacity-form differencing).

Pinned by facts outside the oracle's formulas: the waves sum to the jump and
are the eigenvectors (-Z, 1) / (Z, 1) of the two media; a uniform medium
reduces every scheme to the constant-coefficient acoustics solver (itself
pinned); the transmission and reflection coefficients at an impedance jump;
a uniform capacity k equals the same grid stretched by k; and the capacity-
weighted totals sum_i kappa_i Q_i are conserved.
"""
import numpy as np
import pytest

import oracle
from paper_1111_6583_gb300 import workloads as wl


@pytest.mark.parametrize("ndim,d", [(1, 0), (2, 0), (2, 1)])
def test_vc_waves_are_eigenvectors_and_sum_to_jump(ndim, d):
    spec = (wl.random_1d("acoustics_vc", 8) if ndim == 1
            else wl.random_smooth_2d("acoustics_vc", 8, 8))
    P = oracle.make_problem(spec)
    m = P.num_eqn
    n = 1 + d
    rng = np.random.default_rng(5 + d)
    for _ in range(30):
        ql, qr = rng.normal(size=m), rng.normal(size=m)
        al = np.array([rng.uniform(0.5, 4), rng.uniform(0.3, 2), 1.0])
        ar = np.array([rng.uniform(0.5, 4), rng.uniform(0.3, 2), 1.0])
        W, s, am, ap = oracle.riemann(P, d, ql, qr, al, ar)
        # the two acoustic waves carry the jumps of p and the normal velocity
        # (the tangential jump sits in a zero-speed wave that is not formed)
        dq = (qr - ql)[[0, n]]
        assert np.allclose(W.sum(axis=0)[[0, n]], dq, rtol=0, atol=1e-14 * (1 + np.abs(dq).max()))
        Zl, Zr = al[0] * al[1], ar[0] * ar[1]
        assert s[0] == -al[1] and s[1] == ar[1]
        assert abs(W[0][0] + Zl * W[0][n]) <= 1e-14 * (1 + abs(W[0][0]))
        assert abs(W[1][0] - Zr * W[1][n]) <= 1e-14 * (1 + abs(W[1][0]))
        if ndim == 2:
            assert W[0][2 - d] == 0.0 and W[1][2 - d] == 0.0
        assert np.allclose(am, s[0] * W[0]) and np.allclose(ap, s[1] * W[1])


def _uniform_pair(ndim, scheme, **kw):
    """The same problem as varying-medium acoustics with uniform (rho, c) and
    as constant-coefficient acoustics (K = rho c^2)."""
    rho, c = 1.7, 0.8
    if ndim == 1:
        sv = wl.random_1d("acoustics_vc", 120, jump=True, scheme=scheme, num_aux=2, **kw)
        sc = wl.random_1d("acoustics", 120, jump=True, scheme=scheme, params=[rho, rho * c * c],
                          **kw)
    else:
        sv = wl.random_smooth_2d("acoustics_vc", 48, 36, scheme=scheme, num_aux=2, **kw)
        sc = wl.random_smooth_2d("acoustics", 48, 36, scheme=scheme, params=[rho, rho * c * c],
                                 **kw)
    sv["q0"] = sc["q0"].copy()
    shape = sc["q0"].shape[1:]
    sv["aux"] = np.stack([np.full(shape, rho), np.full(shape, c)])
    return sv, sc


@pytest.mark.parametrize("ndim,scheme,transverse",
                         [(1, "classic", 0), (2, "classic", 2), (2, "classic", 1),
                          (1, "sharpclaw", 0), (2, "sharpclaw", 0)])
def test_uniform_medium_is_constant_acoustics(ndim, scheme, transverse):
    kw = {"transverse": transverse} if ndim == 2 else {}
    sv, sc = _uniform_pair(ndim, scheme, **kw)
    Pv, Pc = oracle.make_problem(sv), oracle.make_problem(sc)
    qv, qc = sv["q0"], sc["q0"]
    dt = 0.4 / sv["n"][0]
    for _ in range(4):
        qv, cv = oracle.step(Pv, qv, sv["aux"], dt)
        qc, cc = oracle.step(Pc, qc, None, dt)
    assert np.abs(qv - qc).max() <= 1e-13 * np.abs(qc).max()
    assert abs(cv - cc) <= 1e-14 * cc


def test_transmission_and_reflection_at_an_impedance_jump():
    """A right-going pressure pulse meets the interface between (rho, c) =
    (1, 1) and (4, 0.5): the transmitted and reflected pressure amplitudes
    are 2 Z_r/(Z_l + Z_r) and (Z_r - Z_l)/(Z_l + Z_r) of the incident one."""
    n = 3000
    x = (np.arange(n) + 0.5) / n * 2.0 - 1.0
    rho = np.where(x < 0.0, 1.0, 4.0)
    c = np.where(x < 0.0, 1.0, 0.5)
    p = np.exp(-400 * (x + 0.5) ** 2)
    q0 = np.stack([p, p / 1.0])  # right-going in the left medium: u = p / Z_l
    spec = wl.random_1d("acoustics_vc", n, num_aux=2, bc=("extrap", "extrap"))
    spec.update(q0=q0, aux=np.stack([rho, c]), lower=[-1.0], upper=[1.0])
    q, info = oracle.evolve(oracle.make_problem(spec), q0, spec["aux"], t_end=0.8)
    assert info["status"] == "ok"
    Zl, Zr = 1.0, 2.0
    left = q[0][x < 0.0]
    right = q[0][x > 0.0]
    T = right.max()
    Rf = left.max() if abs(left.max()) > abs(left.min()) else left.min()
    assert abs(T - 2 * Zr / (Zl + Zr)) < 0.02
    assert abs(Rf - (Zr - Zl) / (Zl + Zr)) < 0.02


@pytest.mark.parametrize("ndim,scheme,split", [(1, "classic", 0), (2, "classic", 0),
                                               (2, "classic", 1), (1, "sharpclaw", 0),
                                               (2, "sharpclaw", 0)])
def test_uniform_capacity_is_a_stretched_grid(ndim, scheme, split):
    """kappa q_t + f(q)_x = 0 with kappa = k everywhere is the problem on a
    grid k times wider: same states, same Courant numbers (unsplit, and with
    dimensional splitting)."""
    k = 1.6
    if ndim == 1:
        s1 = wl.random_1d("sw_roe", 96, scheme=scheme, char_decomp=0)
        s1.update(num_aux=1, capa_index=0, aux=np.full((1, 96), k))
        s2 = wl.random_1d("sw_roe", 96, scheme=scheme, char_decomp=0)
        s2["upper"] = [k]
    else:
        kw = {"dim_split": 1, "transverse": 0} if split else {}
        s1 = wl.random_smooth_2d("sw_roe", 40, 30, scheme=scheme, char_decomp=0, **kw)
        s1.update(num_aux=1, capa_index=0, aux=np.full((1, 30, 40), k))
        s2 = wl.random_smooth_2d("sw_roe", 40, 30, scheme=scheme, char_decomp=0, **kw)
        s2["upper"] = [k, k]
    P1, P2 = oracle.make_problem(s1), oracle.make_problem(s2)
    q1, q2 = s1["q0"], s2["q0"]
    dt = 0.3 / s1["n"][0]
    for _ in range(3):
        q1, c1 = oracle.step(P1, q1, s1["aux"], dt)
        q2, c2 = oracle.step(P2, q2, None, dt)
    assert np.abs(q1 - q2).max() <= 1e-13 * np.abs(q2).max()
    assert abs(c1 - c2) <= 1e-14 * c2


@pytest.mark.parametrize("ndim,scheme", [(1, "classic"), (2, "classic"), (1, "sharpclaw"),
                                         (2, "sharpclaw")])
def test_capacity_weighted_totals_are_conserved(ndim, scheme):
    """Shallow water (a conservation law; the varying-medium acoustics system
    is not in conservation form) with a varying capacity, periodic."""
    if ndim == 1:
        spec = wl.random_1d("sw_roe", 150, scheme=scheme, char_decomp=0)
        x = (np.arange(150) + 0.5) / 150
        kap = (1.0 + 0.4 * np.sin(2 * np.pi * x))[None]
    else:
        spec = wl.random_smooth_2d("sw_roe", 48, 36, scheme=scheme, char_decomp=0)
        X, Y = np.meshgrid((np.arange(48) + 0.5) / 48, (np.arange(36) + 0.5) / 36, indexing="xy")
        kap = (1.0 + 0.4 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y))[None]
    spec.update(num_aux=1, capa_index=0, aux=np.ascontiguousarray(kap))
    P = oracle.make_problem(spec)
    kap = spec["aux"][0]
    q = spec["q0"]
    t0 = (q * kap).reshape(q.shape[0], -1).sum(axis=1)
    for _ in range(4):
        q, _ = oracle.step(P, q, spec["aux"], 0.3 / spec["n"][0])
    t1 = (q * kap).reshape(q.shape[0], -1).sum(axis=1)
    assert np.abs(t1 - t0).max() <= 1e-12 * np.abs(q * kap).sum()



@pytest.mark.parametrize("d", [0, 1])
def test_vc_transverse_split_is_the_neighbour_riemann_solution(d):
    """B^- a is (speed -c_below) times the down-going wave of the transverse
    Riemann problem between the cell below and the cell holding a (the jump
    a split into (-Z_below, 1) and (Z_cell, 1) in (p, v_t)); B^+ a likewise
    with the cell above and the up-going (Z_above, 1) wave."""
    spec = wl.random_smooth_2d("acoustics_vc", 8, 8)
    P = oracle.make_problem(spec)
    t = 2 - d
    rng = np.random.default_rng(11 + d)
    for _ in range(20):
        am_, ac_, ap_ = ([rng.uniform(0.5, 3), rng.uniform(0.3, 2), 1.0] for _ in range(3))
        a = rng.normal(size=3)
        bm, bp = oracle.transverse_vc(P, d, np.array(am_), np.array(ac_), np.array(ap_), a)
        Zm, Zc, Zp = am_[0] * am_[1], ac_[0] * ac_[1], ap_[0] * ap_[1]
        # decomposition solved here by a linear solve, not the oracle's formula
        wd = np.linalg.solve(np.array([[-Zm, Zc], [1.0, 1.0]]), [a[0], a[t]])
        wu = np.linalg.solve(np.array([[-Zc, Zp], [1.0, 1.0]]), [a[0], a[t]])
        down = -am_[1] * wd[0] * np.array([-Zm, 1.0])
        up = ap_[1] * wu[1] * np.array([Zp, 1.0])
        assert np.allclose(bm[[0, t]], down, rtol=1e-13, atol=1e-14)
        assert np.allclose(bp[[0, t]], up, rtol=1e-13, atol=1e-14)
        assert bm[1 + d] == 0.0 and bp[1 + d] == 0.0


def test_vc_order_uniform_versus_smooth_medium():
    """Measured property of the wave form with cell-centred coefficients
    (recorded, not a correctness criterion): Lax-Wendroff waves converge at
    second order in a uniform medium and at first order in a smoothly varying
    one (the f-wave elasticity solver stays second order there)."""
    def run(n, vary):
        sp = wl.random_1d("acoustics_vc", n, num_aux=2, jump=False, lim="none")
        x = (np.arange(n) + 0.5) / n
        if vary:
            rho, c = 1.0 + 0.5 * np.sin(2 * np.pi * x), 1.0 + 0.3 * np.cos(2 * np.pi * x)
        else:
            rho, c = np.full(n, 1.3), np.full(n, 0.9)
        p = np.exp(-30 * (x - 0.5) ** 2)
        sp.update(q0=np.stack([p, 0 * p]), aux=np.stack([rho, c]))
        P = oracle.make_problem(sp)
        q = sp["q0"]
        for _ in range(n // 3):
            q, _ = oracle.step(P, q, sp["aux"], 0.4 / n)
        return q

    def ratio(vary):
        s = {n: run(n, vary) for n in (96, 192, 384)}
        co = lambda q: 0.5 * (q[:, 0::2] + q[:, 1::2])
        return (np.abs(s[96] - co(s[192])).mean() / np.abs(s[192] - co(s[384])).mean())
    assert ratio(False) > 3.7
    assert 1.7 < ratio(True) < 2.4
