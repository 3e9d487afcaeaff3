"""Pins for the oracle's WENO reconstructions of odd order 2r-1 (Sec. 2.1 and
the PyWENO subsection: reconstruction coefficients, optimal weights and
smoothness coefficients of any order) and for SharpClaw with WENO7/WENO9.

Each pin checks a fact fixed by the mathematics, not the oracle's own
formulas: the published fifth-order coefficients of Jiang and Shu, the
closed form of the optimal weights, exactness on polynomials, the value of
the smoothness indicator on polynomial data, design-order convergence, and
conservation / scalar invariances of the semi-discrete operator.
"""
import math
from fractions import Fraction
from math import comb

import numpy as np
import pytest

import oracle
from oracle.weno_coeffs import weno_coefficients
from paper_1111_6583_gb300 import workloads as wl


def _cell_averages(coef, offsets):
    """Exact cell averages (unit cells centred at the offsets) of the
    polynomial with the given monomial coefficients."""
    P = np.polynomial.Polynomial(coef)
    I = P.integ()
    return np.array([I(o + 0.5) - I(o - 0.5) for o in offsets])


def test_fifth_order_coefficients_are_jiang_shu():
    """r = 3 gives the Jiang-Shu WENO5: candidate values (2a-7b+11c)/6,
    (-b+5c+2d)/6, (2c+5d-e)/6, weights 1/10, 6/10, 3/10 and smoothness
    13/12 (second difference)^2 + 1/4 (one-sided first difference)^2."""
    c, d, B = weno_coefficients(3)
    F = Fraction
    assert c == [[F(2, 6), F(-7, 6), F(11, 6)], [F(-1, 6), F(5, 6), F(2, 6)],
                 [F(2, 6), F(5, 6), F(-1, 6)]]
    assert d == [F(1, 10), F(6, 10), F(3, 10)]
    rng = np.random.default_rng(4)
    for _ in range(20):
        a, b, cc, dd, e = [F(int(x)) for x in rng.integers(-50, 50, 5)]
        beta = [F(13, 12) * (a - 2 * b + cc) ** 2 + F(1, 4) * (a - 4 * b + 3 * cc) ** 2,
                F(13, 12) * (b - 2 * cc + dd) ** 2 + F(1, 4) * (b - dd) ** 2,
                F(13, 12) * (cc - 2 * dd + e) ** 2 + F(1, 4) * (3 * cc - 4 * dd + e) ** 2]
        v = [a, b, cc, dd, e]
        for k in range(3):
            q = sum(B[k][i][j] * v[k + i] * v[k + j] for i in range(3) for j in range(3))
            assert q == beta[k]


def test_generic_order_five_equals_weno5():
    rng = np.random.default_rng(5)
    for scale in (1e-4, 1.0, 1e3):
        for _ in range(20):
            v = rng.normal(size=5) * scale
            assert abs(oracle.weno_r(3, v) - oracle.weno5(v)) <= 1e-14 * np.abs(v).max()


@pytest.mark.parametrize("r", range(2, 10))
def test_optimal_weights_closed_form(r):
    """d_k = C(r, k) C(r-1, k) / C(2r-1, r-1) (stencil 0 leftmost): positive,
    summing to one; r = 4 gives 1/35, 12/35, 18/35, 4/35 (Balsara-Shu)."""
    _, d, _ = weno_coefficients(r)
    want = [Fraction(comb(r, k) * comb(r - 1, k), comb(2 * r - 1, r - 1)) for k in range(r)]
    assert d == want
    assert sum(d) == 1 and all(x > 0 for x in d)
    if r == 4:
        assert d == [Fraction(1, 35), Fraction(12, 35), Fraction(18, 35), Fraction(4, 35)]


@pytest.mark.parametrize("r", range(3, 10))
def test_linear_weights_exact_to_degree_2r_minus_2(r):
    """With the nonlinear weights equal to the optimal ones (epsilon far above
    every smoothness indicator), the reconstruction is the value at the cell
    edge of the degree-(2r-2) polynomial with the given averages."""
    rng = np.random.default_rng(r)
    for _ in range(5):
        coef = rng.normal(size=2 * r - 1) / float(r) ** np.arange(2 * r - 1)
        v = _cell_averages(coef, range(-(r - 1), r))
        exact = np.polynomial.Polynomial(coef)(0.5)
        assert abs(oracle.weno_r(r, v, 1e30) - exact) <= 1e-14 * max(1.0, np.abs(v).max())


@pytest.mark.parametrize("r", range(3, 10))
def test_every_stencil_exact_to_degree_r_minus_1(r):
    """Each candidate is exact for polynomials of degree r-1, so the
    reconstruction is exact for them whatever the nonlinear weights."""
    rng = np.random.default_rng(10 + r)
    for _ in range(5):
        coef = rng.normal(size=r) / float(r) ** np.arange(r)
        v = _cell_averages(coef, range(-(r - 1), r))
        exact = np.polynomial.Polynomial(coef)(0.5)
        for eps in (1e-6, 1e-40):
            assert abs(oracle.weno_r(r, v, eps) - exact) <= 1e-13 * max(1.0, np.abs(v).max())


@pytest.mark.parametrize("r", range(2, 10))
def test_smoothness_indicator_on_polynomial_data(r):
    """For data that are averages of a polynomial f of degree <= r-1, every
    candidate polynomial is f itself, so beta_k = sum_{l=1}^{r-1}
    int_{-1/2}^{1/2} (f^(l))^2 dx for every k; zero for constants."""
    _, _, B = weno_coefficients(r)
    rng = np.random.default_rng(20 + r)
    for _ in range(3):
        coef = rng.normal(size=r) / float(r) ** np.arange(r)
        v = _cell_averages(coef, range(-(r - 1), r))
        f = np.polynomial.Polynomial(coef)
        want = 0.0
        for l in range(1, r):
            g = f.deriv(l) ** 2
            G = g.integ()
            want += G(0.5) - G(-0.5)
        for k in range(r):
            Bk = np.array([[float(x) for x in row] for row in B[k]])
            vk = v[k:k + r]
            # tolerance: rounding of the quadratic form's terms
            assert abs(vk @ Bk @ vk - want) <= 1e-14 * (np.abs(vk) @ np.abs(Bk) @ np.abs(vk))
    vk = np.full(r, 3.7)
    for k in range(r):
        Bk = np.array([[float(x) for x in row] for row in B[k]])
        assert abs(vk @ Bk @ vk) <= 1e-14 * (np.abs(vk) @ np.abs(Bk) @ np.abs(vk))


@pytest.mark.parametrize("r", range(3, 10))
def test_design_order_on_smooth_data(r):
    """Order 2r-1 with the optimal weights; at least 2r-2 with the Jiang-Shu
    weights (epsilon 1e-6) at a point where f' != 0, on these grids.  From
    order 11 on, the grids stay coarse (8 and 16 cells across the unit) so
    that the errors (down to 1e-13) stay above FP64 round-off; there the
    observed order still approaches 2r-1 from below (10.8, 12.7, 14.7, 16.6),
    hence the wider margin."""
    F = lambda x: -np.cos(2 * np.pi * x) / (2 * np.pi) + np.exp(x)
    f = lambda x: np.sin(2 * np.pi * x) + np.exp(x)
    x0 = 0.3
    Ns = (20, 40, 80) if r == 3 else ((10, 20, 40) if r <= 5 else (8, 16))
    margin = 0.1 if r <= 5 else 0.5
    for eps, need in ((1e30, 2 * r - 1 - margin), (1e-6, 2 * r - 2 - 0.5)):
        errs = []
        for N in Ns:
            h = 1.0 / N
            offs = np.arange(-(r - 1), r)
            v = np.array([(F(x0 + (o + 0.5) * h) - F(x0 + (o - 0.5) * h)) / h for o in offs])
            errs.append(abs(oracle.weno_r(r, v, eps) - f(x0 + 0.5 * h)))
        assert math.log2(errs[-2] / errs[-1]) >= need, (eps, errs)


@pytest.mark.parametrize("order", [7, 9, 11, 13])
def test_sharpclaw_operator_order_on_advection(orc, order):
    """Semi-discrete operator of linear advection (u = 1, periodic) on the
    averages of a smooth function: L(Q)_i against the exact
    -(f(x_{i+1/2}) - f(x_{i-1/2}))/dx converges at the WENO order (optimal
    weights, so the design order shows on coarse grids)."""
    errs = []
    Ns = {7: (32, 64), 9: (16, 32), 11: (24, 48), 13: (24, 48)}[order]
    for N in Ns:
        spec = wl.random_1d("advection", N, jump=False, scheme="sharpclaw", char_decomp=0,
                            weno_order=order, weno_eps=1e30, params=[1.0])
        x = (np.arange(N + 1)) / N
        Fx = -np.cos(2 * np.pi * x) / (2 * np.pi) + np.sin(4 * np.pi * x) / (4 * np.pi)
        fx = np.sin(2 * np.pi * x) + np.cos(4 * np.pi * x)
        spec["q0"] = ((Fx[1:] - Fx[:-1]) * N)[None, :].copy()
        P = orc.make_problem(spec)
        L, _ = orc.sharp_L(P, spec["q0"], None)
        exact = -(fx[1:] - fx[:-1]) * N
        errs.append(np.abs(L[0] - exact).max())
    assert math.log2(errs[0] / errs[1]) >= order - 0.3, errs


@pytest.mark.parametrize("order", [5, 7, 9, 11, 13, 15, 17])
def test_sharpclaw_high_order_conserves_and_is_scalar_invariant(orc, order):
    """Periodic 2D Euler: sum of L over the grid vanishes (telescoping
    fluctuations); scalar advection: characteristic- and component-wise
    reconstruction agree."""
    spec = wl.random_smooth_2d("euler_roe", 24, 20, scheme="sharpclaw", char_decomp=1,
                               weno_order=order)
    P = orc.make_problem(spec)
    L, _ = orc.sharp_L(P, spec["q0"], None)
    scale = np.abs(L).max()
    for k in range(L.shape[0]):
        assert abs(L[k].sum()) <= 1e-12 * scale * L[k].size
    sa = wl.random_smooth_2d("advection", 24, 20, scheme="sharpclaw", char_decomp=0,
                             weno_order=order)
    sb = dict(sa, char_decomp=1)
    La, _ = orc.sharp_L(orc.make_problem(sa), sa["q0"], None)
    Lb, _ = orc.sharp_L(orc.make_problem(sb), sb["q0"], None)
    assert np.abs(La - Lb).max() <= 1e-13 * np.abs(La).max()


def test_sharpclaw_weno7_resolves_a_discontinuity_without_overshoot(orc):
    """A square pulse advected one period with WENO7 + SSP(10,4): conserved
    mass, and no over/undershoot beyond a few percent of the jump (the
    nonlinear weights suppress the Gibbs oscillation a linear seventh-order
    scheme would make)."""
    N = 200
    x = (np.arange(N) + 0.5) / N
    q0 = np.where((x > 0.3) & (x < 0.6), 1.0, 0.0)[None, :].copy()
    spec = wl.random_1d("advection", N, jump=False, scheme="sharpclaw", char_decomp=0,
                        weno_order=7, time_integrator="ssp104", cfl_desired=2.0,
                        cfl_max=2.5, params=[1.0])
    spec["q0"] = q0
    P = orc.make_problem(spec)
    q, info = orc.evolve(P, q0, None, t_end=1.0)
    assert info["status"] == "ok" and info["t"] == 1.0
    assert abs(q.sum() - q0.sum()) <= 1e-12 * q0.sum()
    assert q.max() <= 1.05 and q.min() >= -0.05


def _edge_exact(r, v, eps):
    """The WENO edge value of the definitions in exact rational arithmetic, on
    the doubles nearest the exact coefficients (the tables the oracle reads)
    and the double inputs v."""
    c, d, B = weno_coefficients(r)
    V = [Fraction(x) for x in v]
    e = Fraction(eps)
    num, den = Fraction(0), Fraction(0)
    for k in range(r):
        q = sum(Fraction(float(c[k][j])) * V[k + j] for j in range(r))
        beta = sum(Fraction(float(B[k][a][b])) * (V[k + a] - V[k]) * (V[k + b] - V[k])
                   for a in range(r) for b in range(r))
        alpha = Fraction(float(d[k])) / ((e + beta) * (e + beta))
        num += alpha * q
        den += alpha
    return float(num / den)


def _edge_plain(r, v, eps):
    """The same definitions summed plainly in double precision."""
    c, d, B = weno_coefficients(r)
    al, qs = [], []
    for k in range(r):
        q = 0.0
        for j in range(r):
            q += float(c[k][j]) * v[k + j]
        beta = 0.0
        for a in range(r):
            for b in range(r):
                beta += float(B[k][a][b]) * (v[k + a] - v[k]) * (v[k + b] - v[k])
        qs.append(q)
        al.append(float(d[k]) / ((eps + beta) * (eps + beta)))
    s = sum(al)
    return sum((a / s) * q for a, q in zip(al, qs))


@pytest.mark.parametrize("r", [4, 5, 6, 7, 8, 9])
def test_edge_value_is_the_definitions_accurately(r):
    """On smooth data, smooth data with a small jump (intermediate weights), a
    kink and noise, the oracle's edge value equals the exact rational
    evaluation of the definitions on the same doubles to 1e-12 relative (what
    remains is the candidate sums' rounding, a few ulps of sum |c_kj v_j|).
    Plain double sums of the smoothness forms -- terms of size |B| dv^2
    against beta of size dv^2 -- miss by 1e-10 and more at order 17 on the
    same data, which is why the oracle evaluates the forms by error-free
    transformations."""
    rng = np.random.Generator(np.random.PCG64(6583 + r))
    n = 2 * r - 1
    i = np.arange(n)
    families = [
        lambda: np.sin(rng.uniform(0, 6) + i * rng.uniform(0.002, 0.1)) * rng.uniform(0.5, 3.0),
        lambda: (np.sin(rng.uniform(0, 6) + i * rng.uniform(0.01, 0.1)) +
                 np.where(i >= rng.integers(1, n), rng.uniform(1e-4, 1e-2), 0.0)),
        lambda: np.abs(i - rng.uniform(3, n - 3)) * rng.uniform(0.01, 0.1),
        lambda: rng.normal(size=n),
    ]
    worst, worst_plain = 0.0, 0.0
    for t in range(80):
        v = [float(y) for y in families[t % len(families)]()]
        ex = _edge_exact(r, v, 1e-6)
        got = oracle.weno_r(r, np.array(v))
        worst = max(worst, abs(got - ex) / abs(ex))
        worst_plain = max(worst_plain, abs(_edge_plain(r, v, 1e-6) - ex) / abs(ex))
    assert worst <= 1e-12, worst
    if r == 9:
        assert worst_plain > 1e-10, worst_plain
