"""The closed forms the FP64 kernels use for the limited wave strength of the
constant-coefficient solvers (advection, constant-medium acoustics): with
theta = u / a (u the upwind strength, a the wave's own), phi(theta) a equals
sgn(a) g(|u|, |a|) for same-signed u and a and 0 otherwise, where g is

    minmod    min(|u|, |a|)
    superbee  max(min(2|u|, |a|), min(|u|, 2|a|))
    MC        min(|a + u| / 2, 2|a|, 2|u|)
    van Leer  2 |u| |a| / (|u| + |a|)

and "none" gives a.  Checked here against a times the oracle's phi (the
limiter functions of Eq. (lwflux)'s limited waves) on random strengths over
six decades, on the breakpoints of each limiter (theta = 1/3, 1/2, 1, 2, 3),
and on zero strengths, so that a wrong constant, a swapped argument or a
lost sign fails."""
import numpy as np
import pytest

import oracle

LIMS = ["minmod", "superbee", "mc", "vanleer", "none"]


def closed_form(lim, u, a):
    if lim == "none":
        return a
    same = (u > 0 and a > 0) or (u < 0 and a < 0)
    au, aa = abs(u), abs(a)
    if lim == "minmod":
        g = min(au, aa)
    elif lim == "superbee":
        g = max(min(2 * au, aa), min(au, 2 * aa))
    elif lim == "vanleer":
        g = 2 * au * aa / (au + aa) if same else 0.0
    else:
        g = min(0.5 * abs(a + u), min(2 * aa, 2 * au))
    g = g if same else 0.0
    return -g if a < 0 else g


def reference(lim, u, a):
    # a zero wave gets no correction (the oracle's zero-norm rule)
    if a == 0.0:
        return 0.0
    return a * oracle.phi(lim, u / a)


@pytest.mark.parametrize("lim", LIMS)
def test_random_strengths(lim):
    rng = np.random.Generator(np.random.PCG64(6583))
    for _ in range(4000):
        a = rng.normal() * 10.0 ** rng.uniform(-3, 3)
        u = rng.normal() * 10.0 ** rng.uniform(-3, 3)
        ref = reference(lim, u, a)
        got = closed_form(lim, u, a)
        assert abs(got - ref) <= 4e-16 * max(abs(ref), abs(a)), (lim, u, a, got, ref)


@pytest.mark.parametrize("lim", LIMS)
@pytest.mark.parametrize("theta", [1 / 3, 0.5, 1.0, 2.0, 3.0, 0.0, -1.0, -0.25])
@pytest.mark.parametrize("a", [1.7, -0.6])
def test_breakpoints_and_signs(lim, theta, a):
    u = theta * a
    ref = reference(lim, u, a)
    got = closed_form(lim, u, a)
    assert abs(got - ref) <= 4e-16 * abs(a), (lim, theta, a, got, ref)


@pytest.mark.parametrize("lim", LIMS)
def test_zero_strengths(lim):
    assert closed_form(lim, 0.0, 0.0) == 0.0
    assert closed_form(lim, 1.3, 0.0) == 0.0
    assert closed_form(lim, 0.0, -2.0) == (-2.0 if lim == "none" else 0.0)
