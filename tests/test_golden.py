"""Checks against the cited fixtures under tests/golden/: values the paper
prints (the shock-bubble post-shock state of Sec. 7.2, the checkerboard rule
of Sec. 7.3) and Toro's tabulated star state of Sod's problem, which pins the
exact Riemann solver that the oracle's Sod convergence pins compare with.
"""
import os

import numpy as np
import pytest

from paper_1111_6583_gb300 import workloads as wl
from tests.exact_riemann import euler_exact

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _kv(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = (t.strip() for t in line.split("=", 1))
            out[k] = float(v)
    return out


def test_shock_bubble_post_shock_state():
    g = _kv("shock_bubble_post_shock.txt")
    rho, u, p = wl.post_shock_state_from_pressure(g["p_behind"], g["gamma"], g["rho_ahead"],
                                                  g["p_ahead"])
    assert p == pytest.approx(g["p_behind"], rel=1e-14)
    assert abs(rho - g["rho_behind"]) <= g["tol"]
    assert abs(u - g["u_behind"]) <= g["tol"]
    # the axisymmetric workload carries that state behind the shock and at inflow
    spec = wl.shock_bubble_axisym(nx=64, ny=16, sub=2)
    assert spec["q0"][0, 0, 0] == pytest.approx(rho, rel=1e-14)
    assert spec["q0"][1, 0, 0] == pytest.approx(rho * u, rel=1e-14)
    assert spec["inflow"][0] == pytest.approx(rho, rel=1e-14)


def test_checkerboard_medium_points():
    rows = np.loadtxt(os.path.join(GOLDEN, "checkerboard_points.txt"))
    rho, K = wl.checkerboard_medium(rows[:, 0], rows[:, 1])
    assert np.array_equal(K, rows[:, 2]) and np.array_equal(rho, rows[:, 3])


def test_exact_sod_star_state_matches_toro():
    s = _kv("sod_star_state.txt")
    # sample the left and right star regions (between the rarefaction tail
    # and the contact, and between the contact and the shock)
    out = euler_exact(s["rho_l"], s["u_l"], s["p_l"], s["rho_r"], s["u_r"], s["p_r"],
                      s["gamma"], np.array([0.5, 1.3]))
    tol = s["tol"]
    assert abs(out[2, 0] - s["p_star"]) <= tol and abs(out[2, 1] - s["p_star"]) <= tol
    assert abs(out[1, 0] - s["u_star"]) <= tol and abs(out[1, 1] - s["u_star"]) <= tol
    assert abs(out[0, 0] - s["rho_star_l"]) <= tol
    assert abs(out[0, 1] - s["rho_star_r"]) <= tol
