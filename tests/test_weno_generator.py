"""The generator of the GPU's WENO 7..17 reconstructions (csrc/gen_weno.py)
against the oracle's independent derivation (oracle/weno_coeffs.py), exactly
in rational arithmetic: candidate coefficients, optimal weights and
smoothness forms (Sec. 3.3, PyWENO), the emitted sum-of-squares form of each
smoothness indicator (orders 7..13), and the full form's coefficients as
emitted (orders 15, 17).  No GPU needed."""
import importlib.util
import os
from fractions import Fraction

import pytest

from oracle import weno_coeffs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gen():
    path = os.path.join(ROOT, "paper_1111_6583_gb300", "csrc", "gen_weno.py")
    spec = importlib.util.spec_from_file_location("gen_weno", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("r", range(3, 10))
def test_generator_matches_the_oracle_exactly(gen, r):
    c_g, d_g, B_g = gen.derive(r)
    c_o, d_o, B_o = weno_coeffs.weno_coefficients(r)
    assert [list(map(Fraction, row)) for row in c_g] == c_o
    assert list(map(Fraction, d_g)) == d_o
    assert [[list(map(Fraction, row)) for row in Bk] for Bk in B_g] == B_o


@pytest.mark.parametrize("r", range(3, 10))
def test_emitted_sum_of_squares_is_the_smoothness_form(gen, r):
    """beta_k = sum_i D_i (sum_j L[j][i] dv_j)^2 on dv_j = v_j - v_0 equals the
    quadratic form B_k on the differences (B_k annihilates constants)."""
    _, _, B = gen.derive(r)
    for Bk in B:
        L, D = gen.ldl_on_differences(Bk)
        n = r - 1
        for a in range(n):
            for b in range(n):
                s = sum(D[i] * L[a][i] * L[b][i] for i in range(n))
                assert s == Bk[a + 1][b + 1]
        # constants: rows and columns of B_k sum to zero
        for a in range(r):
            assert sum(Bk[a]) == 0


@pytest.mark.parametrize("r", [8, 9])
def test_emitted_tables_are_the_coefficients(gen, r):
    """Orders 15 and 17: the emitted tables hold, entry by entry, the doubles
    nearest the exact candidate coefficients, optimal weights and smoothness
    forms (on the differences, a, b >= 1)."""
    import re
    c, d, B = gen.derive(r)
    text = gen.emit(r)
    o = 2 * r - 1

    def table(name):
        body = text.split("kWeno%d%s" % (o, name))[1].split(";")[0]
        return [float(x) for x in re.findall(r"-?\d[\d.e+-]*", body.split("=")[1])]

    assert table("C") == [float(x) for row in c for x in row]
    assert table("D") == [float(x) for x in d]
    assert table("B") == [float(B[k][a][b]) for k in range(r) for a in range(1, r)
                          for b in range(1, r)]


def test_generated_header_is_current(gen):
    """weno_hi.cuh is what the generator writes today."""
    here = os.path.join(ROOT, "paper_1111_6583_gb300", "csrc")
    assert open(os.path.join(here, "weno_hi.cuh")).read() == gen.render()
