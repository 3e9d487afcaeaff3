"""The generator of the GPU's WENO 7..13 reconstructions (csrc/gen_weno.py)
against the oracle's independent derivation (oracle/weno_coeffs.py), exactly
in rational arithmetic: candidate coefficients, optimal weights and
smoothness forms (Sec. 3.3, PyWENO), and the emitted sum-of-squares
form of each smoothness indicator.  No GPU needed."""
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


def test_generated_header_is_current(gen):
    """weno_hi.cuh is what the generator writes today."""
    here = os.path.join(ROOT, "paper_1111_6583_gb300", "csrc")
    assert open(os.path.join(here, "weno_hi.cuh")).read() == gen.render()
