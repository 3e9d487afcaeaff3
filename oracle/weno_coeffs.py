"""WENO coefficients of odd order 2r-1 from their definitions, in exact
rational arithmetic (Sec. 3.3 (PyWENO): reconstruction
coefficients, optimal linear weights and smoothness coefficients computed
symbolically for any order).

TEST INFRASTRUCTURE ONLY (part of the oracle): the tests, the smoke check and
the benchmark's CPU baseline are its only users.

Conventions.  Cells have unit width; cell o covers [o - 1/2, o + 1/2] and the
target cell is o = 0.  The left-biased value at its right edge x = 1/2 is
reconstructed from the 2r-1 averages v[0..2r-2] of cells -(r-1)..(r-1).
Candidate stencil k (k = 0..r-1) is v[k..k+r-1].

  * p_k: the polynomial of degree r-1 whose cell averages over stencil k are
    the data; the reconstruction coefficients c[k][j] give p_k(1/2) =
    sum_j c[k][j] v[k+j].
  * P: the same over all 2r-1 cells (degree 2r-2); the optimal weights d_k
    satisfy sum_k d_k p_k(1/2) = P(1/2) for all data.
  * beta_k = sum_{l=1}^{r-1} dx^(2l-1) int_cell (d^l p_k / dx^l)^2 dx (Jiang-
    Shu smoothness indicator; dx = 1 here, and the expression is invariant
    under the grid scale), a quadratic form B[k] in v[k..k+r-1].
"""
from fractions import Fraction
from functools import lru_cache
from math import factorial


def _solve(A, b):
    """Exact Gaussian elimination (A square, rows of Fractions)."""
    n = len(A)
    M = [list(A[i]) + [b[i]] for i in range(n)]
    for c in range(n):
        p = next(i for i in range(c, n) if M[i][c] != 0)
        M[c], M[p] = M[p], M[c]
        for i in range(n):
            if i != c and M[i][c] != 0:
                f = M[i][c] / M[c][c]
                M[i] = [x - f * y for x, y in zip(M[i], M[c])]
    return [M[i][n] / M[i][i] for i in range(n)]


def _inverse(A):
    n = len(A)
    cols = [_solve(A, [Fraction(int(i == j)) for i in range(n)]) for j in range(n)]
    return [[cols[j][i] for j in range(n)] for i in range(n)]


def _avg_matrix(offsets, deg):
    """M[j][n] = average of x^n over cell offsets[j]."""
    h = Fraction(1, 2)
    return [[((o + h) ** (n + 1) - (o - h) ** (n + 1)) / (n + 1) for n in range(deg + 1)]
            for o in offsets]


def _edge_coeffs(offsets):
    """Coefficients of the interpolant's value at x = 1/2 and the inverse of
    the cell-average matrix (monomial coefficients from the data)."""
    Ainv = _inverse(_avg_matrix(offsets, len(offsets) - 1))
    h = Fraction(1, 2)
    c = [sum(h ** n * Ainv[n][j] for n in range(len(offsets))) for j in range(len(offsets))]
    return c, Ainv


def _int_cell(p):
    """Integral of x^p over [-1/2, 1/2]."""
    return Fraction(0) if p % 2 else Fraction(2, p + 1) * Fraction(1, 2) ** (p + 1)


@lru_cache(maxsize=None)
def weno_coefficients(r):
    """(c, d, B) as Fractions: c[k][j], d[k], B[k][a][b] for 2 <= r <= 9."""
    if not 2 <= r <= 9:
        raise ValueError("r must be in 2..9 (orders 3..17)")
    c, B = [], []
    for k in range(r):
        offs = [-(r - 1) + k + j for j in range(r)]
        ck, Ainv = _edge_coeffs(offs)
        c.append(ck)
        Bk = [[Fraction(0)] * r for _ in range(r)]
        for l in range(1, r):
            for n1 in range(l, r):
                f1 = Fraction(factorial(n1), factorial(n1 - l))
                for n2 in range(l, r):
                    f2 = Fraction(factorial(n2), factorial(n2 - l))
                    w = f1 * f2 * _int_cell(n1 - l + n2 - l)
                    if w == 0:
                        continue
                    for a in range(r):
                        for b in range(r):
                            Bk[a][b] += w * Ainv[n1][a] * Ainv[n2][b]
        B.append(Bk)
    big, _ = _edge_coeffs(list(range(-(r - 1), r)))
    # equations j = 0..r-1 are triangular in d (only stencils k <= j reach v[j])
    d = []
    for j in range(r):
        acc = big[j] - sum(d[k] * c[k][j - k] for k in range(j))
        d.append(acc / c[j][0])
    # the remaining equations must hold too
    for j in range(r, 2 * r - 1):
        s = sum(d[k] * c[k][j - k] for k in range(r) if 0 <= j - k < r)
        if s != big[j]:
            raise ArithmeticError("optimal weights inconsistent at r=%d" % r)
    return c, d, B


def weno_tables(r):
    """The coefficients as floats in the layout the C oracle reads:
    c[k*r + j], d[k], B[(k*r + a)*r + b]."""
    c, d, B = weno_coefficients(r)
    cf = [float(c[k][j]) for k in range(r) for j in range(r)]
    df = [float(x) for x in d]
    bf = [float(B[k][a][b]) for k in range(r) for a in range(r) for b in range(r)]
    return cf, df, bf
