"""Generate weno_hi.cuh: device WENO reconstructions of odd order 2r-1 > 5
(Sec. 3.3: reconstruction coefficients, optimal
weights and smoothness coefficients derived symbolically for any order, then
emitted as straight-line kernels).

Derivation (exact rationals).  Unit cells, target cell [-1/2, 1/2], value at
its right edge x = 1/2 from the averages v[0..2r-2] of cells -(r-1)..(r-1);
candidate stencil k = v[k..k+r-1].

  * Candidate polynomial p_k = W' where W interpolates the primitive function
    at the r+1 cell edges of the stencil (W at the m-th edge = sum of the
    first m averages), so the weight of v_j in p_k is sum_{m>j} l_m'(x) with
    l_m the Lagrange basis on the edges.
  * Optimal weights d_k: sum_k d_k p_k(1/2) equals the same construction on
    all 2r-1 cells; solved from the rightmost cell inwards.
  * Smoothness beta_k = sum_{l=1}^{r-1} int (p_k^(l))^2 dx, a quadratic form
    that vanishes on constants; on the differences v[k+j] - v[k] (j >= 1) it
    is positive definite and is emitted as sum_i D_i y_i^2 with y = L^T dv
    (exact LDL^T), which keeps the rounding of beta small where the data
    are nearly constant.  Orders 15 and 17 (r = 8, 9) have form coefficients
    in the thousands: there both the form's rounded coefficients and a plain
    sum of its terms carry errors far above beta, so these orders are
    emitted as tables in constant memory (the doubles nearest c, d and B)
    and one out-of-line function per precision that follows the definitions
    step by step -- q_k = sum_j c_kj v_{k+j}; beta_k = sum_a sum_b B_ab dv_a
    dv_b by error-free products and a compensated sum (Ogita, Rump and Oishi,
    "Accurate sum and dot product"); alpha_k = d_k / (eps + beta_k)^2; sum_k
    alpha_k q_k / sum alpha -- each operation rounded once, in that order:
    the value of the definition on those doubles to about one rounding, at a
    cost these rarely used orders can bear.

Run: python gen_weno.py  (rewrites weno_hi.cuh beside this file).
"""
import os
from fractions import Fraction as Fr

ORDERS_R = (4, 5, 6, 7, 8, 9)  # WENO7 .. WENO17
FULL_FORM_R = 8  # from this r on, the full quadratic form (see above)


# --- polynomials as coefficient lists (lowest degree first) ---------------
def padd(a, b):
    n = max(len(a), len(b))
    return [(a[i] if i < len(a) else 0) + (b[i] if i < len(b) else 0) for i in range(n)]


def pmul(a, b):
    out = [Fr(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def pder(a, times=1):
    for _ in range(times):
        a = [i * a[i] for i in range(1, len(a))] or [Fr(0)]
    return a


def peval(a, x):
    return sum(c * x ** i for i, c in enumerate(a))


def pint_cell(a):
    """integral over [-1/2, 1/2]"""
    h = Fr(1, 2)
    return sum(c * (h ** (i + 1) - (-h) ** (i + 1)) / (i + 1) for i, c in enumerate(a))


def lagrange(nodes, m):
    poly = [Fr(1)]
    for i, x in enumerate(nodes):
        if i != m:
            poly = pmul(poly, [-x / (nodes[m] - x), Fr(1) / (nodes[m] - x)])
    return poly


def stencil_polys(first, ncell):
    """weight polynomials P_j(x) of the averages of cells first..first+ncell-1"""
    edges = [Fr(first) - Fr(1, 2) + m for m in range(ncell + 1)]
    dl = [pder(lagrange(edges, m)) for m in range(ncell + 1)]
    polys = []
    for j in range(ncell):
        acc = [Fr(0)]
        for m in range(j + 1, ncell + 1):
            acc = padd(acc, dl[m])
        polys.append(acc)
    return polys


def derive(r):
    half = Fr(1, 2)
    c, B = [], []
    for k in range(r):
        P = stencil_polys(-(r - 1) + k, r)
        c.append([peval(p, half) for p in P])
        Bk = [[Fr(0)] * r for _ in range(r)]
        for a in range(r):
            for b in range(r):
                Bk[a][b] = sum(pint_cell(pmul(pder(P[a], l), pder(P[b], l))) for l in range(1, r))
        B.append(Bk)
    big = [peval(p, half) for p in stencil_polys(-(r - 1), 2 * r - 1)]
    d = [Fr(0)] * r
    for k in range(r - 1, -1, -1):
        j = k + r - 1  # rightmost cell of stencil k; stencils > k already known
        acc = big[j] - sum(d[kk] * c[kk][j - kk] for kk in range(k + 1, r) if j - kk < r)
        d[k] = acc / c[k][r - 1]
    for j in range(2 * r - 1):
        assert sum(d[k] * c[k][j - k] for k in range(r) if 0 <= j - k < r) == big[j]
    assert sum(d) == 1
    return c, d, B


def ldl_on_differences(Bk):
    """beta(v) = dv^T A dv with dv_j = v_j - v_0 (j = 1..r-1), A = B[1:,1:];
    returns (Lcols, D) with beta = sum_i D_i (sum_{j>=i} L[j][i] dv_j)^2."""
    n = len(Bk) - 1
    A = [[Bk[i + 1][j + 1] for j in range(n)] for i in range(n)]
    L = [[Fr(int(i == j)) for j in range(n)] for i in range(n)]
    D = [Fr(0)] * n
    for j in range(n):
        D[j] = A[j][j] - sum(L[j][k] ** 2 * D[k] for k in range(j))
        assert D[j] > 0
        for i in range(j + 1, n):
            L[i][j] = (A[i][j] - sum(L[i][k] * L[j][k] * D[k] for k in range(j))) / D[j]
    return L, D


def lit(x):
    return "R(%s)" % repr(float(x))


def emit_tables(r):
    """orders from FULL_FORM_R on: coefficient tables and the stepwise form"""
    c, d, B = derive(r)
    n = 2 * r - 1
    o = 2 * r - 1
    out = []
    out.append("// WENO%d coefficients: candidates c[k][j], optimal weights d[k], smoothness" % o)
    out.append("// forms B[k][a-1][b-1] on the differences v[k+a] - v[k] (a, b >= 1)")
    out.append("static __constant__ double kWeno%dC[%d][%d] = {" % (o, r, r))
    for k in range(r):
        out.append("    {%s}," % ", ".join(repr(float(x)) for x in c[k]))
    out.append("};")
    out.append("static __constant__ double kWeno%dD[%d] = {%s};"
               % (o, r, ", ".join(repr(float(x)) for x in d)))
    out.append("static __constant__ double kWeno%dB[%d][%d][%d] = {" % (o, r, r - 1, r - 1))
    for k in range(r):
        rows = ["{%s}" % ", ".join(repr(float(B[k][a][b])) for b in range(1, r))
                for a in range(1, r)]
        out.append("    {%s}," % ", ".join(rows))
    out.append("};")
    out.append("// WENO%d: left-biased value at the right edge of the centre cell of" % o)
    out.append("// v[0..%d], stepwise from the definitions (see gen_weno.py)." % (n - 1))
    out.append("template <typename R>")
    out.append("__device__ __noinline__ R weno%d(const R (&v)[%d], R eps) {" % (o, n))
    out.append("  R qk[%d], al[%d];" % (r, r))
    out.append("  R sum = R(0);")
    out.append("#pragma unroll 1")
    out.append("  for (int k = 0; k < %d; ++k) {" % r)
    out.append("    R q = R(0), beta;")
    out.append("    for (int j = 0; j < %d; ++j) q = add_rn(q, mul_rn((R)kWeno%dC[k][j], v[k + j]));"
               % (r, o))
    out.append("    // beta: error-free products and a compensated sum (the zero terms of")
    out.append("    // dv_0 = 0 are left out: they change neither part)")
    out.append("    R hi = R(0), lo = R(0);")
    out.append("    for (int a = 1; a < %d; ++a) {" % r)
    out.append("      const R da = v[k + a] - v[k];")
    out.append("      for (int b = 1; b < %d; ++b) {" % r)
    out.append("        const R db = v[k + b] - v[k];")
    out.append("        const R bab = (R)kWeno%dB[k][a - 1][b - 1];" % o)
    out.append("        const R x = mul_rn(bab, da), xe = fma_rn(bab, da, -x);")
    out.append("        const R y = mul_rn(x, db), ye = fma_rn(x, db, -y);")
    out.append("        const R s = add_rn(hi, y), z = sub_rn(s, hi);")
    out.append("        const R se = add_rn(sub_rn(hi, sub_rn(s, z)), sub_rn(y, z));")
    out.append("        hi = s;")
    out.append("        lo = add_rn(lo, add_rn(add_rn(se, ye), mul_rn(xe, db)));")
    out.append("      }")
    out.append("    }")
    out.append("    beta = add_rn(hi, lo);")
    out.append("    qk[k] = q;")
    out.append("    const R e = add_rn(eps, beta);")
    out.append("    al[k] = (R)kWeno%dD[k] / mul_rn(e, e);" % o)
    out.append("    sum = add_rn(sum, al[k]);")
    out.append("  }")
    out.append("  R out = R(0);")
    out.append("#pragma unroll 1")
    out.append("  for (int k = 0; k < %d; ++k) out = add_rn(out, mul_rn(al[k] / sum, qk[k]));" % r)
    out.append("  return out;")
    out.append("}")
    return "\n".join(out)


def emit(r):
    if r >= FULL_FORM_R:
        return emit_tables(r)
    c, d, B = derive(r)
    n = 2 * r - 1
    out = []
    out.append("// WENO%d: left-biased value at the right edge of the centre cell of" % (2 * r - 1))
    out.append("// v[0..%d]; optimal weights %s." % (n - 1, ", ".join(str(x) for x in d)))
    out.append("template <typename R>")
    out.append("__device__ __forceinline__ R weno%d(const R (&v)[%d], R eps) {" % (2 * r - 1, n))
    for k in range(r):
        terms = " + ".join("%s * v[%d]" % (lit(c[k][j]), k + j) for j in range(r))
        out.append("  const R q%d = %s;" % (k, terms))
    for k in range(r):
        for j in range(1, r):
            out.append("  const R d%d_%d = v[%d] - v[%d];" % (k, j, k + j, k))
        L, D = ldl_on_differences(B[k])
        ys = []
        for i in range(r - 1):
            terms = " + ".join("%s * d%d_%d" % (lit(L[j][i]), k, j + 1) for j in range(i, r - 1)
                               if L[j][i] != 0)
            out.append("  const R y%d_%d = %s;" % (k, i, terms))
            ys.append("%s * (y%d_%d * y%d_%d)" % (lit(D[i]), k, i, k, i))
        out.append("  const R b%d = %s;" % (k, " + ".join(ys)))
    for k in range(r):
        out.append("  const R e%d = eps + b%d;" % (k, k))
        out.append("  const R s%d = e%d * e%d;" % (k, k, k))
    out.append("  if constexpr (sizeof(R) == 8) {")
    out.append("    // alpha_k = d_k / s_k scaled by the product of all s: one division")
    for k in range(r):
        prod = " * ".join("s%d" % j for j in range(r) if j != k)
        out.append("    const R w%d = %s * (%s);" % (k, lit(d[k]), prod))
    num = " + ".join("w%d * q%d" % (k, k) for k in range(r))
    den = " + ".join("w%d" % k for k in range(r))
    out.append("    return FM<R>::div(%s, %s);" % (num, den))
    out.append("  } else {")
    out.append("    // FP32: a product of %d squared indicators can overflow" % (r - 1))
    for k in range(r):
        out.append("    const R w%d = FM<R>::div(%s, s%d);" % (k, lit(d[k]), k))
    out.append("    return FM<R>::div(%s, %s);" % (num, den))
    out.append("  }")
    out.append("}")
    return "\n".join(out)


def render():
    """the text of weno_hi.cuh"""
    parts = ["// weno_hi.cuh -- generated by gen_weno.py from exact rational derivations;",
             "// do not edit.  Higher-order WENO reconstructions (Sec. 3.3, PyWENO",
             "// subsection) used by the SharpClaw stage kernel.",
             "#pragma once", "", '#include "riemann.cuh"', "", "namespace claw {", "",
             "// operations rounded once each (never fused or reordered)",
             "__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }",
             "__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }",
             "__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }",
             "__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }",
             "__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }",
             "__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }",
             "__device__ __forceinline__ double fma_rn(double a, double b, double c) {",
             "  return __fma_rn(a, b, c);",
             "}",
             "__device__ __forceinline__ float fma_rn(float a, float b, float c) {",
             "  return __fmaf_rn(a, b, c);",
             "}",
             ""]
    for r in ORDERS_R:
        parts.append(emit(r))
        parts.append("")
    parts.append("}  // namespace claw")
    return "\n".join(parts) + "\n"


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "weno_hi.cuh"), "w") as f:
        f.write(render())


if __name__ == "__main__":
    main()
