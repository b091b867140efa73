"""Generate dg_tables.cuh: compile-time Gauss–Legendre rules and Legendre values for the kernels.

Nodes are the roots of P_n found by sympy at 40 digits (real_roots of the exact polynomial), weights
w = 2 / ((1 - x^2) P_n'(x)^2); tabulated values are P_l(x_q) and P_l'(x_q) for l <= 3, rounded once
to double. Run: python gen_tables.py > dg_tables.cuh (the committed header is this script's output).
"""
import sympy as sp

X = sp.Symbol("x")
LMAX = 3
RULES = range(1, 9)  # 1..8 points: k+1 for the scheme, up to k+5 for projections


def fmt(v):
    f = float(sp.N(v, 40))
    return repr(0.0 if abs(f) < 1e-30 else f)   # exact zeros come back as ~1e-41 from nroots


def main():
    out = []
    out.append("// Generated by gen_tables.py: Gauss–Legendre rules on [-1,1] and Legendre values at the nodes.")
    out.append("// Do not edit by hand.")
    out.append("#pragma once")
    out.append("#include <cuda_runtime.h>")
    out.append("namespace dgk {")
    out.append("template <int N> struct GaussRule;")
    for n in RULES:
        Pn = sp.legendre(n, X)
        dPn = sp.diff(Pn, X)
        roots = sorted(sp.Poly(Pn, X).nroots(n=40))
        xs = [sp.re(r) for r in roots]
        ws = [2 / ((1 - r ** 2) * dPn.subs(X, r) ** 2) for r in xs]
        P = [[sp.legendre(l, X).subs(X, r) for r in xs] for l in range(LMAX + 4)]
        dP = [[sp.diff(sp.legendre(l, X), X).subs(X, r) for r in xs] for l in range(LMAX + 4)]
        hd = "  __host__ __device__ static constexpr double "
        out.append("template <> struct GaussRule<%d> {" % n)
        out.append("  static constexpr int n = %d;" % n)
        out.append(hd + "x(int i) { constexpr double a[%d] = {%s}; return a[i]; }" % (
            n, ", ".join(fmt(v) for v in xs)))
        out.append(hd + "w(int i) { constexpr double a[%d] = {%s}; return a[i]; }" % (
            n, ", ".join(fmt(v) for v in ws)))
        out.append("  // P(l, q) = P_l(x_q), dP(l, q) = P_l'(x_q), l = 0..%d" % (LMAX + 3))
        out.append(hd + "P(int l, int i) {\n    constexpr double a[%d][%d] = {%s};\n    return a[l][i];\n  }" % (
            LMAX + 4, n, ", ".join("{" + ", ".join(fmt(v) for v in row) + "}" for row in P)))
        out.append(hd + "dP(int l, int i) {\n    constexpr double a[%d][%d] = {%s};\n    return a[l][i];\n  }" % (
            LMAX + 4, n, ", ".join("{" + ", ".join(fmt(v) for v in row) + "}" for row in dP)))
        out.append("};")
    out.append("}  // namespace dgk")
    print("\n".join(out))


if __name__ == "__main__":
    main()
