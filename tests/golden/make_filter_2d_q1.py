"""Write filter_2d_q1.txt: the jump-filter damping of one 2D Euler Q1 cell, derived with sympy.

The example: a 3x3 mesh of square cells, h_x = h_y = 1/10, outflow boundaries. Every cell holds
the constant state (rho, m_x, m_y, E) = (1, 0, 0, 5/2) except the centre cell, whose density is
rho = 1 + xi/10 + eta/20 + xi*eta/50 on the reference cell. Only the density jumps.

From the paper: Eq. (para:damp22d)-(para:damp22d1) with (c_fx, c_fy) = (h_y beta^x, h_x beta^y) /
(4 lambda_{p,q} Hbar) (Section 3.2), edge norms by the trapezoidal rule over each edge's two corners
(Section 2.2), derivatives in physical coordinates, beta = |u| + c and Hbar = (E + p)/rho at the
cell average. Nothing here calls the oracle: the corner derivatives come from sympy's symbolic
differentiation of the polynomial written in physical coordinates.
"""
import os

import sympy as sp

x, y = sp.symbols("x y")
h = sp.Rational(1, 10)
xi, eta = 2 * x / h, 2 * y / h                      # centre cell occupies [-h/2, h/2]^2
rho_c = 1 + xi / 10 + eta / 20 + xi * eta / 50
rho_n = sp.Integer(1)                              # every neighbour is constant
gamma = sp.Rational(7, 5)
p_avg = (gamma - 1) * sp.Rational(5, 2)            # momentum zero
c = sp.sqrt(gamma * p_avg / 1)
beta = c                                           # |u| + c with u = 0, both directions
Hbar = (sp.Rational(5, 2) + p_avg) / 1


def d(expr, a1, a2):
    return sp.diff(expr, x, a1, y, a2) if (a1 or a2) else expr


def edge_jump(a1, a2, vertical):
    """(1/|e|) int over the cell's two edges of |[d^alpha rho]|, trapezoidal rule (two corners)."""
    s = 0
    for side in (-1, 1):
        for corner in (-1, 1):
            px, py = (side * h / 2, corner * h / 2) if vertical else (corner * h / 2, side * h / 2)
            own = d(rho_c, a1, a2).subs({x: px, y: py})
            nb = d(rho_n, a1, a2)                  # neighbour's value at the same point
            s += sp.Rational(1, 2) * sp.Abs(own - nb)
    return sp.nsimplify(s)


k = 1
lines = []
for (pp, qq) in [(1, 0), (0, 1), (1, 1)]:
    l = pp + qq
    lam = pp * (pp + 1) + qq * (qq + 1)
    cfx = h * beta / (4 * lam * Hbar)
    cfy = h * beta / (4 * lam * Hbar)
    sx = h * edge_jump(0, 0, True)
    sy = h * edge_jump(0, 0, False)
    for m in range(1, l + 1):
        tv = sum(edge_jump(a1, m - a1, True) for a1 in range(0, m + 1) if a1 <= k and m - a1 <= k)
        th = sum(edge_jump(a1, m - a1, False) for a1 in range(0, m + 1) if a1 <= k and m - a1 <= k)
        sx += m * (m + 1) * h ** (m + 1) * tv
        sy += m * (m + 1) * h ** (m + 1) * th
    sigma_l = cfx * sx + cfy * sy
    sigma = sp.simplify(sigma_l * (2 / h) * (2 / h) * lam)
    lines.append("%d %d %s %.17g" % (pp, qq, sigma, float(sigma)))

out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "filter_2d_q1.txt")
with open(out, "w") as f:
    f.write("# p q sigma^{p,q} (exact) sigma^{p,q} (float); generated by make_filter_2d_q1.py\n")
    f.write("# 2D Euler Q1, 3x3 outflow mesh, h=1/10, centre rho = 1 + xi/10 + eta/20 + xi*eta/50\n")
    f.write("# Eqs. (para:damp22d)-(para:damp22d1), Section 3.2 (c_fx, c_fy), trapezoidal edge norms\n")
    f.write("\n".join(lines) + "\n")
print(open(out).read())
