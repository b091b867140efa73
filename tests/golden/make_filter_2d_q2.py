"""Write filter_2d_q2.txt: the jump-filter damping of every mode of one 2D Euler Q2 cell, derived
with sympy from the paper's formulas (no oracle code is used).

The example: a 3x3 mesh of rectangular cells, h_x = 1/10, h_y = 1/16 (so h_x != h_y and the two
c_f factors differ), outflow boundaries. Only the centre cell and its four face neighbours enter
the centre cell's damping. Every one of these five cells holds its own Q2 polynomial in all four
conservative variables (rho, m_x, m_y, E): the neighbours are not constant, density and energy
jump across every edge, the mixed modes (2,1), (1,2), (2,2) are non-zero, and the centre cell's
average velocity is non-zero in both directions (beta^x != beta^y).

From the paper, Section 2.2 and Section 3.2:
  sigma^{p,q}    = sigma_{l} (2/h_x) (2/h_y) lambda_{p,q},  lambda_{p,q} = p(p+1) + q(q+1),
                   l = p + q                                          (Eq. para:damp22d)
  sigma_{l}      = c_fx (h_x ||[u]||_V + sum_{m=1..l} m(m+1) h_x^{m+1} sum_{|a|=m} ||[d^a u]||_V)
                 + c_fy (h_y ||[u]||_H + sum_{m=1..l} m(m+1) h_y^{m+1} sum_{|a|=m} ||[d^a u]||_H)
                                                                      (Eq. para:damp22d1)
  (c_fx, c_fy)   = (h_y beta^x, h_x beta^y) / (4 lambda_{p,q} Hbar)   (Section 3.2, Euler)
  ||[w]||_V      = (1/h_y) int over the left and right edges of |jump of w|, by the trapezoidal
                   rule over each edge's two corners (Section 2.2), physical derivatives
  beta^x = |u_bar| + c_bar, beta^y = |v_bar| + c_bar, Hbar = (E_bar + p_bar)/rho_bar at the centre
  cell's average; for the system the damping is the max over the four components, taken per mode
  on the combined x + y expression (Section 2.3, Eq. para:dampsystems1d carried to 2D).
Multi-indices a = (a1, a2) run over a1, a2 <= 2 (the Q2 space), |a| up to 4.

Each cell's polynomial is written in physical coordinates (x, y) with sympy's Legendre
polynomials of the cell's own reference coordinates, and differentiated symbolically.
"""
import os

import sympy as sp

x, y = sp.symbols("x y")
K = 2
HX = sp.Rational(1, 10)
HY = sp.Rational(1, 16)
GAMMA = sp.Rational(7, 5)
R = sp.Rational

# Legendre coefficients u[v][(p, q)] of the five cells (centre at the origin); the rest are zero.
CELLS = {
    "C": [  # centre
        {(0, 0): R(1), (1, 0): R(1, 10), (0, 1): R(-1, 20), (2, 0): R(1, 40), (1, 1): R(1, 50),
         (0, 2): R(-1, 60), (2, 1): R(1, 70), (1, 2): R(-1, 80), (2, 2): R(1, 90)},
        {(0, 0): R(3, 10), (1, 0): R(1, 50), (0, 1): R(1, 100), (2, 2): R(-1, 200)},
        {(0, 0): R(-1, 5), (1, 0): R(-1, 100), (0, 1): R(1, 40), (1, 2): R(1, 300)},
        {(0, 0): R(5, 2), (1, 0): R(-1, 40), (0, 1): R(1, 50), (2, 0): R(3, 40), (1, 1): R(-1, 30),
         (0, 2): R(1, 20), (2, 1): R(-1, 25), (1, 2): R(1, 35), (2, 2): R(-1, 45)},
    ],
    "L": [
        {(0, 0): R(8, 5), (1, 0): R(1, 30), (0, 2): R(1, 50), (2, 1): R(-1, 60)},
        {(0, 0): R(1, 4), (1, 0): R(1, 80)},
        {(0, 0): R(-1, 10), (0, 1): R(1, 90)},
        {(0, 0): R(51, 20), (1, 0): R(1, 20), (2, 0): R(-1, 15), (1, 2): R(1, 40)},
    ],
    "R": [
        {(0, 0): R(1, 2), (0, 1): R(-1, 25), (2, 0): R(1, 35), (2, 2): R(1, 100)},
        {(0, 0): R(7, 20), (0, 1): R(-1, 70)},
        {(0, 0): R(-3, 10), (1, 1): R(1, 120)},
        {(0, 0): R(49, 20), (0, 1): R(1, 12), (1, 1): R(1, 18), (0, 2): R(-1, 22)},
    ],
    "B": [
        {(0, 0): R(3, 2), (1, 0): R(-1, 40), (1, 1): R(1, 45), (0, 2): R(1, 55)},
        {(0, 0): R(1, 5), (0, 1): R(1, 60)},
        {(0, 0): R(-1, 4), (1, 0): R(1, 75)},
        {(0, 0): R(63, 25), (2, 0): R(1, 16), (0, 1): R(-1, 14), (2, 1): R(1, 24)},
    ],
    "T": [
        {(0, 0): R(3, 5), (0, 1): R(1, 15), (1, 2): R(-1, 65), (2, 0): R(-1, 85)},
        {(0, 0): R(2, 5), (1, 0): R(-1, 90)},
        {(0, 0): R(-3, 20), (0, 2): R(1, 110)},
        {(0, 0): R(62, 25), (1, 0): R(1, 9), (0, 2): R(1, 13), (2, 2): R(-1, 17)},
    ],
}
# cell centres relative to the centre cell, and their flat index on the 3x3 mesh (x fastest)
OFFSET = {"C": (0, 0), "L": (-1, 0), "R": (1, 0), "B": (0, -1), "T": (0, 1)}
INDEX = {"C": 4, "L": 3, "R": 5, "B": 1, "T": 7}


def poly(name, v):
    """The cell's polynomial of variable v in physical coordinates."""
    ox, oy = OFFSET[name]
    xi = 2 * (x - ox * HX) / HX
    eta = 2 * (y - oy * HY) / HY
    return sum(c * sp.legendre(pp, xi) * sp.legendre(qq, eta) for (pp, qq), c in CELLS[name][v].items())


def d(expr, a1, a2):
    if a1:
        expr = sp.diff(expr, x, a1)
    if a2:
        expr = sp.diff(expr, y, a2)
    return expr


def edge_norm(v, a1, a2, vertical):
    """||[d^a u_v]|| over the centre cell's two vertical (or horizontal) edges: per edge the
    trapezoidal rule over its two corners of |own - neighbour|, divided by the edge length."""
    s = 0
    own = d(poly("C", v), a1, a2)
    for side, nb_name in ((-1, "L" if vertical else "B"), (1, "R" if vertical else "T")):
        nb = d(poly(nb_name, v), a1, a2)
        for corner in (-1, 1):
            pt = {x: side * HX / 2, y: corner * HY / 2} if vertical else {x: corner * HX / 2, y: side * HY / 2}
            s += R(1, 2) * sp.Abs(own.subs(pt) - nb.subs(pt))
    return sp.nsimplify(s)


def main():
    # average state of the centre cell and its wave speeds / enthalpy
    rho, mx, my, E = (CELLS["C"][v][(0, 0)] for v in range(4))
    ub, vb = mx / rho, my / rho
    p_avg = (GAMMA - 1) * (E - (mx * mx + my * my) / (2 * rho))
    c = sp.sqrt(GAMMA * p_avg / rho)
    bx, by = sp.Abs(ub) + c, sp.Abs(vb) + c
    Hbar = (E + p_avg) / rho

    # jump norms per variable, multi-index and direction
    JV = {(v, a1, a2): edge_norm(v, a1, a2, True) for v in range(4) for a1 in range(K + 1) for a2 in range(K + 1)}
    JH = {(v, a1, a2): edge_norm(v, a1, a2, False) for v in range(4) for a1 in range(K + 1) for a2 in range(K + 1)}

    lines = []
    for qq in range(K + 1):
        for pp in range(K + 1):
            if pp == 0 and qq == 0:
                continue
            l = pp + qq
            lam = pp * (pp + 1) + qq * (qq + 1)
            cfx = HY * bx / (4 * lam * Hbar)
            cfy = HX * by / (4 * lam * Hbar)
            per_var = []
            for v in range(4):
                sx = HX * JV[(v, 0, 0)]
                sy = HY * JH[(v, 0, 0)]
                for m in range(1, l + 1):
                    tv = sum(JV[(v, a1, m - a1)] for a1 in range(0, m + 1) if a1 <= K and m - a1 <= K)
                    th = sum(JH[(v, a1, m - a1)] for a1 in range(0, m + 1) if a1 <= K and m - a1 <= K)
                    sx += m * (m + 1) * HX ** (m + 1) * tv
                    sy += m * (m + 1) * HY ** (m + 1) * th
                per_var.append(cfx * sx + cfy * sy)
            vals = [sp.N(e, 40) for e in per_var]
            vmax = max(range(4), key=lambda i: vals[i])
            sigma = per_var[vmax] * (2 / HX) * (2 / HY) * lam
            lines.append("%d %d %d %s" % (pp, qq, vmax, sp.N(sigma, 25)))

    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "filter_2d_q2.txt")
    with open(out, "w") as f:
        f.write("# p q argmax-variable sigma^{p,q}; generated by make_filter_2d_q2.py (sympy, no oracle)\n")
        f.write("# 2D Euler Q2, 3x3 outflow mesh, h_x = 1/10, h_y = 1/16, centre cell = flat index 4\n")
        f.write("# Eqs. (para:damp22d)-(para:damp22d1), Section 3.2 (c_fx, c_fy), trapezoidal edge norms,\n")
        f.write("# max over components; the cells' coefficients are listed in make_filter_2d_q2.py\n")
        f.write("\n".join(lines) + "\n")
    print(open(out).read())


if __name__ == "__main__":
    main()
