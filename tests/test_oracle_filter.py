"""Pins for the oracle's jump filter.

- Hand-computed single-cell damping factors (1D Burgers P1/P2, 1D Euler P1) from
  Eqs. (para:damp2)-(para:damp21) and the Euler choice c_f^l = beta/(4 l(l+1)) / Hbar (Section 3.1).
- A 2D Euler Q1 cell whose damping was derived symbolically by tests/golden/make_filter_2d_q1.py
- A 2D Euler Q2 cell (non-square cells, non-constant neighbours, every mode up to (2,2)) whose
  damping was derived symbolically by tests/golden/make_filter_2d_q2.py
  (sympy, from Eqs. (para:damp22d)-(para:damp22d1) and Section 3.2), independent of the oracle.
- Invariants fixed by the method: sigma^0 = 0 (cell averages untouched, Eq. timespli:1dscalar);
  the filter is the identity on a global polynomial of degree <= k; systems take the max over
  components (Eq. para:dampsystems1d); the 2D damping of y-invariant data equals h_x times the 1D
  damping (substituting Section 3.2's c_f into Eq. para:damp22d versus Section 3.1's into Eq. para:damp2).
"""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def three_cells(k, eq=O.EQ_BURGERS):
    return O.Problem(dim=1, nx=3, x0=0.0, x1=0.3, k=k, eq=eq, bc=(O.BC_OUTFLOW,) * 4)


def test_burgers_p1_hand_example():
    p = three_cells(1)
    u = np.zeros(p.shape)
    u[0, 0, :] = [0.0, 1.0, 1.0]
    u[0, 1, :] = [0.0, 0.5, 0.0]
    s = O.filter_sigma(p, u)
    # J_0 = 1, J_1 = 20, sigma_{j,1} = 0.0625, sigma^1 = 50
    assert s[1, 1] == pytest.approx(50.0, rel=1e-14)
    out = O.filter(p, u, 1e-3)
    assert out[0, 1, 1] == pytest.approx(0.475614712250357, rel=1e-14)
    assert out[0, 0, 1] == u[0, 0, 1]


def test_burgers_p2_hand_example():
    p = three_cells(2)
    u = np.zeros(p.shape)
    u[0, 0, :] = [0.0, 1.0, 1.0]
    u[0, 1, :] = [0.0, 0.5, 0.0]
    u[0, 2, :] = [0.0, 0.25, 0.0]
    s = O.filter_sigma(p, u)
    # J = (1.5, 30, 600): sigma^1 = 75, sigma^2 = 435
    assert s[1, 1] == pytest.approx(75.0, rel=1e-14)
    assert s[2, 1] == pytest.approx(435.0, rel=1e-14)
    out = O.filter(p, u, 1e-3)
    assert out[0, 1, 1] / u[0, 1, 1] == pytest.approx(0.927743486328553, rel=1e-14)
    assert out[0, 2, 1] / u[0, 2, 1] == pytest.approx(0.647264667078035, rel=1e-14)


def test_euler_p1_hand_example():
    p = three_cells(1, O.EQ_EULER)
    u = np.zeros(p.shape)
    u[0, 0, :] = 1.0
    u[2, 0, :] = 2.5
    u[0, 1, 1] = 0.1
    s = O.filter_sigma(p, u)
    # beta = c = sqrt(1.4), Hbar = 3.5, rho jumps J_0 = 0.2, J_1 = 4
    assert s[1, 1] == pytest.approx(3.380617018914066, rel=1e-14)
    out = O.filter(p, u, 1e-3)
    assert out[0, 1, 1] / u[0, 1, 1] == pytest.approx(0.996625090832968, rel=1e-14)


def test_global_sigma_burgers_p2_hand_example():
    # Eq. (para:damp) with c_f = c_f^l: one coefficient for every mode from the jumps of all orders
    # up to k, sigma^l = beta / h^2 (h J_0 + 2 h^2 J_1 + 6 h^3 J_2) = 435 for l = 1 and l = 2 (the
    # mode-dependent filter's sigma^2 of the same cell)
    p = three_cells(2)
    p.filter_kind = O.FILTER_GLOBAL
    u = np.zeros(p.shape)
    u[0, 0, :] = [0.0, 1.0, 1.0]
    u[0, 1, :] = [0.0, 0.5, 0.0]
    u[0, 2, :] = [0.0, 0.25, 0.0]
    s = O.filter_sigma(p, u)
    assert s[1, 1] == pytest.approx(435.0, rel=1e-14)
    assert s[2, 1] == pytest.approx(435.0, rel=1e-14)


def test_oedg_burgers_p2_hand_example():
    # Section 2.1's OEDG form: sigma^{l,OE} = c (h J_0 + sum_{m<=l} (2m+1)/m! h^{m+1} J_m) / h^2,
    # c = beta / (2 (2k-1) N), N = ||u - avg(u)||_inf. Cell averages (0, 1, 1): avg = 2/3; the largest
    # deviation is at the centre cell's Gauss point xi = +sqrt(3/5), where u = 1 + 0.5 sqrt(3/5)
    # + 0.25 P_2 = 1 + 0.5 sqrt(3/5) + 0.1. With J = (1.5, 30, 600), h = 0.1, beta = 1, k = 2:
    # sigma^1 = (0.15 + 0.9) / 0.01 / (6 N) = 17.5 / N, sigma^2 = (1.05 + 1.5) / 0.01 / (6 N) = 42.5 / N
    p = three_cells(2)
    p.filter_kind = O.FILTER_OEDG
    u = np.zeros(p.shape)
    u[0, 0, :] = [0.0, 1.0, 1.0]
    u[0, 1, :] = [0.0, 0.5, 0.0]
    u[0, 2, :] = [0.0, 0.25, 0.0]
    N = 1.0 + 0.5 * math.sqrt(0.6) + 0.1 - 2.0 / 3.0
    assert O.oedg_norms(p, u)[0] == pytest.approx(N, rel=1e-14)
    s = O.filter_sigma(p, u)
    assert s[1, 1] == pytest.approx(17.5 / N, rel=1e-13)
    assert s[2, 1] == pytest.approx(42.5 / N, rel=1e-13)
    assert s[0, 1] == 0.0


def test_oedg_euler_p1_hand_example():
    # Only the density jumps (J_0 = 0.2, J_1 = 4 as in the jump-filter example); each component
    # has its own normaliser: N_rho = 0.1 / sqrt(3) (the density's deviation at the Gauss points of
    # the centre cell, every average being 1), N = 0 for momentum and energy (their c^OE is 0).
    # sigma^1 = sqrt(1.4) / (2 N_rho) (0.1 * 0.2 + 3 * 0.01 * 4) / 0.01 = 70 sqrt(4.2); no 1/Hbar
    p = three_cells(1, O.EQ_EULER)
    p.filter_kind = O.FILTER_OEDG
    u = np.zeros(p.shape)
    u[0, 0, :] = 1.0
    u[2, 0, :] = 2.5
    u[0, 1, 1] = 0.1
    n = O.oedg_norms(p, u)
    assert n[0] == pytest.approx(0.1 / math.sqrt(3.0), rel=1e-14) and n[1] == 0.0 and n[2] == 0.0
    s = O.filter_sigma(p, u)
    assert s[1, 1] == pytest.approx(70.0 * math.sqrt(4.2), rel=1e-13)


@pytest.mark.parametrize("kind", [O.FILTER_GLOBAL, O.FILTER_OEDG])
def test_variants_2d_reduce_to_1d_on_y_invariant_data(kind):
    # y-invariant data: no horizontal jumps, the vertical edge averages equal the 1D end jumps. The
    # global coefficient keeps the jump filter's 2D scaling (h_x times the 1D value); the OEDG form
    # divides each direction by its own h, so it gives the 1D value itself.
    k = 2
    rng = np.random.default_rng(5)
    p1 = O.Problem(dim=1, nx=7, x0=0.0, x1=0.7, k=k, eq=O.EQ_EULER, bc=(O.BC_PERIODIC,) * 4, filter_kind=kind)
    p2 = O.Problem(dim=2, nx=7, ny=4, x0=0.0, x1=0.7, y0=0.0, y1=0.4, k=k, eq=O.EQ_EULER,
                   bc=(O.BC_PERIODIC,) * 4, filter_kind=kind)
    u1 = np.zeros(p1.shape)
    u1[0, 0] = rng.uniform(1.0, 2.0, 7)
    u1[1, 0] = rng.uniform(-0.3, 0.3, 7)
    u1[2, 0] = rng.uniform(4.0, 6.0, 7)
    u1[:, 1:] = rng.uniform(-0.05, 0.05, (3, k, 7))
    u2 = np.zeros(p2.shape)
    for j in range(4):
        cells = slice(7 * j, 7 * j + 7)
        u2[0, :k + 1, cells] = u1[0]          # modes (p, 0): p = 0..k
        u2[1, :k + 1, cells] = u1[1]
        u2[3, :k + 1, cells] = u1[2]
    s1 = O.filter_sigma(p1, u1)
    s2 = O.filter_sigma(p2, u2)
    scale = p2.hx if kind == O.FILTER_GLOBAL else 1.0
    for pdeg in range(1, k + 1):
        np.testing.assert_allclose(s2[pdeg, :7], scale * s1[pdeg], rtol=1e-12)


def test_global_sigma_q2_symbolic_example():
    # the global coefficient takes every derivative order (|alpha| <= 4 for Q2) for every mode; with
    # Section 3.2's c_f the lambda_{p,q} cancels, so every mode gets the symbolic example's (2,2) value
    p, u, rows = _q2_example()
    p.filter_kind = O.FILTER_GLOBAL
    top = [val for pp, qq, _, val in rows if (pp, qq) == (2, 2)][0]
    s = O.filter_sigma(p, u)
    for pp, qq, _, _ in rows:
        assert s[pp + 3 * qq, 4] == pytest.approx(top, rel=1e-13)


def test_outflow_ghost_is_the_cell_average():
    # outflow boundary reading: the ghost cell holds the constant state of the interior cell's
    # average. Burgers P1, h = 0.1, boundary cell [1, 0.5], neighbours [1, 0]: left face jumps
    # |0.5 - 1| = 0.5 and |10 - 0| = 10, right face 0.5 and 10: J_0 = 1, J_1 = 20, sigma^1 = 50
    p = three_cells(1)
    u = np.zeros(p.shape)
    u[0, 0, :] = [1.0, 1.0, 1.0]
    u[0, 1, :] = [0.5, 0.0, 0.0]
    s = O.filter_sigma(p, u)
    assert s[1, 0] == pytest.approx(50.0, rel=1e-14)
    # the constant right boundary cell sees no jump at its outflow face
    assert s[1, 2] == 0.0


def _golden_2d():
    rows = []
    with open(os.path.join(GOLDEN, "filter_2d_q1.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            pp, qq, _, val = line.split()
            rows.append((int(pp), int(qq), float(val)))
    return rows


def test_euler_2d_q1_symbolic_example():
    p = O.Problem(dim=2, nx=3, ny=3, x0=0, x1=0.3, y0=0, y1=0.3, k=1, eq=O.EQ_EULER,
                  bc=(O.BC_OUTFLOW,) * 4)
    u = np.zeros(p.shape)
    u[0, 0, :] = 1.0
    u[3, 0, :] = 2.5
    centre = 4
    u[0, 1, centre] = 0.1    # (p,q) = (1,0)
    u[0, 2, centre] = 0.05   # (0,1)
    u[0, 3, centre] = 0.02   # (1,1)
    s = O.filter_sigma(p, u)
    for pp, qq, val in _golden_2d():
        m = pp + 2 * qq
        assert s[m, centre] == pytest.approx(val, rel=1e-13)


def _q2_example():
    """The five cells of tests/golden/make_filter_2d_q2.py (read from that script) on its 3x3 mesh."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_q2", os.path.join(GOLDEN, "make_filter_2d_q2.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    p = O.Problem(dim=2, nx=3, ny=3, x0=0, x1=0.3, y0=0, y1=3.0 / 16.0, k=2, eq=O.EQ_EULER,
                  bc=(O.BC_OUTFLOW,) * 4)
    u = np.zeros(p.shape)
    u[0, 0, :] = 1.0            # the four corner cells: a constant physical state (not used)
    u[3, 0, :] = 2.5
    for name, cell in mod.INDEX.items():
        for v in range(4):
            u[v, :, cell] = 0.0
            for (pp, qq), c in mod.CELLS[name][v].items():
                u[v, pp + 3 * qq, cell] = float(c)
    rows = []
    with open(os.path.join(GOLDEN, "filter_2d_q2.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            pp, qq, vmax, val = line.split()
            rows.append((int(pp), int(qq), int(vmax), float(val)))
    return p, u, rows


def test_euler_2d_q2_symbolic_example():
    # all eight non-constant modes, including (2,1), (1,2), (2,2) (multi-indices up to |a| = 4),
    # non-square cells, non-constant neighbours, the max over components switching variable
    p, u, rows = _q2_example()
    assert len(rows) == 8 and {r[2] for r in rows} == {0, 3}
    s = O.filter_sigma(p, u)
    for pp, qq, _, val in rows:
        assert s[pp + 3 * qq, 4] == pytest.approx(val, rel=1e-13), (pp, qq)


def test_euler_2d_q2_symbolic_example_filter_factors():
    # the filter applies exp(-sigma^{p,q} dt) to each mode and leaves the averages
    p, u, rows = _q2_example()
    dt_ = 1e-3
    out = O.filter(p, u, dt_)
    np.testing.assert_array_equal(out[:, 0, 4], u[:, 0, 4])
    for pp, qq, _, val in rows:
        m = pp + 3 * qq
        np.testing.assert_allclose(out[:, m, 4], u[:, m, 4] * np.exp(-val * dt_), rtol=1e-13, atol=0)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_filter_leaves_cell_averages(k):
    rng = np.random.default_rng(k)
    p = O.Problem(dim=1, nx=17, k=k, eq=O.EQ_BURGERS)
    u = rng.normal(size=p.shape)
    out = O.filter(p, u, 0.3)
    np.testing.assert_array_equal(out[:, 0, :], u[:, 0, :])
    assert np.all(np.abs(out[:, 1:, :]) <= np.abs(u[:, 1:, :]))


@pytest.mark.parametrize("k", [1, 2, 3])
def test_filter_identity_on_global_polynomial_1d(k):
    # the projection of a global polynomial of degree <= k has no jumps of any order: sigma = 0
    p = O.Problem(dim=1, nx=9, x0=-1.0, x1=2.0, k=k, eq=O.EQ_ADVECTION, bc=(O.BC_OUTFLOW,) * 4)
    u = np.zeros(p.shape)
    coeffs = [0.3, -1.1, 0.7, 0.25][: k + 1]
    for i in range(p.nx):
        xc = p.x0 + (i + 0.5) * p.hx
        # Legendre coefficients of sum_d coeffs[d] x^d on the cell, from an exact (k+1)-point fit
        xs, ws = O.gauss(k + 2)
        vals = [sum(c * (xc + 0.5 * p.hx * s) ** d for d, c in enumerate(coeffs)) for s in xs]
        for l in range(k + 1):
            u[0, l, i] = sum(w * v * O.legendre(l, s) for s, w, v in zip(xs, ws, vals)) * (2 * l + 1) / 2
    s = O.filter_sigma(p, u)
    # away from the outflow boundary every jump of every order vanishes (the boundary cells see the
    # ghost, a constant state, so a non-constant polynomial has a jump there)
    assert np.max(np.abs(s[:, 1:-1])) < 1e-9
    np.testing.assert_allclose(O.filter(p, u, 1.0)[:, :, 1:-1], u[:, :, 1:-1], rtol=0, atol=1e-13)


def test_filter_identity_on_global_polynomial_2d():
    p = O.Problem(dim=2, nx=4, ny=5, x0=0, x1=1, y0=0, y1=1.25, k=2, eq=O.EQ_ADVECTION,
                  bc=(O.BC_OUTFLOW,) * 4, adv=(1.0, 0.5))
    u = np.zeros(p.shape)
    for j in range(p.ny):
        for i in range(p.nx):
            c = i + p.nx * j
            xc, yc = (i + 0.5) * p.hx, (j + 0.5) * p.hy
            # f(x,y) = 0.5 + x - 2y + 0.3 x y + 0.4 x^2 y: in each cell a Q2 polynomial
            a, b = 0.5 * p.hx, 0.5 * p.hy
            # expand in xi, eta: x = xc + a xi, y = yc + b eta; collect monomials, convert to Legendre
            mono = np.zeros((3, 3))
            mono[0, 0] += 0.5 + xc - 2 * yc + 0.3 * xc * yc + 0.4 * xc * xc * yc
            mono[1, 0] += a + 0.3 * a * yc + 0.8 * xc * a * yc
            mono[0, 1] += -2 * b + 0.3 * xc * b + 0.4 * xc * xc * b
            mono[1, 1] += 0.3 * a * b + 0.8 * xc * a * b
            mono[2, 0] += 0.4 * a * a * yc
            mono[2, 1] += 0.4 * a * a * b
            # x^2 = (P0 + 2 P2)/3 in each variable
            to_leg = np.array([[1, 0, 1 / 3], [0, 1, 0], [0, 0, 2 / 3]])
            leg = to_leg @ mono @ to_leg.T
            for qq in range(3):
                for pp in range(3):
                    u[0, pp + 3 * qq, c] = leg[pp, qq]
    s = O.filter_sigma(p, u).reshape(p.nmodes, p.ny, p.nx)
    assert np.max(np.abs(s[:, 1:-1, 1:-1])) < 1e-8


def test_systems_take_max_over_components():
    p = three_cells(2, O.EQ_EULER)
    base = np.zeros(p.shape)
    base[0, 0, :] = 1.0
    base[2, 0, :] = 2.5
    ua = base.copy()
    ua[0, 1, 1] = 0.05          # density jump only
    ub = base.copy()
    ub[2, 2, 1] = 0.2           # energy jump only
    uab = base.copy()
    uab[0, 1, 1] = 0.05
    uab[2, 2, 1] = 0.2
    sa, sb, sab = O.filter_sigma(p, ua), O.filter_sigma(p, ub), O.filter_sigma(p, uab)
    np.testing.assert_allclose(sab[:, 1], np.maximum(sa[:, 1], sb[:, 1]), rtol=1e-14)
    assert sa[1, 1] > 0 and sb[1, 1] > 0


@pytest.mark.parametrize("k", [1, 2])
def test_2d_damping_of_y_invariant_data_is_hx_times_1d(k):
    rng = np.random.default_rng(11 + k)
    nx = 7
    p1 = O.Problem(dim=1, nx=nx, x0=0, x1=0.7, k=k, eq=O.EQ_EULER)
    p2 = O.Problem(dim=2, nx=nx, ny=3, x0=0, x1=0.7, y0=0, y1=0.3, k=k, eq=O.EQ_EULER)
    u1 = np.zeros(p1.shape)
    u1[0, 0, :] = 1 + 0.3 * rng.random(nx)
    u1[1, 0, :] = 0.2 * rng.random(nx)
    u1[2, 0, :] = 2.5 + rng.random(nx)
    u1[:, 1:, :] = 0.02 * rng.normal(size=(3, k, nx))
    u2 = np.zeros(p2.shape)
    for v2, v1 in ((0, 0), (1, 1), (3, 2)):
        for l in range(k + 1):
            u2[v2, l, :] = np.tile(u1[v1, l, :], 3)      # mode (l, 0), constant in y
    s1 = O.filter_sigma(p1, u1)
    s2 = O.filter_sigma(p2, u2)
    for l in range(1, k + 1):
        np.testing.assert_allclose(s2[l, :nx], p1.hx * s1[l, :], rtol=1e-12)
