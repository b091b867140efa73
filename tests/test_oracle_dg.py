"""Pins for the oracle's DG operator, SSP-RK3 stepping, projection and exact solutions.

- Table 1 of the paper (Example 3.1, Burgers on (-pi, pi), u0 = 1/2 + sin x, T = 0.5): the errors
  "without filter" are reproduced (errors at the scheme's k+1 Gauss points per cell, L2 not
  normalised by the domain). Values: tests/golden/table1_burgers.txt (copied from the paper).
- The "with filter" columns in the asymptotic regime, and the approach of the order to k+1.
- Conservation (Section 2.4, v = 1), L2 energy decay for linear advection (Theorem 2.1 with the
  filter contracting every mode), k+1 convergence for smooth 1D/2D problems (Theorem 2.2).
- 2D operator on y-invariant data equals the 1D operator (filter off): two code paths.
- Exact Riemann solver: Rankine–Hugoniot jump conditions and isentropic fan relations.
- Isentropic vortex of Example 3.4(a): an exact solution of the 2D Euler equations (finite
  difference residual of the conservation law at sample points).
"""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
BURGERS_T1 = [0.5, 1.0, 1.0, 0.0]  # a, b, w, phi: u0 = a + b sin(w x + phi)


def table1():
    rows = {}
    with open(os.path.join(GOLDEN, "table1_burgers.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, n, l2f, lif, l2, li = line.split()
            rows[(int(k), int(n))] = tuple(map(float, (l2f, lif, l2, li)))
    return rows


def run_table1(k, N, filt):
    p = O.Problem(dim=1, nx=N, x0=-math.pi, x1=math.pi, k=k, eq=O.EQ_BURGERS, filter=filt, cfl=0.1)
    u = O.project(p, O.IC_SINE, BURGERS_T1)
    u, t, n = O.advance(p, u, 0.0, 0.5)
    assert t == 0.5
    _, l2, li = O.errors(p, u, O.EX_BURGERS, BURGERS_T1 + [2 * math.pi], 0.5, nq_err=k + 1)
    return l2, li


@pytest.mark.parametrize("k,N,tol", [(1, 20, 0.02), (1, 40, 0.02), (1, 80, 0.02), (1, 160, 0.02),
                                     (1, 320, 0.02), (2, 20, 0.02), (2, 40, 0.02), (2, 160, 0.02),
                                     (2, 320, 0.02), (3, 20, 0.1), (3, 40, 0.06)])
def test_table1_without_filter(k, N, tol):
    # P1 and P2 agree to the three printed digits; P3 to a few per cent. The P2, N=80 entry is left
    # out: it is printed as 2.13E-05, which contradicts the paper's own order column (the order 2.89
    # to N=160 implies 1.81e-6 * 2**2.89 = 1.34e-5, the value this oracle gives).
    l2, li = run_table1(k, N, 0)
    _, _, pl2, pli = table1()[(k, N)]
    assert l2 == pytest.approx(pl2, rel=tol)
    assert li == pytest.approx(pli, rel=tol)


def test_table1_p2_n80_matches_the_order_column():
    l2, _ = run_table1(2, 80, 0)
    _, _, pl2_160, _ = table1()[(2, 160)]
    assert l2 == pytest.approx(pl2_160 * 2 ** 2.89, rel=0.02)


@pytest.mark.parametrize("k,N", [(1, 20), (1, 40), (1, 80), (1, 160), (1, 320), (2, 320)])
def test_table1_with_filter_asymptotic(k, N):
    l2, li = run_table1(k, N, 1)
    pl2, pli, _, _ = table1()[(k, N)]
    assert l2 == pytest.approx(pl2, rel=0.35)
    assert li == pytest.approx(pli, rel=0.35)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_burgers_smooth_convergence_rescaled(k):
    # u0 = 0.5 + sin(pi x) on [0,2], periodic, t = 0.1 (before the steepening switches the filter
    # on hard); the filtered scheme converges at order about k+1 (Theorem 2.2)
    errs = []
    Ns = [40, 80, 160]
    for N in Ns:
        p = O.Problem(dim=1, nx=N, x0=0.0, x1=2.0, k=k, eq=O.EQ_BURGERS, filter=1, cfl=0.1)
        prm = [0.5, 1.0, math.pi, 0.0]
        u = O.project(p, O.IC_SINE, prm)
        u, t, n = O.advance(p, u, 0.0, 0.1)
        errs.append(O.errors(p, u, O.EX_BURGERS, prm + [2.0], 0.1)[0])
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert orders[-1] > k + 1 - 0.3, orders


@pytest.mark.parametrize("k", [1, 2, 3])
def test_conservation_periodic_burgers_with_filter(k):
    p = O.Problem(dim=1, nx=50, x0=0.0, x1=2.0, k=k, eq=O.EQ_BURGERS, filter=1, cfl=0.1)
    u = O.project(p, O.IC_SINE, [0.5, 1.0, math.pi, 0.0])
    m0 = O.mass(p, u)[0]
    for _ in range(100):
        u = O.step(p, u, O.dt(p, u))
    assert abs(O.mass(p, u)[0] - m0) <= 1e-13 * abs(m0) + 1e-15


def test_conservation_euler_2d_periodic():
    p = O.Problem(dim=2, nx=8, ny=6, x0=0, x1=1, y0=0, y1=0.75, k=2, eq=O.EQ_EULER, filter=1)
    u = O.project(p, O.IC_VORTEX2D, [0.5, 0.375, 2.0, 0.0])
    m0 = O.mass(p, u)
    for _ in range(20):
        u = O.step(p, u, O.dt(p, u))
    np.testing.assert_allclose(O.mass(p, u), m0, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("filt", [0, 1])
def test_l2_energy_nonincreasing_linear_advection(filt):
    # with LLF = upwind for c > 0 and CFL 0.1, RK3-DG is L2-stable; the filter contracts every mode
    p = O.Problem(dim=1, nx=40, x0=0.0, x1=1.0, k=2, eq=O.EQ_ADVECTION, adv=(1.0, 0.0), filter=filt)
    u = np.zeros(p.shape)
    u[0, 0, :] = np.where(np.arange(40) < 20, 1.0, 0.0)   # square wave: the filter is active
    u[0, 1, :] = 0.1 * np.sin(np.arange(40))
    e_prev = O.energy(p, u)
    for _ in range(60):
        u = O.step(p, u, O.dt(p, u))
        e = O.energy(p, u)
        assert e <= e_prev * (1 + 1e-14)
        e_prev = e


def test_l2_energy_nonincreasing_2d_advection():
    p = O.Problem(dim=2, nx=10, ny=10, k=1, eq=O.EQ_ADVECTION, adv=(1.0, 0.5), filter=1)
    rng = np.random.default_rng(3)
    u = 0.2 * rng.normal(size=p.shape)
    e_prev = O.energy(p, u)
    for _ in range(30):
        u = O.step(p, u, O.dt(p, u))
        e = O.energy(p, u)
        assert e <= e_prev * (1 + 1e-14)
        e_prev = e


@pytest.mark.parametrize("k", [1, 2, 3])
def test_projection_reproduces_polynomials(k):
    # L2 projection: a constant is reproduced exactly; sin(x) against closed-form Legendre moments
    p = O.Problem(dim=1, nx=4, x0=0.0, x1=4.0, k=k, eq=O.EQ_BURGERS)
    # constant state: all higher modes zero, mode 0 exact
    u = O.project(p, O.IC_SINE, [0.7, 0.0, 1.0, 0.0])
    np.testing.assert_allclose(u[0, 0], 0.7, rtol=1e-15)
    np.testing.assert_allclose(u[0, 1:], 0.0, atol=1e-15)
    # sin projection: mode l of sin(x) on a cell equals (2l+1)/2 int sin(xc + h s/2) P_l(s) ds;
    # for l = 1 the integral is closed form: 3/2 * (2/(a^2)) (sin a - a cos a) cos xc, a = h/2
    u = O.project(p, O.IC_SINE, [0.0, 1.0, 1.0, 0.0], nq_init=12)
    a = 0.5
    for i in range(4):
        xc = i + 0.5
        assert u[0, 0, i] == pytest.approx(math.sin(xc) * math.sin(a) / a, rel=1e-13)
        assert u[0, 1, i] == pytest.approx(1.5 * 2 / a ** 2 * (math.sin(a) - a * math.cos(a)) * math.cos(xc),
                                           rel=1e-12, abs=1e-14)


def test_2d_operator_reduces_to_1d_without_filter():
    rng = np.random.default_rng(5)
    nx, k = 6, 2
    p1 = O.Problem(dim=1, nx=nx, x0=0, x1=0.6, k=k, eq=O.EQ_EULER, filter=0)
    p2 = O.Problem(dim=2, nx=nx, ny=2, x0=0, x1=0.6, y0=0, y1=0.2, k=k, eq=O.EQ_EULER, filter=0)
    u1 = np.zeros(p1.shape)
    u1[0, 0] = 1 + 0.2 * rng.random(nx)
    u1[1, 0] = 0.3 * rng.random(nx)
    u1[2, 0] = 2.5 + rng.random(nx)
    u1[:, 1:] = 0.01 * rng.normal(size=(3, k, nx))
    u2 = np.zeros(p2.shape)
    for v2, v1 in ((0, 0), (1, 1), (3, 2)):
        for l in range(k + 1):
            u2[v2, l] = np.tile(u1[v1, l], 2)
    R1 = O.residual(p1, u1)
    R2 = O.residual(p2, u2)
    for v2, v1 in ((0, 0), (1, 1), (3, 2)):
        for l in range(k + 1):
            np.testing.assert_allclose(R2[v2, l, :nx], R1[v1, l], rtol=1e-11, atol=1e-11)
    assert np.max(np.abs(R2[2])) < 1e-11                      # no y-momentum generated
    assert np.max(np.abs(R2[:, k + 1:])) < 1e-11              # no y-dependent modes generated


@pytest.mark.parametrize("k", [1, 2])
def test_entropy_wave_convergence(k):
    prm = [1.0, 0.2, 2 * math.pi, 1.0, 1.0]
    errs = []
    for N in (16, 32, 64):
        p = O.Problem(dim=1, nx=N, k=k, eq=O.EQ_EULER, filter=1, cfl=0.1)
        u = O.project(p, O.IC_ENTROPY1D, prm)
        u, t, n = O.advance(p, u, 0.0, 0.1)
        errs.append(O.errors(p, u, O.EX_ENTROPY1D, prm, 0.1, var=0)[1])
    order = math.log2(errs[-2] / errs[-1])
    assert order > k + 1 - 0.35, errs


def test_vortex_convergence_2d_q1():
    errs = []
    for N in (8, 16, 32):
        p = O.Problem(dim=2, nx=N, ny=N, x0=0, x1=10, y0=-5, y1=5, k=1, eq=O.EQ_EULER, filter=1)
        prm = [5.0, 0.0, 5.0, 0.0]
        u = O.project(p, O.IC_VORTEX2D, prm)
        u, t, n = O.advance(p, u, 0.0, 0.5)
        errs.append(O.errors(p, u, O.EX_VORTEX2D, prm[:3], 0.5, var=0)[1])
    order = math.log2(errs[-2] / errs[-1])
    assert order > 1.7, errs


def test_riemann_exact_jump_conditions():
    g = 1.4
    WL, WR = [1.0, 0.0, 1.0], [0.125, 0.0, 0.1]      # left rarefaction, right shock
    # sample finely, locate the right-moving shock and check Rankine–Hugoniot across it
    xs = np.linspace(-2, 2, 40001)
    W = np.array([O.riemann_exact(g, WL, WR, x) for x in xs])
    rho = W[:, 0]
    jumps = np.nonzero(np.abs(np.diff(rho)) > 0.01)[0]   # the fan is continuous: only 2 jumps
    assert len(jumps) == 2
    c, i = int(jumps[0]), int(jumps[1])                  # contact, then the right shock
    A, B = W[i - 2], W[i + 3]                          # states on both sides of the shock
    s = xs[i]

    def cons(w):
        return np.array([w[0], w[0] * w[1], w[2] / (g - 1) + 0.5 * w[0] * w[1] ** 2])

    def flx(w):
        E = w[2] / (g - 1) + 0.5 * w[0] * w[1] ** 2
        return np.array([w[0] * w[1], w[0] * w[1] ** 2 + w[2], w[1] * (E + w[2])])

    jump_f = flx(A) - flx(B)
    jump_u = cons(A) - cons(B)
    np.testing.assert_allclose(jump_f, s * jump_u, rtol=2e-3, atol=2e-3)
    # across the contact: pressure and velocity continuous, density jumps
    assert abs(W[c - 2, 2] - W[c + 3, 2]) < 1e-12
    assert abs(W[c - 2, 1] - W[c + 3, 1]) < 1e-12
    assert abs(W[c - 2, 0] - W[c + 3, 0]) > 0.05
    # inside the rarefaction fan p / rho^gamma equals the left state's value, u + 2c/(g-1) constant
    fan = W[(xs > -1.0) & (xs < -0.2)]
    ent = fan[:, 2] / fan[:, 0] ** g
    np.testing.assert_allclose(ent, 1.0, rtol=1e-12)
    riem = fan[:, 1] + 2 * np.sqrt(g * fan[:, 2] / fan[:, 0]) / (g - 1)
    np.testing.assert_allclose(riem, 2 * math.sqrt(g) / (g - 1), rtol=1e-12)


def test_vortex_is_exact_euler_solution():
    g, x0, y0, beta = 1.4, 5.0, 0.0, 5.0

    def U(x, y, t):
        r, u, v, p = O.vortex_exact(g, x0, y0, beta, 10.0, 10.0, x, y, t)
        return np.array([r, r * u, r * v, p / (g - 1) + 0.5 * r * (u * u + v * v)])

    def F(x, y, t):
        r, u, v, p = O.vortex_exact(g, x0, y0, beta, 10.0, 10.0, x, y, t)
        E = p / (g - 1) + 0.5 * r * (u * u + v * v)
        fx = np.array([r * u, r * u * u + p, r * u * v, u * (E + p)])
        fy = np.array([r * v, r * u * v, r * v * v + p, v * (E + p)])
        return fx, fy

    e = 1e-5
    for (x, y, t) in [(5.3, 0.4, 0.0), (4.2, -0.7, 0.3), (6.1, 0.9, 1.0)]:
        dUdt = (U(x, y, t + e) - U(x, y, t - e)) / (2 * e)
        dFx = (F(x + e, y, t)[0] - F(x - e, y, t)[0]) / (2 * e)
        dFy = (F(x, y + e, t)[1] - F(x, y - e, t)[1]) / (2 * e)
        np.testing.assert_allclose(dUdt + dFx + dFy, 0.0, atol=1e-7)
