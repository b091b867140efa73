"""Pins for the oracle's hybrid limiter (Algorithm 1: jump indicator, troubled cells blended with the
jump filter by omega_j = (max eta - eta_j) / (max eta - 1)): hand-computed indicators, the 2D-to-1D
reduction, the blend's end points, and the scheme-level reductions."""
import math

import numpy as np
import pytest

import oracle as O


def burgers1d(nx=4, h=0.1, k=1, bc=O.BC_PERIODIC):
    return O.Problem(dim=1, nx=nx, x0=0.0, x1=nx * h, k=k, eq=O.EQ_BURGERS, bc=(bc,) * 4, hybrid=1)


def test_indicator_1d_hand_computed():
    # u = a + b xi per cell; end values a -+ b. Periodic, h = 0.1.
    p = burgers1d()
    u = np.zeros(p.shape)
    u[0, 0] = [1.0, 2.0, 2.0, 0.5]
    u[0, 1] = [0.5, 0.0, -0.25, 0.0]
    left = u[0, 0] - u[0, 1]           # value at xi = -1
    right = u[0, 0] + u[0, 1]          # value at xi = +1
    eta = O.jump_indicator(p, u)
    for j in range(4):
        jl = abs(left[j] - right[(j - 1) % 4])
        jr = abs(left[(j + 1) % 4] - right[j])
        assert eta[j] == pytest.approx((jl + jr) / 0.2, rel=1e-15)
    # cell 0: left jump |0.5 - 0.5| = 0, right jump |2 - 1.5| = 0.5 -> eta = 2.5
    assert eta[0] == pytest.approx(2.5, rel=1e-15)


def test_indicator_outflow_ghost_is_the_cell_average():
    p = burgers1d(nx=3, bc=O.BC_OUTFLOW)
    u = np.zeros(p.shape)
    u[0, 0] = [1.0, 1.0, 1.0]
    u[0, 1] = [0.3, 0.0, 0.0]          # first cell: ends 0.7 and 1.3 against ghost 1.0 and neighbour 1.0
    eta = O.jump_indicator(p, u)
    assert eta[0] == pytest.approx((0.3 + 0.3) / 0.2, rel=1e-14)
    assert eta[1] == pytest.approx(0.3 / 0.2, rel=1e-14)
    assert eta[2] == 0.0


def test_indicator_2d_reduces_to_1d_on_y_invariant_data():
    rng = np.random.default_rng(5)
    p1 = O.Problem(dim=1, nx=12, x0=0.0, x1=1.2, k=2, eq=O.EQ_EULER, hybrid=1)
    p2 = O.Problem(dim=2, nx=12, ny=5, x0=0.0, x1=1.2, y0=0.0, y1=0.5, k=2, eq=O.EQ_EULER, hybrid=1)
    u1 = np.zeros(p1.shape)
    u1[:, 0] = [[1.0], [0.2], [2.5]] + rng.uniform(-0.1, 0.1, (3, 12))
    u1[:, 1:] = rng.uniform(-0.2, 0.2, (3, 2, 12))
    u2 = np.zeros(p2.shape)
    var2 = [0, 1, 3]                                  # rho, m_x, E; m_y = 0
    for j in range(5):
        for v1, v2 in enumerate(var2):
            for l in range(3):                        # mode (p = l, q = 0) has index l
                u2[v2, l, j * 12:(j + 1) * 12] = u1[v1, l]
    e1 = O.jump_indicator(p1, u1)
    e2 = O.jump_indicator(p2, u2).reshape(5, 12)
    for j in range(5):
        np.testing.assert_allclose(e2[j], e1, rtol=1e-14, atol=1e-14)


def test_hybrid_blend_end_points():
    # one large jump: the cells beside it are troubled, the max cell gets u^lim, the others u^DG
    p = burgers1d(nx=6, k=2)
    rng = np.random.default_rng(1)
    u = np.zeros(p.shape)
    u[0, 0] = [1.0, 1.0, 1.0, 1.5, 1.5, 1.5]
    u[0, 1] = [0.0, 0.0, 0.02, 0.0, 0.0, 0.0]
    u[0, 2] = rng.uniform(-0.01, 0.01, 6)
    dt = 0.004
    eta = O.jump_indicator(p, u)
    lim = O.filter(p, u, dt)
    out = O.hybrid(p, u, dt)
    emax = eta.max()
    assert emax > 1.0
    for j in range(6):
        if eta[j] <= 1.0:
            np.testing.assert_array_equal(out[:, :, j], u[:, :, j])
        elif eta[j] == emax:
            np.testing.assert_allclose(out[:, :, j], lim[:, :, j], rtol=1e-15, atol=1e-17)
        else:
            w = (emax - eta[j]) / (emax - 1.0)
            np.testing.assert_allclose(out[:, :, j], w * u[:, :, j] + (1 - w) * lim[:, :, j], rtol=1e-14)
    np.testing.assert_array_equal(out[:, 0], u[:, 0])          # averages untouched


def test_hybrid_is_plain_rkdg_when_nothing_is_troubled():
    # smooth, resolved data: every eta <= 1, so each stage keeps the unfiltered DG solution
    base = dict(dim=1, nx=160, x0=0.0, x1=2.0, k=2, eq=O.EQ_BURGERS, bc=(O.BC_PERIODIC,) * 4)
    ph = O.Problem(**base, filter=1, hybrid=1)
    pn = O.Problem(**base, filter=0)
    u0 = O.project(ph, O.IC_SINE, [0.5, 0.05, math.pi, 0.0])
    assert O.jump_indicator(ph, u0).max() < 1.0
    uh, th, nh = O.advance(ph, u0, 0.0, 0.2, 10 ** 6)
    un, tn, nn = O.advance(pn, u0, 0.0, 0.2, 10 ** 6)
    assert nh == nn and th == tn
    np.testing.assert_array_equal(uh, un)


def test_hybrid_shock_tube_stays_bounded():
    p = O.Problem(dim=1, nx=200, x0=0.0, x1=1.0, k=2, eq=O.EQ_EULER, bc=(O.BC_OUTFLOW,) * 4, hybrid=1)
    u0 = O.project(p, O.IC_RIEMANN1D, [1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 0.5])   # Sod
    u, t, n = O.advance(p, u0, 0.0, 0.2, 10 ** 6)
    assert t == 0.2
    rho = u[0, 0]
    assert rho.min() > 0.125 - 0.01 and rho.max() < 1.0 + 0.01
