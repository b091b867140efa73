"""Pins for the oracle's Zhang–Shu positivity-preserving limiter (applied after the jump filter, as
the paper does in Section 3.2): closed-form scaling factors on hand-built cells, unchanged averages,
identity on admissible cells, admissibility afterwards, and a near-vacuum double rarefaction."""
import numpy as np
import pytest

import oracle as O


def one_cell(k=1):
    return O.Problem(dim=1, nx=1, x0=0.0, x1=0.1, k=k, eq=O.EQ_EULER, bc=(O.BC_PERIODIC,) * 4, positivity=1)


def test_density_scaling_closed_form():
    p = one_cell(1)
    u = np.zeros(p.shape)
    u[0, :, 0] = [1.0, 1.5]          # rho(-1) = -0.5
    u[2, 0, 0] = 2.5
    out = O.positivity(p, u)
    eps_r = 1e-3 * 1.0                 # the density margin: 1e-3 of the cell average
    theta1 = (1.0 - eps_r) / (1.0 - (-0.5))
    assert out[0, 1, 0] == pytest.approx(1.5 * theta1, rel=1e-14)
    assert out[0, 0, 0] == u[0, 0, 0] and out[2, 0, 0] == u[2, 0, 0]


@pytest.mark.parametrize("dim", [1, 2])
def test_lobatto_midline_points_closed_form(dim):
    # k = 3: rho = 1 + 2.5 P_2(x) is -0.25 at x = 0 but positive at the 4 Gauss nodes (0.18 at
    # +-0.34, 2.3 at +-0.86) and at the ends (3.5). Zhang and Shu's set takes the 3-point
    # Gauss-Lobatto node 0 as well (2N - 3 >= k), so the limiter acts: theta_1 = (1 - eps_r) / 1.25
    # with the density margin eps_r = 1e-3 rho_bar = 1e-3.
    if dim == 1:
        p = O.Problem(dim=1, nx=1, x0=0.0, x1=0.1, k=3, eq=O.EQ_EULER, bc=(O.BC_PERIODIC,) * 4, positivity=1)
    else:
        p = O.Problem(dim=2, nx=1, ny=1, x0=0.0, x1=0.1, y0=0.0, y1=0.1, k=3, eq=O.EQ_EULER,
                      bc=(O.BC_PERIODIC,) * 4, positivity=1)
    u = np.zeros(p.shape)
    u[0, 0, 0] = 1.0
    u[0, 2, 0] = 2.5                 # mode 2 = P_2(x) (P_0(y) in 2D)
    u[-1, 0, 0] = 2.5                # E = 2.5 at rest: p = 1 everywhere
    xs, _ = O.gauss(4)
    assert min(1.0 + 2.5 * (1.5 * x * x - 0.5) for x in xs) > 0.0
    out = O.positivity(p, u)
    theta1 = (1.0 - 1e-3) / 1.25
    assert out[0, 2, 0] == pytest.approx(2.5 * theta1, rel=1e-14)
    assert O.evaluate(p, out, 0, 0.0, 0.3)[0] == pytest.approx(1e-3, abs=1e-14)


def test_pressure_scaling_closed_form():
    p = one_cell(1)
    u = np.zeros(p.shape)
    u[0, 0, 0] = 1.0
    u[2, :, 0] = [2.5, 3.0]          # E(-1) = -0.5 -> p < 0 at the left end only
    out = O.positivity(p, u)
    # the pressure margin: min(1e-3 (rho_bar + |E_bar|), rho_bar, p_bar) = 1e-3 (1 + 2.5)
    eps = 1e-3 * 3.5
    # p(u_bar + t d) = 0.4 (2.5 - 3 t) = eps  ->  t = (2.5 - eps / 0.4) / 3
    theta2 = (2.5 - eps / 0.4) / 3.0
    assert out[2, 1, 0] == pytest.approx(3.0 * theta2, rel=1e-12)


@pytest.mark.parametrize("dim,k", [(1, 2), (1, 3), (2, 1), (2, 2), (2, 3)])
def test_limited_state_is_admissible_and_conservative(dim, k):
    rng = np.random.default_rng(10 * dim + k)
    if dim == 1:
        p = O.Problem(dim=1, nx=40, k=k, eq=O.EQ_EULER, positivity=1)
        avg = [(0.2, 1.0), (-0.3, 0.3), (0.5, 2.0)]
    else:
        p = O.Problem(dim=2, nx=8, ny=6, k=k, eq=O.EQ_EULER, positivity=1)
        avg = [(0.2, 1.0), (-0.3, 0.3), (-0.3, 0.3), (0.5, 2.0)]
    u = np.zeros(p.shape)
    for v, (lo, hi) in enumerate(avg):
        u[v, 0] = rng.uniform(lo, hi, p.ncell)
        u[v, 1:] = rng.uniform(-1.0, 1.0, (p.nmodes - 1, p.ncell))   # wild: many bad points
    out = O.positivity(p, u)
    np.testing.assert_array_equal(out[:, 0], u[:, 0])
    nq = k + 1
    xs, _ = O.gauss(nq)
    # Zhang and Shu's set: Gauss nodes crossed with the N-point Gauss-Lobatto nodes, 2N - 3 >= k
    # (N = 2: the ends; N = 3: the ends and 0), plus the volume Gauss points of the scheme
    lob = [-1.0, 1.0] if 2 * 2 - 3 >= k else [-1.0, 0.0, 1.0]
    if dim == 1:
        pts = [(x, 0.0) for x in list(xs) + lob]
    else:
        pts = [(a, b) for a in xs for b in xs] + [(s, x) for x in xs for s in lob] + \
            [(x, s) for x in xs for s in lob]
    for c in range(p.ncell):
        ub = out[:, 0, c]
        pbar = 0.4 * (ub[-1] - 0.5 * sum(ub[i] ** 2 for i in range(1, len(ub) - 1)) / ub[0])
        eps_r = 1e-3 * ub[0]                                        # the margins, per cell
        eps_p = min(1e-3 * (ub[0] + abs(ub[-1])), ub[0], pbar)
        for (xi, eta) in pts:
            val = O.evaluate(p, out, c, xi, eta)
            rho = val[0]
            E = val[-1]
            mom2 = sum(val[i] ** 2 for i in range(1, len(val) - 1))
            pr = 0.4 * (E - 0.5 * mom2 / rho)
            assert rho >= eps_r * (1 - 1e-9) and pr >= eps_p * (1 - 1e-9) - 1e-12


def test_identity_on_admissible_cells():
    p = O.Problem(dim=2, nx=5, ny=4, k=2, eq=O.EQ_EULER, positivity=1)
    u = O.project(p, O.IC_VORTEX2D, [0.5, 0.4, 1.0, 0.0])
    np.testing.assert_array_equal(O.positivity(p, u), u)


def test_quadrant_riemann_needs_the_limiter():
    # seeded four-quadrant data (seed 3, rejected by the unlimited screening): the unlimited Q2
    # scheme loses positivity within a few steps, the limited one reaches T with admissible averages
    from paper_2407_19169_gb300 import inputs as I
    prm = I.quadrant_params(3)
    base = dict(dim=2, nx=24, ny=24, k=2, eq=O.EQ_EULER, bc=(O.BC_OUTFLOW,) * 4)
    p0 = O.Problem(**base)
    with pytest.raises(FloatingPointError):
        O.advance(p0, O.project(p0, O.IC_QUADRANT2D, prm), 0.0, 0.1)
    p1 = O.Problem(**base, positivity=1)
    u, t, n = O.advance(p1, O.project(p1, O.IC_QUADRANT2D, prm), 0.0, 0.1)
    assert t == 0.1 and O.check_physical(p1, u)


def test_rate_takes_the_limiters_points_closed_form():
    # rho = 1 + 0.6 P_1 at rest with constant E: p = 0.4 E everywhere and the sound speed
    # sqrt(gamma p / rho) is largest where rho is smallest, at the left end (rho = 0.4).
    h = 0.1
    on = O.Problem(dim=1, nx=1, x0=0.0, x1=h, k=1, eq=O.EQ_EULER, bc=(O.BC_PERIODIC,) * 4, positivity=1)
    off = O.Problem(dim=1, nx=1, x0=0.0, x1=h, k=1, eq=O.EQ_EULER, bc=(O.BC_PERIODIC,) * 4, positivity=0)
    u = np.zeros(on.shape)
    u[0, :, 0] = [1.0, 0.6]
    u[2, 0, 0] = 2.5
    assert O.max_rate(off, u) == pytest.approx(np.sqrt(1.4 * 1.0 / 1.0) / h, rel=1e-14)
    assert O.max_rate(on, u) == pytest.approx(np.sqrt(1.4 * 1.0 / 0.4) / h, rel=1e-14)


def test_rate_2d_corner_edge_point():
    # 2D: rho = 1 + 0.3 P_1(x) + 0.3 P_1(y) at rest, E = 2.5: on the edges the Gauss points of the
    # left/bottom edges reach rho = 1 - 0.3 - 0.3 / sqrt(3); the volume points stay above that.
    on = O.Problem(dim=2, nx=1, ny=1, x0=0.0, x1=0.1, y0=0.0, y1=0.2, k=1, eq=O.EQ_EULER,
                   bc=(O.BC_PERIODIC,) * 4, positivity=1)
    u = np.zeros(on.shape)
    u[0, 0, 0], u[0, 1, 0], u[0, 2, 0] = 1.0, 0.3, 0.3     # modes (0,0), (1,0), (0,1)
    u[3, 0, 0] = 2.5
    rmin = 1.0 - 0.3 - 0.3 / np.sqrt(3.0)
    c = np.sqrt(1.4 * 1.0 / rmin)
    assert O.max_rate(on, u) == pytest.approx(c / 0.1 + c / 0.2, rel=1e-14)
