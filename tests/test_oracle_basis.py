"""Pins for the oracle's basis layer (Eq. GLbasisequation, Eq. eqn:SL).

Each check compares the oracle against mathematics that does not depend on its code: closed-form
Gauss rules, the closed form of Legendre endpoint derivatives, the Sturm–Liouville identity, and
the Legendre norms.
"""
import math

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.filterwarnings("ignore")


GAUSS_CLOSED = {
    1: ([0.0], [2.0]),
    2: ([-1 / math.sqrt(3), 1 / math.sqrt(3)], [1.0, 1.0]),
    3: ([-math.sqrt(3 / 5), 0.0, math.sqrt(3 / 5)], [5 / 9, 8 / 9, 5 / 9]),
    4: (
        [-math.sqrt(3 / 7 + 2 / 7 * math.sqrt(6 / 5)), -math.sqrt(3 / 7 - 2 / 7 * math.sqrt(6 / 5)),
         math.sqrt(3 / 7 - 2 / 7 * math.sqrt(6 / 5)), math.sqrt(3 / 7 + 2 / 7 * math.sqrt(6 / 5))],
        [(18 - math.sqrt(30)) / 36, (18 + math.sqrt(30)) / 36, (18 + math.sqrt(30)) / 36,
         (18 - math.sqrt(30)) / 36],
    ),
    5: (
        [-1 / 3 * math.sqrt(5 + 2 * math.sqrt(10 / 7)), -1 / 3 * math.sqrt(5 - 2 * math.sqrt(10 / 7)), 0.0,
         1 / 3 * math.sqrt(5 - 2 * math.sqrt(10 / 7)), 1 / 3 * math.sqrt(5 + 2 * math.sqrt(10 / 7))],
        [(322 - 13 * math.sqrt(70)) / 900, (322 + 13 * math.sqrt(70)) / 900, 128 / 225,
         (322 + 13 * math.sqrt(70)) / 900, (322 - 13 * math.sqrt(70)) / 900],
    ),
}


@pytest.mark.parametrize("n", sorted(GAUSS_CLOSED))
def test_gauss_rules_match_closed_forms(n):
    x, w = O.gauss(n)
    xe, we = GAUSS_CLOSED[n]
    np.testing.assert_allclose(x, xe, rtol=0, atol=2e-16 * 4)
    np.testing.assert_allclose(w, we, rtol=0, atol=4e-16 * 4)


@pytest.mark.parametrize("n", range(1, 13))
def test_gauss_rule_integrates_monomials_exactly(n):
    # an n-point rule is exact for degree 2n-1: int x^d = 2/(d+1) for even d, 0 for odd d
    x, w = O.gauss(n)
    for d in range(2 * n):
        exact = 2.0 / (d + 1) if d % 2 == 0 else 0.0
        assert abs(np.dot(w, x ** d) - exact) < 1e-14


@pytest.mark.parametrize("l", range(0, 5))
@pytest.mark.parametrize("m", range(0, 5))
def test_endpoint_derivatives_closed_form(l, m):
    # P_l^{(m)}(1) = (l+m)! / (2^m m! (l-m)!), P_l^{(m)}(-1) = (-1)^{l+m} times that (0 for m > l)
    if m > l:
        expect = 0.0
    else:
        expect = math.factorial(l + m) / (2 ** m * math.factorial(m) * math.factorial(l - m))
    assert O.legendre_deriv(l, m, 1.0) == pytest.approx(expect, abs=1e-13)
    assert O.legendre_deriv(l, m, -1.0) == pytest.approx((-1) ** (l + m) * expect, abs=1e-13)


def test_named_endpoint_values():
    assert O.legendre_deriv(3, 3, 1.0) == pytest.approx(15.0)
    # P_3 = (5x^3 - 3x)/2 has the constant third derivative 15, so the value at -1 is +15 as well
    assert O.legendre_deriv(3, 3, -1.0) == pytest.approx(15.0)
    assert O.legendre_deriv(4, 4, 1.0) == pytest.approx(105.0)
    for l in range(6):
        assert O.legendre(l, 1.0) == pytest.approx(1.0)
        assert O.legendre(l, -1.0) == pytest.approx((-1) ** l)


@pytest.mark.parametrize("l", range(0, 6))
def test_sturm_liouville_identity(l):
    # d/dxi ((1 - xi^2) P_l') + l(l+1) P_l = 0 (Eq. eqn:SL), i.e. (1-x^2)P'' - 2x P' + l(l+1) P = 0
    rng = np.random.default_rng(7 + l)
    for x in rng.uniform(-1, 1, 9):
        lhs = (1 - x * x) * O.legendre_deriv(l, 2, x) - 2 * x * O.legendre_deriv(l, 1, x) \
            + l * (l + 1) * O.legendre(l, x)
        assert abs(lhs) < 1e-12


@pytest.mark.parametrize("l", range(0, 6))
def test_legendre_norms_and_values(l):
    assert O.legendre_norm(l) == pytest.approx(2.0 / (2 * l + 1), rel=1e-14)
    # value recurrence vs derivative-of-monomial form (two independent code paths in the oracle)
    for x in (-0.9, -0.3, 0.1, 0.77):
        assert O.legendre(l, x) == pytest.approx(O.legendre_deriv(l, 0, x), abs=1e-14)
