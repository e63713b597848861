"""Pins for the oracle's regularised incomplete beta I_x(a,b) (Section 4.1,
"Inference"), checked against closed forms, exact rational arithmetic and two
independent libraries -- never against the oracle itself."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O


def exact_ibeta_int(a: int, b: int, x: Fraction) -> Fraction:
    """I_x(a,b) for integer shapes = Pr[Binomial(a+b-1, x) >= a], exactly."""
    n = a + b - 1
    return sum(Fraction(math.comb(n, j)) * x ** j * (1 - x) ** (n - j) for j in range(a, n + 1))


@pytest.mark.parametrize("x", [1e-9, 0.01, 0.3, 0.5, 0.7, 0.99, 1 - 1e-9])
def test_closed_forms(x):
    # I_x(1,1) = x ; I_x(a,1) = x^a ; I_x(1,b) = 1 - (1-x)^b
    assert O.ibeta(1, 1, x) == pytest.approx(x, rel=1e-14, abs=1e-300)
    for a in (2, 5, 33):
        assert O.ibeta(a, 1, x) == pytest.approx(x ** a, rel=1e-12, abs=1e-300)
        assert O.ibeta(1, a, x) == pytest.approx(-math.expm1(a * math.log1p(-x)), rel=1e-12, abs=1e-300)


def test_endpoints_and_symmetry():
    assert O.ibeta(3, 4, 0.0) == 0.0 and O.ibeta(3, 4, 1.0) == 1.0
    for a, b, x in [(3.5, 7.25, 0.2), (40, 12, 0.8), (200, 300, 0.41)]:
        assert O.ibeta(a, b, x) + O.ibeta(b, a, 1 - x) == pytest.approx(1.0, abs=1e-14)


@pytest.mark.parametrize("a,b", [(1, 1), (2, 3), (18, 15), (33, 1), (1, 33), (24, 9), (40, 40), (60, 5)])
def test_exact_binomial_tail(a, b):
    for xf in (0.05, 0.3, 0.5, 0.7, 1 - 0.7, 0.95):
        x = Fraction(xf)                       # the exact binary value of the double
        want = exact_ibeta_int(a, b, x)
        got = Fraction(O.ibeta(a, b, xf))
        if want > Fraction(1, 10 ** 200):
            assert abs(got - want) <= Fraction(1, 10 ** 13) * want + Fraction(1, 10 ** 300)


def test_small_tails_have_relative_accuracy():
    # 1 - I_0.5(1, 65) = 2^-65: never evaluated as 1 - (something near 1)
    assert O.ibeta(65, 1, 0.5) == pytest.approx(2.0 ** -65, rel=1e-13)
    want = exact_ibeta_int(3, 200, Fraction(0.3))
    got = O.ibeta(3, 200, 0.3)
    assert float(want) == pytest.approx(got, rel=1e-12)


def test_against_mpmath_large_shapes():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    rng = np.random.default_rng(0)
    for _ in range(150):
        n = int(rng.integers(32, 2049))
        m = int(rng.integers(0, n + 1))
        a, b = m + 1.0, n - m + 1.0
        x = float(rng.choice([0.5, 1 - 0.7468, 0.2, rng.random()]))
        want = mp.betainc(a, b, 0, x, regularized=True)
        got = O.ibeta(a, b, x)
        if want > mp.mpf("1e-290"):
            assert abs(mp.mpf(got) - want) <= mp.mpf("1e-11") * want + mp.mpf("1e-15") * (1 - want)
        lg = O.log_ibeta(a, b, x)
        if want > 0:
            assert abs(lg - float(mp.log(want))) <= 1e-10 * max(1.0, abs(lg))


def test_against_scipy_nonint_shapes():
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(1)
    for _ in range(300):
        a = float(rng.uniform(0.3, 300)); b = float(rng.uniform(0.3, 300)); x = float(rng.random())
        want = float(sp.betainc(a, b, x))
        assert O.ibeta(a, b, x) == pytest.approx(want, rel=1e-10, abs=1e-14)
