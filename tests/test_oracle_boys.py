"""Pins of the oracle's Boys function (HJO Sec. 9.8) to closed forms and quadrature."""
import math

import numpy as np
import pytest

import oracle


def quad_boys(m, T, n=120):
    x, w = np.polynomial.legendre.leggauss(n)
    t = 0.5 * (x + 1.0)
    return 0.5 * np.sum(w * t ** (2 * m) * np.exp(-T * t * t))


@pytest.mark.parametrize("T", [1e-12, 1e-3, 0.3, 1.7, 5.0, 12.5, 29.9, 39.99, 40.01, 55.0, 120.0, 800.0])
def test_f0_closed_form(T):
    F = oracle.boys(0, T)
    ref = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    assert abs(F[0] - ref) <= 2e-15 * max(1.0, ref)


def test_at_zero():
    F = oracle.boys(16, 0.0)
    assert np.allclose(F, 1.0 / (2 * np.arange(17) + 1), rtol=0, atol=1e-15)


@pytest.mark.parametrize("T", [0.05, 0.9, 3.3, 8.0, 17.0, 33.0, 41.0, 60.0])
def test_against_quadrature(T):
    F = oracle.boys(12, T)
    for m in range(13):
        ref = quad_boys(m, T)
        assert abs(F[m] - ref) <= 1e-13 * ref, (m, T, F[m], ref)


@pytest.mark.parametrize("T", [0.05, 3.3, 17.0, 39.5, 41.0, 75.0])
def test_against_arbitrary_precision(T):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    F = oracle.boys(12, T)
    for m in range(13):
        ref = mp.quad(lambda t: t ** (2 * m) * mp.e ** (-T * t * t), [0, 1])
        assert abs(F[m] - float(ref)) <= 2e-15 * float(ref), (m, T)


@pytest.mark.parametrize("T", [0.2, 6.0, 25.0, 45.0])
def test_recursion_identity(T):
    F = oracle.boys(10, T)
    for m in range(1, 11):
        # (2m-1) F_{m-1} = 2T F_m + exp(-T)
        assert abs((2 * m - 1) * F[m - 1] - (2 * T * F[m] + math.exp(-T))) < 1e-14


def test_large_t_asymptote():
    T = 200.0
    F = oracle.boys(8, T)
    for m in range(9):
        ref = math.prod(range(2 * m - 1, 0, -2)) / 2 ** (m + 1) * math.sqrt(math.pi / T ** (2 * m + 1))
        assert abs(F[m] / ref - 1.0) < 1e-13
