"""Pins of the oracle's Boys function F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt.

Pinned against (1) mpmath's incomplete gamma function at 30 digits,
F_m(T) = gamma(m + 1/2, 0..T) / (2 T^{m+1/2}); (2) the closed forms
F_m(0) = 1/(2m+1) and F_0(T) = (1/2) sqrt(pi/T) erf(sqrt T); (3) the
recursion identity (2m+1) F_m = 2T F_{m+1} + exp(-T) on both sides of the
oracle's series / asymptotic switch at T = 30.
"""
import math

import numpy as np
import pytest

import oracle

mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 30

T_GRID = [0.0, 1e-12, 1e-6, 0.01, 0.3, 1.0, 2.5, 7.0, 12.0, 20.0, 29.999, 30.0, 30.001,
          35.0, 50.0, 117.0, 1000.0, 1e5]


def boys_mp(m, T):
    if T == 0:
        return mpmath.mpf(1) / (2 * m + 1)
    T = mpmath.mpf(T)
    return mpmath.gammainc(m + mpmath.mpf(1) / 2, 0, T) / (2 * T ** (m + mpmath.mpf(1) / 2))


@pytest.mark.parametrize("T", T_GRID)
def test_boys_vs_mpmath(T):
    mmax = 16
    F = oracle.boys(mmax, T)
    for m in range(mmax + 1):
        ref = float(boys_mp(m, T))
        assert F[m] == pytest.approx(ref, rel=2e-14, abs=0.0), (m, T)


def test_boys_at_zero():
    F = oracle.boys(16, 0.0)
    for m in range(17):
        assert F[m] == pytest.approx(1.0 / (2 * m + 1), rel=1e-15)


@pytest.mark.parametrize("T", [1e-3, 0.5, 3.0, 29.0, 31.0, 80.0])
def test_boys_f0_erf(T):
    F = oracle.boys(0, T)
    assert F[0] == pytest.approx(0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T)), rel=1e-14)


@pytest.mark.parametrize("T", [0.2, 5.0, 29.5, 30.5, 60.0])
def test_boys_recursion_identity(T):
    F = oracle.boys(12, T)
    e = math.exp(-T)
    for m in range(12):
        lhs = (2 * m + 1) * F[m]
        rhs = 2 * T * F[m + 1] + e
        assert lhs == pytest.approx(rhs, rel=1e-14)


def test_boys_monotone_in_m_and_T():
    Ts = np.linspace(0.0, 60.0, 241)
    prev = None
    for T in Ts:
        F = oracle.boys(10, T)
        assert np.all(np.diff(F) < 0)
        if prev is not None:
            assert np.all(F <= prev)
        prev = F
