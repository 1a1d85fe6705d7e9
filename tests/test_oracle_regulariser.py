"""The oracle's DSRG regulariser against an extended-precision evaluation.

Eqs. T1_1st and T2_1st scale every amplitude by R_s(D) = (1 - exp(-s D^2)) / D,
whose limit at D = 0 is 0.  The oracle evaluates it as -expm1(-s D^2) / D and
switches to the series s D (1 - s D^2 / 2) below s D^2 = 1e-12.  Here both
branches and the switch point are compared with the definition evaluated in
60-digit arithmetic (mpmath), so a wrong sign, a dropped series term or a
switch on the wrong side shows up as more than a few ulps of error.
"""
import numpy as np
import pytest

from oracle.dsrg import regulariser

mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 60

EPS = np.finfo(np.float64).eps


def _exact(s, D):
    """(1 - exp(-s D^2)) / D with 60 significant digits (0 at D = 0)."""
    if D == 0.0:
        return mpmath.mpf(0)
    s_, D_ = mpmath.mpf(float(s)), mpmath.mpf(float(D))
    return (1 - mpmath.exp(-s_ * D_ * D_)) / D_


def _grid(s):
    # magnitudes from 1e-12 to 50, every decade plus points straddling the
    # series switch s D^2 = 1e-12 (D* = 1e-6 / sqrt(s)) and the scale 1/sqrt(s)
    mags = list(np.logspace(-12, np.log10(50.0), 73))
    dstar = 1e-6 / np.sqrt(s)
    mags += [dstar * f for f in (0.5, 0.999999, 1.0, 1.000001, 2.0)]
    mags += [f / np.sqrt(s) for f in (0.1, 0.5, 1.0, 2.0, 6.0)]
    mags += [np.nextafter(dstar, 0.0), np.nextafter(dstar, 1.0)]
    return np.array(sorted(set(mags)))


@pytest.mark.parametrize("s", [0.5, 1e6, 1e-3])
def test_regulariser_matches_extended_precision(s):
    mags = _grid(s)
    D = np.concatenate([mags, -mags])
    got = regulariser(s, D)
    for d, g in zip(D, got):
        want = _exact(s, d)
        if want == 0:
            assert g == 0.0
            continue
        rel = abs((mpmath.mpf(float(g)) - want) / want)
        assert rel < 4 * EPS, (s, d, float(g), float(want), float(rel))


@pytest.mark.parametrize("s", [0.5, 1e6])
def test_regulariser_limit_and_symmetry(s):
    """R(0) = 0 exactly, R is odd, and R(D) -> s D for small D."""
    assert regulariser(s, np.array([0.0]))[0] == 0.0
    assert regulariser(s, np.array([-0.0]))[0] == 0.0
    D = np.array([1e-12, 3e-10, 7e-9, 1e-7, 0.3, 5.0])
    np.testing.assert_array_equal(regulariser(s, -D), -regulariser(s, D))
    tiny = np.array([1e-14, 1e-13])
    np.testing.assert_allclose(regulariser(s, tiny), s * tiny, rtol=4 * EPS)


def test_regulariser_large_s_is_one_over_d():
    """s -> infinity (Eq. T2_1st without regularisation): R = 1/D away from 0."""
    D = np.array([0.05, 0.7, 3.0, 42.0])
    np.testing.assert_allclose(regulariser(1e12, D), 1.0 / D, rtol=EPS)
