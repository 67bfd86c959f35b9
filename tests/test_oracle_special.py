"""Pins of the oracle's b_n, incomplete gamma and Sersic flux.

b_n is defined by gamma(2n, b_n) = Gamma(2n)/2 so that the effective radius
encloses half of the light (Sec. 2's "effective radius" extraction).
"""
import math

import numpy as np
import pytest

import oracle


def test_bn_half_exact():
    # n = 1/2: P(1, b) = 1 - e^{-b} = 1/2  ->  b = ln 2
    assert abs(oracle.bn(0.5) - math.log(2.0)) < 1e-15


def test_bn_one_closed_form():
    # n = 1: P(2, b) = 1 - (1 + b) e^{-b} = 1/2
    b = oracle.bn(1.0)
    assert abs((1.0 + b) * math.exp(-b) - 0.5) < 1e-15
    assert abs(b - 1.678346990016661) < 1e-14


@pytest.mark.parametrize("n", [0.2, 0.5, 0.8, 1.0, 1.5, 2.0, 3.0, 4.0, 5.5, 6.0, 8.0, 10.0])
def test_bn_matches_library_inverse(n):
    from scipy.special import gammaincinv
    assert abs(oracle.bn(n) - gammaincinv(2.0 * n, 0.5)) < 1e-13 * max(1.0, n)


@pytest.mark.parametrize("n", [1.0, 1.5, 2.0, 4.0, 8.0, 10.0])
def test_bn_asymptotic_series(n):
    # Ciotti & Bertin (1999) asymptotic expansion to O(n^-2); the remainder is
    # bounded by the size of its next term, 131 / (1148175 n^3)
    cb = 2 * n - 1.0 / 3 + 4.0 / (405 * n) + 46.0 / (25515 * n * n)
    assert abs(oracle.bn(n) - cb) < 131.0 / (1148175.0 * n ** 3)


@pytest.mark.parametrize("a,x", [(0.4, 0.1), (1.0, 0.7), (2.0, 3.0), (8.0, 7.5),
                                 (12.0, 20.0), (20.0, 19.0), (3.3, 0.01)])
def test_gammainc_matches_library(a, x):
    from scipy.special import gammainc
    assert abs(oracle.gammainc_lower(a, x) - gammainc(a, x)) < 1e-14


def test_gammainc_exponential_case():
    # P(1, x) = 1 - e^{-x}
    for x in [0.01, 0.5, 2.0, 9.0]:
        assert abs(oracle.gammainc_lower(1.0, x) - (1.0 - math.exp(-x))) < 1e-15


def test_sersic_flux_closed_form_values():
    # n = 1/2 is a Gaussian: I = 2 I_e exp(-ln2 r^2/r_e^2), flux = 2 I_e pi q r_e^2 / ln 2
    Ie, re, q = 1.3, 5.0, 0.6
    F = oracle.sersic_flux(Ie, re, 0.5, q)
    assert abs(F - 2 * Ie * math.pi * q * re * re / math.log(2.0)) < 1e-12 * F
    # n = 1 is an exponential disk: I_0 = I_e e^{b_1}, r_s = r_e / b_1, flux 2 pi q I_0 r_s^2
    b1 = oracle.bn(1.0)
    F1 = oracle.sersic_flux(Ie, re, 1.0, q)
    assert abs(F1 - 2 * math.pi * q * Ie * math.exp(b1) * (re / b1) ** 2) < 1e-12 * F1
    # the 64x64 workload's component: n=4, r_e=8, q=0.7, I_e=1
    assert abs(oracle.sersic_flux(1.0, 8.0, 4.0, 0.7) - 1015.402470816) < 1e-8
