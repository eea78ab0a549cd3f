"""Pins for the oracle's Im g(-t) (Appendix A) against the paper's own decomposition.

The oracle evaluates Im g(-t) by rotating the Fourier integral onto the imaginary
frequency axis.  These tests check it against a different route: the paper's
split g = g_1 + g_2 + delta g (Appendix A and A.1), with g_1 and g_2 transformed
in closed form as printed, and delta g transformed numerically by QUADPACK's
oscillatory Fourier routine (no cutoff), plus the small- and large-t limits.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import img_minus_t


def _g(xi, s):
    # Appendix A, first equation
    return -1j * xi * (1 + 1j * s / xi) * (1 + 1j * s / (2 * xi)) / np.sqrt(1 + 1j * s / xi)


def _paper_img(t, s):
    sqrt_i = np.exp(1j * math.pi / 4)
    g1 = lambda xi: xi / 1j + s                                  # large-xi limit
    g2 = lambda xi: sqrt_i / 2 * s**1.5 / np.sqrt(xi)            # small-xi limit
    # delta g -> -sigma as xi -> 0 (g - g_2 = O(xi^{1/2}))
    dg = lambda xi: (-s + 0j) if xi == 0.0 else _g(xi, s) - g1(xi) - g2(xi)
    re_part = quad(lambda x: dg(x).real, 0, np.inf, weight="sin", wvar=t, limlst=200)[0]
    im_part = quad(lambda x: dg(x).imag, 0, np.inf, weight="cos", wvar=t, limlst=200)[0]
    im_dg = (re_part + im_part) / (2 * math.pi)
    return im_dg + (1 / t**2 + s / t) / (2 * math.pi) + s**1.5 / (4 * math.sqrt(math.pi) * math.sqrt(t))


@pytest.mark.parametrize("sigma", [1.0, 10.0])
@pytest.mark.parametrize("t", [0.05, 0.3, 1.0, 3.0, 10.0])
def test_img_matches_paper_decomposition(t, sigma):
    ours = float(img_minus_t(np.array([t]), sigma)[0])
    ref = _paper_img(t, sigma)
    assert ours == pytest.approx(ref, rel=2e-7)


def test_img_small_t_limit_is_g1():
    # t -> 0: Im g(-t) - (1/2pi)(1/t^2 + sigma/t) grows only like t^{-1/2}
    for s in (0.5, 1.0, 3.0):
        t = np.array([1e-3, 1e-4, 1e-5])
        lead = (1 / t**2 + s / t) / (2 * math.pi)
        rel = np.abs(img_minus_t(t, s) / lead - 1.0)
        assert np.all(rel < 5 * t**1.5 * (1 + s) ** 1.5)
        assert rel[2] < rel[0]


def test_img_large_t_limit_is_g2():
    # t -> infinity: Im g(-t) -> sigma^{3/2} / (4 sqrt(pi) sqrt(t)), relative correction O(1/(sigma t))
    for s in (0.5, 1.0, 3.0):
        t = np.array([1e3, 1e4, 1e5]) / s
        lead = s**1.5 / (4 * math.sqrt(math.pi) * np.sqrt(t))
        rel = np.abs(img_minus_t(t, s) / lead - 1.0)
        assert np.all(rel < 2.0 / (s * t))
        assert rel[2] < rel[1] < rel[0]


def test_img_sigma_zero_is_massless_kernel():
    t = np.array([0.01, 0.1, 1.0])
    assert np.allclose(img_minus_t(t, 0.0), 1 / (2 * math.pi * t**2), rtol=1e-15)
    # continuity in sigma
    assert np.allclose(img_minus_t(t, 1e-8), 1 / (2 * math.pi * t**2), rtol=1e-6)


@pytest.mark.parametrize("t", [0.02, 0.5, 4.0])
def test_zinv_form_is_transform_of_minus_i_omega_g(t):
    # -i omega(xi) g(xi) = -(xi + i sigma)(xi + i sigma/2); on xi = i eta it is (eta+sigma)(eta+sigma/2)
    s = 1.3
    lap = quad(lambda e: (e + s) * (e + s / 2) * math.exp(-e * t), 0, np.inf, epsabs=0, epsrel=1e-13)[0] / (2 * math.pi)
    from oracle.casimir_oracle import ZINV_FACTOR
    ours = float(img_minus_t(np.array([t]), s, "zinv")[0])
    assert ours == pytest.approx(ZINV_FACTOR * lap, rel=1e-12)
    printed = (2 / t**3 + 1.5 * s / t**2 + 0.5 * s**2 / t) / (2 * math.pi)   # Appendix A.2 as printed
    assert lap == pytest.approx(printed, rel=1e-12)
