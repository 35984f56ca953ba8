"""Pins for the oracle's Legendre sums, kernel model and tabulated kernel (Eq. 1, Eq. 9)."""
import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss
from scipy.special import eval_legendre

import oracle as O
from paper_1409_4441_gb300 import inputs


def test_legendre_sum_matches_scipy():
    g = np.random.default_rng(0)
    c = g.standard_normal(81)
    z = np.concatenate([np.linspace(-1, 1, 11), [0.999999, -0.3]])
    ref = sum((2 * l + 1) / (4 * np.pi) * c[l] * eval_legendre(l, z) for l in range(81))
    np.testing.assert_allclose(O.legendre_sum(c, z), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_legendre_derivative_closed_form():
    # P'_l(z) = l (z P_l - P_{l-1}) / (z^2 - 1)
    g = np.random.default_rng(1)
    c = g.standard_normal(41)
    z = np.array([-0.7, -0.1, 0.2, 0.55, 0.9])
    dref = sum((2 * l + 1) / (4 * np.pi) * c[l] * l *
               (z * eval_legendre(l, z) - eval_legendre(l - 1, z)) / (z * z - 1)
               for l in range(1, 41))
    _, d = O.legendre_sum(c, z, deriv=True)
    np.testing.assert_allclose(d, dref, rtol=1e-11)


def test_unit_norm_and_transform_roundtrip():
    """int K dOmega = c_0 (unit-norm kernel when c_0 = 1), and
    2 pi int K P_l dz recovers c_l: the normalisation of the operator in Eq. 1."""
    lmax = 60
    c = inputs.perturbed_coeffs(O.gaussian_beam(lmax, np.radians(10.0)), 0.1, 3)
    x, w = leggauss(200)
    K = O.legendre_sum(c, x)
    assert 2 * np.pi * np.sum(w * K) == pytest.approx(c[0], rel=1e-13)
    P = O.legendre_matrix(lmax, x)
    np.testing.assert_allclose(2 * np.pi * (P.T @ (w * K)), c, atol=1e-12)


def test_gaussian_beam_closed_form_and_small_sigma_limit():
    fwhm = np.radians(1.0)
    sig = fwhm / np.sqrt(8 * np.log(2))
    b = O.gaussian_beam(2000, fwhm)
    assert b[0] == 1.0
    assert b[100] == pytest.approx(np.exp(-100 * 101 * sig * sig / 2), rel=1e-14)
    # real-space limit: K(theta) -> exp(-theta^2 / 2 sigma^2) / (2 pi sigma^2), O(sigma^2) error
    theta = np.array([0.0, 0.5, 1.0, 2.0]) * sig
    K = O.legendre_sum(b, np.cos(theta))
    ref = np.exp(-theta ** 2 / (2 * sig * sig)) / (2 * np.pi * sig * sig)
    np.testing.assert_allclose(K, ref, rtol=20 * sig * sig)


def test_hermite_table_interpolation_error():
    """The tabulated kernel (cubic Hermite in the chord) reproduces the Legendre sum
    to better than 1e-7 of its peak with ~100 intervals per l_max wavelength."""
    lmax = 1535
    fwhm = np.radians(20 / 60)
    tc = np.radians(90 / 60)
    c = O.gaussian_beam(lmax, fwhm)
    c[:257] = 0.0  # an oscillating high-pass real-space kernel
    dc = O.chord_cut(tc)
    n_int = int(np.ceil(96 * dc * lmax / (2 * np.pi)))
    tK, tD = O.hermite_nodes(c, tc, n_int)
    d = np.random.default_rng(5).uniform(0, dc, 20000)
    d = np.concatenate([d, [0.0, dc, dc * 1e-3]])
    exact = O.legendre_sum(c, 1 - d * d / 2)
    approx = O.hermite_eval(tK, tD, tc, d)
    assert np.abs(approx - exact).max() <= 1e-7 * np.abs(exact).max()
    # nodes are exact
    np.testing.assert_allclose(O.hermite_eval(tK, tD, tc, np.arange(n_int + 1) * dc / n_int),
                               tK, atol=1e-15 * np.abs(tK).max())
