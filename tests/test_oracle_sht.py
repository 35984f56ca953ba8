"""Pins for the oracle's spherical-harmonic transforms (harmonic half of Fig. 1, spectra of Sec. 3)."""
import numpy as np
import pytest
from scipy.special import sph_harm_y

import oracle as O
from paper_1409_4441_gb300 import inputs


def test_lambda_matches_scipy_up_to_phase():
    lmax = 40
    th = np.array([0.01, 0.3, 1.0, 1.5707, 2.2, 3.1])
    lam = O.lambda_table(lmax, np.cos(th))
    for l in range(lmax + 1):
        for m in range(l + 1):
            ref = (sph_harm_y(l, m, th, 0.0) * (-1) ** m).real
            np.testing.assert_allclose(lam[:, O.alm_index(lmax, l, m)], ref, atol=1e-13)


@pytest.mark.parametrize("theta_deg", [0.05, 4.2, 30.0, 89.9])
def test_unsold_theorem_at_high_l(theta_deg):
    """sum_m |Y_lm|^2 = (2l+1)/(4 pi) at any point (up to the ~l*eps rounding of the
    forward recurrence): pins the normalisation and the scaled recurrence where
    lambda_mm underflows double precision."""
    lmax = 4096
    lam = O.lambda_table(lmax, [np.cos(np.radians(theta_deg))])[0]
    for l in (1, 100, 2048, 4096):
        v = lam[[O.alm_index(lmax, l, m) for m in range(l + 1)]]
        assert (v[0] ** 2 + 2 * np.sum(v[1:] ** 2)) / ((2 * l + 1) / (4 * np.pi)) == \
            pytest.approx(1.0, abs=1e-9)


def test_synthesis_of_single_harmonics():
    nside, lmax = 4, 8
    v = O.pix2vec(nside)
    th = np.arccos(np.clip(v[:, 2], -1, 1))
    phi = np.arctan2(v[:, 1], v[:, 0])
    for l, m in [(0, 0), (3, 0), (4, 1), (7, 5), (8, 8)]:
        alm = np.zeros(O.n_alm(lmax), complex)
        alm[O.alm_index(lmax, l, m)] = 0.3 - 0.7j if m else 0.9
        Y = sph_harm_y(l, m, th, phi) * (-1) ** m
        ref = (alm[O.alm_index(lmax, l, m)] * Y).real * (1 if m == 0 else 2)
        np.testing.assert_allclose(O.alm2map(nside, alm, lmax), ref, atol=1e-13)


@pytest.mark.parametrize("nside,lmax", [(4, 12), (8, 23)])
def test_addition_theorem_brute_equals_sht(nside, lmax):
    """The two oracle paths agree: with theta_cut = pi and K the full Legendre sum,
    sum_j K(theta_ij) m_j dOmega = alm2map(k_l map2alm(m)) to FP64 rounding."""
    m = inputs.white_noise_map(nside, 11)
    k = inputs.perturbed_coeffs(np.ones(lmax + 1), 0.5, 12)
    b, _ = O.brute_conv(nside, m, np.pi, c=k)
    s = O.sht_conv(nside, m, k)
    np.testing.assert_allclose(b, s, atol=1e-12 * np.abs(b).max())


def test_alm2cl_and_eps_cl_closed_forms():
    lmax = 5
    alm = np.zeros(O.n_alm(lmax), complex)
    alm[O.alm_index(lmax, 3, 0)] = 2.0
    alm[O.alm_index(lmax, 3, 2)] = 1.0 + 1.0j
    cl = O.alm2cl(alm, lmax)
    assert cl[3] == pytest.approx((4.0 + 2 * 2.0) / 7)
    assert np.count_nonzero(cl) == 1
    c = np.linspace(1, 2, 10)
    assert O.eps_cl(c * (1 + 3e-6), c) == pytest.approx(3e-6, rel=1e-9)


def test_grf_spectrum_statistics():
    """map2alm(alm2map(a)) recovers a band-limited field to the percent-level
    accuracy of HEALPix equal-weight quadrature, and alm2cl of the draw matches
    the input spectrum within cosmic variance."""
    nside, lmax = 32, 40
    cl = inputs.cl_grf(lmax)
    alm = inputs.grf_alm(lmax, cl, 21)
    mp = O.alm2map(nside, alm, lmax)
    back = O.map2alm(nside, mp, lmax)
    np.testing.assert_allclose(back, alm, atol=1e-2 * np.abs(alm).max())
    est = O.alm2cl(alm, lmax)
    ell = np.arange(lmax + 1)
    # sample variance of C_l is 2 C_l^2 / (2l+1): check the bulk within 5 sigma
    z = (est[2:] - cl[2:]) / (cl[2:] * np.sqrt(2.0 / (2 * ell[2:] + 1)))
    assert np.abs(z).max() < 5
