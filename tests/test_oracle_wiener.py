"""Noise-dominated (Wiener-weighted) splits (Sec. 2, Eq. 2: for Wiener filtering the input
spectrum weighting the fit is C_l^2 / (C_l + N)).  Where noise dominates, the high-l part of
the kernel carries little output power, so the Sec. 2 scan finds splits at least as cheap at
the same Eq. 6 bound; the weighted fit is also checked to minimise its own Eq. 2 residual."""
import numpy as np

import oracle as O
from paper_1409_4441_gb300 import inputs


def _wiener(lmax, noise):
    c = inputs.cl_grf(lmax)
    return c * c / (c + noise)


def test_wiener_weighting_fits_its_own_residual_best():
    lmax, lcut, tc = 383, 64, np.radians(3.0)
    b = O.gaussian_beam(lmax, np.radians(1.0))
    cw = _wiener(lmax, 1e-7)
    sw = O.split_lsq(b, lcut, tc, cl_in=cw)
    sf = O.split_lsq(b, lcut, tc, cl_in=None)
    # each fit is best under its own weighting (up to the SVD truncation)
    assert O.sigma_rms(b, sw["K_tilde"], cw) <= 1.05 * O.sigma_rms(b, sf["K_tilde"], cw)
    assert O.sigma_rms(b, sf["K_tilde"]) <= 1.05 * O.sigma_rms(b, sw["K_tilde"])


def test_noise_dominated_scan_is_no_more_expensive():
    lmax = 255
    b = O.gaussian_beam(lmax, np.radians(1.5))
    grid = np.radians(np.array([180, 270, 360, 450]) / 60)
    c_signal = inputs.cl_grf(lmax)
    c_wiener = _wiener(lmax, 1e-6)   # noise above signal from l ~ 1000 / 10 ~ 100
    best_s, _ = O.scan_split(b, grid, bound=1e-3, cl_in=c_signal)
    best_w, _ = O.scan_split(b, grid, bound=1e-3, cl_in=c_wiener)
    assert best_w is not None
    if best_s is not None:
        assert best_w[3] <= best_s[3]
