"""Accuracy of the dphi weight tables of the cap gather (the `exact_weights = 0` default).

For a fixed ring pair the kernel weight depends on the pixel pair only through
x = dphi / 2: w(x) = K(u(x)) with u^2 = A + B sin^2 x in K_r-table units.  The library
tabulates w in cubic Hermite cells of width dx = rho / max|du/dx| (rho = 2 table intervals,
stretched up to 3 where a ring pair needs more cells than a CTA holds).  This checks, with an
independent numpy construction on a high-passed Gaussian-beam kernel (Legendre sum, Sec. 2's
K_r shape), that interpolating the K_r table that way stays within the bound the header
states: at most 3e-7 of the kernel's peak, rms about 1e-8, over ring-pair geometries from
the same ring (A = 0) to pairs near the cut and whole-ring windows.
"""
import numpy as np
import pytest

LMAX, LCUT, FWHM = 1024, 256, np.radians(20.0 / 60.0)
THETA_CUT = np.radians(16.0)


def _kernel_nodes(n_int):
    """K and dK/du (per table interval) at the n_int + 1 table nodes uniform in chord."""
    ell = np.arange(LMAX + 1)
    sig = FWHM / np.sqrt(8 * np.log(2))
    b = np.exp(-0.5 * ell * (ell + 1) * sig ** 2)
    b[: LCUT + 1] = 0.0
    coef = (2 * ell + 1) / (4 * np.pi) * b
    dc = 2 * np.sin(THETA_CUT / 2)
    d = np.arange(n_int + 1.0) * dc / n_int
    z = 1 - 0.5 * d * d
    p0, p1 = np.ones_like(z), z.copy()
    q0, q1 = np.zeros_like(z), np.ones_like(z)  # P'_l(z)
    K = coef[0] * p0 + coef[1] * p1
    dK = coef[1] * q1
    for l in range(2, LMAX + 1):
        p2 = ((2 * l - 1) * z * p1 - (l - 1) * p0) / l
        q2 = q0 + (2 * l - 1) * p1
        K += coef[l] * p2
        dK += coef[l] * q2
        p0, p1, q0, q1 = p1, p2, q1, q2
    return K, dK * (-d) * dc / n_int, dc


def _hermite(y0, y1, d0, d1, f):
    return ((2 * f ** 3 - 3 * f ** 2 + 1) * y0 + (f ** 3 - 2 * f ** 2 + f) * d0
            + (-2 * f ** 3 + 3 * f ** 2) * y1 + (f ** 3 - f ** 2) * d1)


def _table(Kn, dKn, n_int, u):
    """The K_r table (cubic Hermite in u), the last cell extrapolated past the cut."""
    i = np.clip(np.floor(u).astype(int), 0, n_int - 1)
    f = u - i
    y0, y1, d0, d1 = Kn[i], Kn[i + 1], dKn[i], dKn[i + 1]
    val = _hermite(y0, y1, d0, d1, f)
    der = ((6 * f ** 2 - 6 * f) * y0 + (3 * f ** 2 - 4 * f + 1) * d0
           + (-6 * f ** 2 + 6 * f) * y1 + (3 * f ** 2 - 2 * f) * d1)
    return val, der


@pytest.mark.parametrize("rho,max_bound,rms_bound", [(2.0, 1e-7, 1e-8), (3.0, 3e-7, 2.5e-8)])
def test_dphi_table_error_within_header_bound(rho, max_bound, rms_bound):
    # the library's automatic table size: about 96 intervals per shortest l_max wavelength
    n_int = int(np.ceil(96.0 * 2 * np.sin(THETA_CUT / 2) * LMAX / (2 * np.pi)))
    Kn, dKn, dc = _kernel_nodes(n_int)
    peak = np.abs(Kn).max()
    sc2 = (n_int / dc) ** 2
    rng = np.random.default_rng(7)
    worst_max = worst_rms = 0.0
    # (ring separation, sin theta of both rings): same ring, neighbours, near the cut,
    # and a ring near the pole whose window is the whole ring
    for dth, st in [(0.0, 0.5), (np.radians(2.0), 0.5), (np.radians(12.0), 0.7),
                    (0.0, 0.05), (np.radians(1.0), 0.1)]:
        A = (2 * np.sin(dth / 2)) ** 2 * sc2
        B = 4 * st * st * sc2
        sx2 = (n_int ** 2 - A) / B
        xc = np.pi / 2 if sx2 >= 1 else np.arcsin(np.sqrt(sx2))
        xs = np.linspace(0, xc, 4001)
        us = np.sqrt(A + B * np.sin(xs) ** 2)
        dmax = np.max(B * np.sin(xs) * np.cos(xs) / np.maximum(us, 1e-30))
        dx = rho / dmax
        nb = int(np.floor(xc / dx)) + 3
        xb = np.arange(nb) * dx
        ub = np.sqrt(A + B * np.sin(xb) ** 2)
        w, dk = _table(Kn, dKn, n_int, ub)
        dw = dk * (B * np.sin(xb) * np.cos(xb) / np.maximum(ub, 1e-30)) * dx
        xt = rng.uniform(0, xc, 100000)
        ref, _ = _table(Kn, dKn, n_int, np.sqrt(A + B * np.sin(xt) ** 2))
        p = xt / dx
        j = np.floor(p).astype(int)
        got = _hermite(w[j], w[j + 1], dw[j], dw[j + 1], p - j)
        err = np.abs(got - ref) / peak
        worst_max = max(worst_max, err.max())
        worst_rms = max(worst_rms, np.sqrt(np.mean(err ** 2)))
    assert worst_max < max_bound, worst_max
    assert worst_rms < rms_bound, worst_rms
