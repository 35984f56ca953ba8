"""The library's kernel split (Sec. 2, Eq. 1-6) checked against the oracle, and the
method-level error of split convolution (Sec. 3, Fig. 6-7, Fig. 10).

The truncated-SVD solution is not unique across readings of Eq. 3 (the library
fits rows l <= l_cut exactly and truncates the real-space block; the oracle
truncates the joint system), so the split is compared by what both must satisfy:
the library's model K~ is the exact transform of the kernel it applies, rows
l <= l_cut are exact, and its Eq. 2 residual is no worse than the oracle's.
"""
import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

import oracle as O
from paper_1409_4441_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
ARC = inputs.ARCMIN


@pytest.fixture(scope="module")
def K():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1409_4441_gb300 import ksconv
    return ksconv


def _exact_transform(c, tc):
    lmax = c.size - 1
    x, w = leggauss(2 * (lmax + 1))
    zc = np.cos(tc)
    z = zc + (x + 1) * (1 - zc) / 2
    w = w * (1 - zc) / 2
    Kr = O.legendre_sum(c, z)
    return 2 * np.pi * (O.legendre_matrix(lmax, z).T @ (w * Kr))


@pytest.mark.parametrize("lmax,fwhm,lcut,tc", [(1535, 20.0, 256, 90.0), (767, 30.0, 128, 150.0)])
def test_lsq_split_properties(K, lmax, fwhm, lcut, tc):
    b = inputs.gaussian_beam(lmax, fwhm * ARC)
    cl = inputs.cl_grf(lmax)
    with K.make_split(b, 64, lcut, tc * ARC, cl_in=cl) as sp:
        info = K.split_info(sp)
        kh, cr, kt = K.split_harmonic(sp), K.split_real_coeffs(sp), K.split_model(sp)
    np.testing.assert_allclose(kt[: lcut + 1], b[: lcut + 1], rtol=0, atol=1e-15)
    model = _exact_transform(cr, tc * ARC)
    model[: lcut + 1] += kh
    np.testing.assert_allclose(model, kt, atol=1e-9 * np.abs(b).max())
    e_lib = O.frac_error(b, kt, cl, alpha=1.0)
    assert info["frac_error"] == pytest.approx(5 * e_lib, rel=1e-9)
    assert info["sigma_rms"] == pytest.approx(O.sigma_rms(b, kt, cl), rel=1e-9)
    ref = O.split_lsq(b, lcut, tc * ARC, cl_in=cl)
    e_orc = O.frac_error(b, ref["K_tilde"], cl, alpha=1.0)
    assert e_lib <= 1.1 * e_orc


def test_split_convolution_power_spectrum_error(K):
    """Sec. 3 experiment on the Planck-like workload scaled to nside 256 (every
    angle x8: l_max = 2 nside, 40' beam, l_cut 128, theta_cut 32 deg): the
    harmonic part (oracle synthesis, the paper's CPU half) plus the GPU
    real-space part against the full harmonic convolution of the same
    band-limited field.  Reports the fractional rms C_l error and the map error."""
    nside, lmax, lcut, fwhm, tc = 256, 512, 128, 40 * ARC, 1920 * ARC
    b = inputs.gaussian_beam(lmax, fwhm)
    cl = inputs.cl_grf(lmax)
    alm = inputs.grf_alm(lmax, cl, inputs.seed_for(2))
    ell = np.concatenate([np.arange(mm, lmax + 1) for mm in range(lmax + 1)])
    m = O.alm2map(nside, alm, lmax).astype(np.float32)
    with K.make_split(b, nside, lcut, tc, cl_in=cl) as sp:
        info = K.split_info(sp)
        kh = K.split_harmonic(sp)
        x = torch.tensor(m, device="cuda")
        y = torch.empty_like(x)
        K.conv_real(sp, x, y)
        torch.cuda.synchronize()
        real = y.cpu().numpy().astype(np.float64)
    kfull = np.zeros(lmax + 1); kfull[: lcut + 1] = kh
    # (a) exact synthesis from the generating a_lm
    full_a = O.alm2map(nside, alm * b[ell], lmax)
    split_a = O.alm2map(nside, alm * kfull[ell], lmax) + real
    # (b) the SHT convolution of the pixelised map, as a CPU library would do it
    full_b = O.sht_conv(nside, m.astype(np.float64), b)
    split_b = O.sht_conv(nside, m.astype(np.float64), kfull) + real
    res = {}
    for tag, sp_, fu in (("a", split_a, full_a), ("b", split_b, full_b)):
        cs = O.alm2cl(O.map2alm(nside, sp_, lmax), lmax)
        cf = O.alm2cl(O.map2alm(nside, fu, lmax), lmax)
        res[tag] = (O.eps_cl(cs, cf, lmin=2), np.sqrt(np.mean((sp_ - fu) ** 2) / np.mean(fu ** 2)))
    print(f"\nnside {nside}: eps_C (exact ref) = {res['a'][0]:.3e}, map err = {res['a'][1]:.3e}; "
          f"eps_C (SHT ref) = {res['b'][0]:.3e}, map err = {res['b'][1]:.3e}; "
          f"Eq.6 estimate (alpha 5) = {info['frac_error']:.3e}")
    assert res["a"][0] < 1e-2


def test_wiener_split_through_the_library(K):
    """Noise-dominated splits (Sec. 2: for Wiener filtering the fit is weighted by
    C_l^2 / (C_l + N); Sec. 4's noise-dominated case).  A library split built with that
    weighting satisfies the same properties as the signal-weighted one (rows l <= l_cut
    exact, model = transform of the applied kernel, Eq. 2 residual no worse than the
    oracle's fit with the same weight) and convolves a map within the oracle's per-pixel
    parity (nside 32, the whole map).  Each weighting fits its own residual best only
    where the SVD cut does not bite: at the paper's 1e-6 cut the Wiener weights push one
    more singular direction below it (139 of 148 kept against 140 for flat weights, in
    the oracle as in the library), so the comparison of the two fits under the Wiener
    weight is made at a 1e-10 cut."""
    lmax, fwhm, lcut, tc = 767, 30.0 * ARC, 128, 150.0 * ARC
    b = inputs.gaussian_beam(lmax, fwhm)
    c = inputs.cl_grf(lmax)
    cw = c * c / (c + 1e-5)           # noise above the signal from l ~ 300
    with K.make_split(b, 64, lcut, tc, cl_in=cw) as sp:
        kt_w = K.split_model(sp)
        cr = K.split_real_coeffs(sp)
        kh = K.split_harmonic(sp)
    with K.make_split(b, 64, lcut, tc, cl_in=cw, svd_rcond=1e-10) as sp:
        kt_w10 = K.split_model(sp)
    with K.make_split(b, 64, lcut, tc, svd_rcond=1e-10) as sp:
        kt_f10 = K.split_model(sp)
    np.testing.assert_allclose(kt_w[: lcut + 1], b[: lcut + 1], rtol=0, atol=1e-15)
    model = _exact_transform(cr, tc)
    model[: lcut + 1] += kh
    np.testing.assert_allclose(model, kt_w, atol=1e-9 * np.abs(b).max())
    ref = O.split_lsq(b, lcut, tc, cl_in=cw)
    assert O.sigma_rms(b, kt_w, cw) <= 1.1 * O.sigma_rms(b, ref["K_tilde"], cw)
    assert O.sigma_rms(b, kt_w10, cw) <= 1.05 * O.sigma_rms(b, kt_f10, cw)
    # the weighted split's real-space part on a map
    nside = 32
    m = inputs.white_noise_map(nside, 17).astype(np.float32)
    with K.make_split(b, nside, lcut, tc, cl_in=cw) as sp:
        n_int = K.split_info(sp)["n_intervals"]
        crs = K.split_real_coeffs(sp)
        x = torch.tensor(m, device="cuda")
        y = torch.full_like(x, float("nan"))
        K.conv_real(sp, x, y)
        K.device_status(sp)
        got = y.cpu().numpy().astype(np.float64)
    out, amb = O.brute_conv(nside, m.astype(np.float64), tc, table=O.hermite_nodes(crs, tc, n_int))
    rms = np.sqrt(np.mean(out ** 2))
    assert not np.isnan(got).any()
    assert (np.abs(got - out) <= 1e-6 * rms + amb).all()
