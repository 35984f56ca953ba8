"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module draws random numbers and states input recipes; it holds none of
the method's arithmetic (no geometry, no Legendre sums, no convolution, no
transform).  Everything is deterministic in its seed (numpy PCG64).

Workloads stand in for the paper's data (Sec. 2-3: Planck-resolution HEALPix
maps, nside 2048, l_max 4096, uniform-noise input maps, Gaussian beams).  The
WMAP 7-year spectrum and the Planck maps are not available, so the recipes use
white noise (the paper's "uniform-noise input map") and Gaussian random fields
with C_l = 1/(l+10)^2.
"""
from __future__ import annotations

import numpy as np

ARCMIN = np.pi / (180.0 * 60.0)
DEG = np.pi / 180.0


def seed_for(family: int, index: int = 0) -> int:
    """Seed recipe: 1409 + 100 * family + map index, family = 1 plain nside-64
    convolution, 2 nside-512 split, 3 nside-2048 split, 4 nside-1024 map stacks
    and ragged batches, 5 surrogate training and the nside-4096 map (0: smoke)."""
    return 1409 + 100 * family + index


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def npix(nside: int) -> int:
    return 12 * nside * nside


def white_noise_map(nside: int, seed: int) -> np.ndarray:
    """i.i.d. N(0, 1) pixel values, FP64, RING order."""
    return rng(seed).standard_normal(npix(nside))


def gaussian_beam(lmax: int, fwhm_rad: float) -> np.ndarray:
    """Kernel input: the Gaussian beam B_l = exp(-l(l+1) sigma^2 / 2),
    sigma = FWHM / sqrt(8 ln 2), for l = 0..lmax."""
    sig = fwhm_rad / np.sqrt(8.0 * np.log(2.0))
    ell = np.arange(lmax + 1)
    return np.exp(-ell * (ell + 1) * sig * sig / 2.0)


def cl_grf(lmax: int) -> np.ndarray:
    """Input power spectrum C_l = 1 / (l + 10)^2."""
    ell = np.arange(lmax + 1)
    return 1.0 / (ell + 10.0) ** 2


def grf_alm(lmax: int, cl, seed: int) -> np.ndarray:
    """Random a_lm ~ N(0, C_l) for m >= 0 (m = 0 real, m > 0 complex with
    variance C_l/2 per component), layout idx(l, m) = m(2 lmax + 1 - m)/2 + l."""
    g = rng(seed)
    cl = np.asarray(cl, float)
    out = []
    for m in range(lmax + 1):
        ell = np.arange(m, lmax + 1)
        s = np.sqrt(cl[ell])
        if m == 0:
            out.append(s * g.standard_normal(ell.size) + 0j)
        else:
            out.append(s * (g.standard_normal(ell.size) + 1j * g.standard_normal(ell.size))
                       / np.sqrt(2.0))
    return np.concatenate(out)


def sample_pixels(nside: int, n: int, seed: int) -> np.ndarray:
    """Sorted output-pixel sample: n uniform random pixels plus structural ones
    (both poles' first rings, the cap/belt boundary rings, the equator, the last
    pixel), so that samples always touch the special geometry."""
    N = npix(nside)
    special = {0, 1, 2, 3, N - 1, N - 4}
    ncap = 2 * nside * (nside - 1)
    for base in (ncap - 1, ncap, ncap + 4 * nside, N // 2, N // 2 + 1, N - ncap - 1, N - ncap):
        if 0 <= base < N:
            special.add(base)
    r = rng(seed).choice(N, size=min(n, N), replace=False)
    return np.unique(np.concatenate([np.fromiter(special, np.int64), r.astype(np.int64)]))


def fwhm_draws(n: int, lo_arcmin: float, hi_arcmin: float, seed: int) -> np.ndarray:
    """n beam widths drawn uniformly in [lo, hi] arcmin, returned in radians."""
    return rng(seed).uniform(lo_arcmin, hi_arcmin, size=n) * ARCMIN


def perturbed_coeffs(base, rel: float, seed: int) -> np.ndarray:
    """Kernel coefficients base_l * (1 + rel * N(0,1)): an arbitrary smooth-ish
    kernel for parity tests that should not depend on a particular split."""
    base = np.asarray(base, float)
    return base * (1.0 + rel * rng(seed).standard_normal(base.size))


# Workload recipes (sizes of the paper's Planck-resolution case, Sec. 2-3).
WORKLOADS = {
    "plain_nside64": dict(nside=64, lmax=191, fwhm=2.0 * DEG, theta_cut=6.0 * DEG, mode="none",
               map="white"),
    "split_nside512": dict(nside=512, lmax=1535, fwhm=20.0 * ARCMIN, lcut=256, mode="lsq", map="grf"),
    "planck_nside2048": dict(nside=2048, lmax=4096, fwhm=5.0 * ARCMIN, lcut=1024, theta_cut=240.0 * ARCMIN,
               mode="lsq", map="grf"),
    "multimap_nside1024": dict(nside=1024, lmax=3071, n_maps=64, fwhm_lo=7.0, fwhm_hi=30.0, mode="lsq",
               map="grf"),
    "surrogate_nside4096": dict(nside=4096, lmax=8192, fwhm=3.0 * ARCMIN, mode="lsq", map="grf"),
}
