"""Pins for the oracle's HEALPix ring geometry (Gorski et al. 2005, used in Sec. 2)."""
import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 32])
def test_counts_and_contiguity(nside):
    z, s, ln, st, ph = O.ring_table(nside)
    assert z.size == 4 * nside - 1
    assert ln.sum() == 12 * nside ** 2
    assert st[0] == 0
    assert np.all(st[1:] == st[:-1] + ln[:-1])
    # ring lengths: 4i in the caps, 4n in the belt
    i = np.arange(1, 4 * nside)
    expect = np.where(i < nside, 4 * i, np.where(i <= 3 * nside, 4 * nside, 4 * (4 * nside - i)))
    assert np.array_equal(ln, expect)
    assert np.all(np.diff(z) < 0)
    np.testing.assert_allclose(s * s + z * z, 1.0, atol=1e-15)


def test_nside1_base_pixels():
    v = O.pix2vec(1)
    z = v[:, 2]
    phi = np.mod(np.arctan2(v[:, 1], v[:, 0]), 2 * np.pi)
    np.testing.assert_allclose(z, [2 / 3] * 4 + [0] * 4 + [-2 / 3] * 4, atol=1e-15)
    q = np.pi / 2
    np.testing.assert_allclose(phi[:4], [q / 2, 3 * q / 2, 5 * q / 2, 7 * q / 2], atol=1e-14)
    np.testing.assert_allclose(phi[4:8], [0, q, 2 * q, 3 * q], atol=1e-14)
    np.testing.assert_allclose(phi[8:], phi[:4], atol=1e-14)


@pytest.mark.parametrize("nside", [2, 8, 64])
def test_unit_vectors_balance_and_equal_area(nside):
    v = O.pix2vec(nside)
    np.testing.assert_allclose(np.linalg.norm(v, axis=1), 1.0, atol=2e-16 * 8)
    assert np.abs(v.sum(axis=0)).max() < 1e-10 * v.shape[0]
    # equal area: the fraction of pixels north of each ring boundary equals the
    # cap area fraction (1 - z)/2 exactly at the cap/belt boundary z = 2/3
    N = v.shape[0]
    ncap = 2 * nside * (nside - 1)
    # pixels in rings 1..n-1 plus half of ring n lie above z = 2/3
    assert (ncap + 2 * nside) / N == pytest.approx((1 - 2 / 3) / 2, abs=1e-15)
    # for every belt ring the pixels north of it (plus half of it) match (1-z)/2
    z, s, ln, st, ph = O.ring_table(nside)
    for r in range(nside - 1, 3 * nside):
        frac = (st[r] + ln[r] / 2) / N
        assert frac == pytest.approx((1 - z[r]) / 2, abs=1e-15)


@pytest.mark.parametrize("nside", [4, 16])
def test_fourfold_and_mirror_symmetry(nside):
    v = O.pix2vec(nside)
    z, s, ln, st, ph = O.ring_table(nside)
    rot = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1.0]])
    for r in range(z.size):
        seg = v[st[r]: st[r] + ln[r]]
        q = ln[r] // 4
        np.testing.assert_allclose(seg @ rot.T, np.roll(seg, -q, axis=0), atol=1e-14)
        rm = z.size - 1 - r  # mirror ring
        segm = v[st[rm]: st[rm] + ln[rm]]
        np.testing.assert_allclose(segm[:, 2], -seg[:, 2], atol=1e-15)
        np.testing.assert_allclose(segm[:, :2], seg[:, :2], atol=1e-14)
