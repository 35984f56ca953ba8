"""Pins for the oracle's all-pairs real-space convolution (Sec. 1-2, Fig. 1 GPU half)."""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_1409_4441_gb300 import inputs


def _vectors_by_hand(nside):
    """Pixel centres straight from the HEALPix formulas, independent loop."""
    out = []
    n = nside
    for i in range(1, 4 * n):
        if i < n:
            z, L, f = 1 - i * i / (3 * n * n), 4 * i, 1
        elif i <= 3 * n:
            z, L, f = (4 * n - 2 * i) / (3 * n), 4 * n, 1 if (i - n) % 2 == 0 else 0
        else:
            ip = 4 * n - i
            z, L, f = -(1 - ip * ip / (3 * n * n)), 4 * ip, 1
        for k in range(L):
            phi = (2 * k + f) * np.pi / L
            s = np.sqrt(1 - z * z)
            out.append((s * np.cos(phi), s * np.sin(phi), z))
    return np.array(out)


@pytest.mark.parametrize("nside", [1, 2])
def test_brute_force_tiny_by_hand(nside):
    v = _vectors_by_hand(nside)
    np.testing.assert_allclose(O.pix2vec(nside), v, atol=1e-15)
    N = v.shape[0]
    m = inputs.white_noise_map(nside, 5)
    c = inputs.perturbed_coeffs(O.gaussian_beam(6, 0.8), 0.2, 6)
    tc = 1.2
    ref = np.zeros(N)
    for i, j in itertools.product(range(N), range(N)):
        cosang = float(np.clip(v[i] @ v[j], -1, 1))
        if np.arccos(cosang) <= tc:
            ref[i] += O.legendre_sum(c, [cosang])[0] * m[j] * 4 * np.pi / N
    got, amb = O.brute_conv(nside, m, tc, c=c)
    np.testing.assert_allclose(got, ref, atol=1e-14)
    assert np.all(amb == 0)


def test_constant_map_and_unit_kernel():
    nside = 8
    c = np.zeros(5); c[0] = 1.0  # K = 1/(4 pi): the unit-integral constant kernel
    out, _ = O.brute_conv(nside, np.full(O.npix(nside), 2.5), np.pi, c=c)
    np.testing.assert_allclose(out, 2.5, rtol=1e-13)


def test_delta_map_gives_kernel_profile():
    nside = 16
    N = O.npix(nside)
    lmax = 47
    c = O.gaussian_beam(lmax, np.radians(8.0))
    tc = np.radians(25.0)
    j0 = 1234
    m = np.zeros(N); m[j0] = 1.0
    out, _ = O.brute_conv(nside, m, tc, c=c)
    v = O.pix2vec(nside)
    cosang = np.clip(v @ v[j0], -1, 1)
    inside = np.arccos(cosang) <= tc
    ref = np.where(inside, O.legendre_sum(c, cosang) * 4 * np.pi / N, 0.0)
    np.testing.assert_allclose(out, ref, atol=1e-15)


def test_quarter_turn_permutes_output():
    nside = 8
    z, s, ln, st, ph = O.ring_table(nside)
    m = inputs.white_noise_map(nside, 7)
    c = O.gaussian_beam(23, np.radians(10.0))
    tc = np.radians(30.0)

    def rot(x):
        y = np.empty_like(x)
        for r in range(z.size):
            y[st[r]: st[r] + ln[r]] = np.roll(x[st[r]: st[r] + ln[r]], ln[r] // 4)
        return y
    a, _ = O.brute_conv(nside, m, tc, c=c)
    b, _ = O.brute_conv(nside, rot(m), tc, c=c)
    np.testing.assert_allclose(b, rot(a), atol=1e-14)


def test_table_mode_matches_exact_mode():
    nside = 16
    lmax = 47
    c = O.gaussian_beam(lmax, np.radians(5.0))
    tc = np.radians(15.0)
    m = inputs.white_noise_map(nside, 8)
    ex, _ = O.brute_conv(nside, m, tc, c=c)
    tab = O.hermite_nodes(c, tc, 2048)
    tb, _ = O.brute_conv(nside, m, tc, table=tab)
    np.testing.assert_allclose(tb, ex, atol=1e-9 * np.abs(ex).max())


def test_pair_counts_match_cap_area():
    nside = 16
    tc = np.radians(12.0)
    cnt = O.count_pairs(nside, tc)
    N = O.npix(nside)
    area = (1 - np.cos(tc)) / 2 * N
    assert abs(cnt.mean() / area - 1) < 0.02
    assert cnt.sum() % 2 == 0  # symmetric relation
    # whole sphere
    assert np.all(O.count_pairs(4, np.pi) == O.npix(4))


def test_ambiguity_bound_flags_boundary_pairs():
    nside = 4
    v = O.pix2vec(nside)
    tc = float(np.arccos(v[0] @ v[5]))  # put a pair exactly on the cut
    m = np.ones(O.npix(nside))
    c = np.zeros(3); c[0] = 1.0
    _, amb = O.brute_conv(nside, m, tc, c=c, out_pix=[0])
    assert amb[0] >= 4 * np.pi / O.npix(nside) / (4 * np.pi) * 0.999


def test_pair_counts_exact_at_nside1():
    """The twelve nside-1 pixels have closed-form centres: z = 2/3 at phi = pi/4 + k pi/2
    (ring 1), z = 0 at phi = k pi/2 (ring 2), z = -2/3 at phi = pi/4 + k pi/2 (ring 3),
    in RING order.  Every pair count within theta_cut, brute force on these vectors,
    equals the oracle's, pixel by pixel, at cuts between each distinct separation."""
    k = np.arange(4)
    z = np.repeat([2.0 / 3.0, 0.0, -2.0 / 3.0], 4)
    phi = np.concatenate([np.pi / 4 + k * np.pi / 2, k * np.pi / 2, np.pi / 4 + k * np.pi / 2])
    s = np.sqrt(1 - z ** 2)
    v = np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)
    d = np.sqrt(((v[:, None, :] - v[None, :, :]) ** 2).sum(-1))  # chord: self pairs exactly 0
    ang = 2 * np.arcsin(np.minimum(d / 2, 1.0))
    seps = np.unique(np.round(ang, 6))  # (antipodes: pi to rounding)
    cuts = (seps[:-1] + seps[1:]) / 2
    assert cuts.size >= 4
    for tc in cuts:
        want = (ang <= tc).sum(axis=1)
        assert np.array_equal(O.count_pairs(1, tc), want), np.degrees(tc)
