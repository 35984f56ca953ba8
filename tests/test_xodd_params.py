"""Host-side sizing of the lockstep gather's odd-step weight tables (ksc_dphi_odd_params,
no device work).

For a fixed ring pair the weight depends on the pixel pair only through the exact integer
|N| (x = dphi / 2 = |N| c).  The lockstep gather tabulates it in cubic cells of 2 lq / m
integers with m odd, at the rational position P = (|N| m + off) / (2 lq): lanes whose
classes are C apart then sit m C cells apart, an odd number.  For ring pairs of the HEALPix
RING grid (geometry written out here from the public ring definitions, as in
test_xtable_params.py) at the benchmark's cut and at a wide cut, the table must: use an odd
m; place the cut exactly (|N| = ncut in the last cubic cell, ncut + 1 in the zero cell);
fit a CTA's cells with its zero cell; keep a cell within 1.5 K_r-table intervals of the
chord where the chord changes fastest unless the cells would not fit (then within 3), and
no wider than the in-cut range; and keep every integer a quarter warp's walk reaches exact.
du/dx is sampled independently of the library's closed-form maximum.
"""
import numpy as np
import pytest

CAP = 4096


@pytest.fixture(scope="module")
def K():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1409_4441_gb300 import ksconv
    return ksconv


def ring(nside, i):
    """z, sin(theta), length of ring i (1-based) of the RING grid."""
    if i < nside:
        z, L = 1 - i * i / (3.0 * nside * nside), 4 * i
    elif i <= 3 * nside:
        z, L = 4.0 / 3 - 2.0 * i / (3 * nside), 4 * nside
    else:
        j = 4 * nside - i
        z, L = -(1 - j * j / (3.0 * nside * nside)), 4 * j
    return z, np.sqrt((1 - z) * (1 + z)), L


def pair(nside, i, iq, theta_cut, n_int):
    zr, sr, L = ring(nside, i)
    zq, sq, Lq = ring(nside, iq)
    dc = 2 * np.sin(theta_cut / 2)
    sc2 = (n_int / dc) ** 2
    A2 = ((zr - zq) ** 2 + (sr - sq) ** 2) * sc2
    B2 = 4 * sr * sq * sc2
    cdp = (1 - 0.5 * dc * dc - zr * zq) / (sr * sq)
    if A2 > dc * dc * sc2 * (1 + 1e-6):
        hw = -1.0
    else:
        dphi = 4 * np.pi if cdp <= -1 else (0.0 if cdp >= 1 else np.arccos(cdp))
        hw = dphi * Lq / (2 * np.pi) + 1
    return A2, B2, np.pi / (2.0 * L * Lq), float(np.float32(hw)), Lq, L


def cells(ncut, m, lq):
    """Index of the zero cell for odd m."""
    return (ncut * m) // (2 * lq) + 1


CASES = [(2048, np.radians(4.0), 4371), (512, np.radians(16.0), 6590)]


@pytest.mark.parametrize("nside,theta_cut,n_int", CASES)
def test_odd_cells_place_the_cut_and_fit(K, nside, theta_cut, n_int):
    rng = np.random.default_rng(12)
    n2 = float(n_int) ** 2
    seen = {"table": 0, "widened": 0, "none": 0}
    for _ in range(300):
        i = int(rng.integers(2, nside))
        span = int(np.ceil(theta_cut / (np.pi / (2 * nside)))) + 2
        iq = int(np.clip(i + rng.integers(-span, span + 1), 1, 4 * nside - 1))
        A2, B2, c, hw, lq, L = pair(nside, i, iq, theta_cut, n_int)
        t = K.dphi_odd_params(A2, B2, c, n_int, hw, lq, 1.0, CAP)
        whole = np.float32(2.0) * np.float32(hw) + np.float32(3.0) >= np.float32(lq)
        if hw < 0 or whole or A2 >= n2 or (n2 - A2) / B2 >= 1.0:
            assert t["nct"] == 0, (i, iq)
            continue
        xcut = np.arcsin(np.sqrt((n2 - A2) / B2))
        ncut = int(np.floor(xcut / c))
        if t["nct"] == 0:
            seen["none"] += 1
            continue
        m, off, nct = t["m"], t["off"], t["nct"]
        D = 2 * lq
        assert m % 2 == 1 and m >= 1
        assert 0 <= off < D
        # the cut in |N|: the largest integer with |N| c <= x_cut, at a cell boundary
        assert t["ncut"] == ncut
        assert ncut * m + off < D * nct <= (ncut + 1) * m + off
        assert nct == cells(ncut, m, lq)
        assert nct + 1 <= CAP
        assert t["width"] == pytest.approx(c * D / m, rel=1e-14)
        # the steepest du/dx, sampled: a cell spans at most 1.5 intervals where the
        # cells fit, and never more than 3
        xs = np.linspace(0.0, xcut, 20001)
        u = np.sqrt(A2 + B2 * np.sin(xs) ** 2)
        dmax = np.max(B2 * np.sin(xs) * np.cos(xs) / np.maximum(u, 1e-300))
        rho = t["width"] * dmax
        assert rho <= 3.0 * (1 + 1e-3)
        assert D / m <= ncut + 1 + 1e-9 or rho <= 1.5 * (1 + 1e-3)
        if rho > 1.5 * (1 + 1e-3):
            # widened only because the next finer odd m would not fit
            assert cells(ncut, m + 2, lq) + 1 > CAP, (i, iq, m)
            seen["widened"] += 1
        else:
            # the least odd m within 1.5 intervals (and the in-cut range)
            if m > 1:
                w2 = c * D / (m - 2)
                assert w2 * dmax > 1.5 * (1 - 1e-3) or D / (m - 2) > ncut + 1
            seen["table"] += 1
        # integers the walk reaches stay exact: |N| below 2^24, |N| m + 2 lq below 2^31
        reach = ncut + 48 * lq + 40 * L
        assert reach < 2 ** 24 and reach * m + D < 2 ** 31
    assert seen["table"] > 0


def test_lanes_sit_an_odd_number_of_cells_apart(K):
    """At one input position, classes C = 3 apart (adjacent lanes of a quarter warp) have
    |N| 2 lq C apart: their cells differ by exactly m C, and the eight lanes of a quarter
    fall in eight different 16-byte bank groups of the table."""
    A2, B2, c, hw, lq, L = pair(2048, 1500, 1580, np.radians(4.0), 4371)
    t = K.dphi_odd_params(A2, B2, c, 4371, hw, lq, 1.0, CAP)
    m, off, D = t["m"], t["off"], 2 * lq
    assert t["nct"] > 0
    for n0 in (0, 7, 12345, t["ncut"] // 3):
        cells_ = [((n0 + D * 3 * l) * m + off) // D for l in range(8)]
        assert all(b - a == 3 * m for a, b in zip(cells_, cells_[1:]))
        assert len({cl % 8 for cl in cells_}) == 8


def test_no_odd_table_for_degenerate_pairs(K):
    # no in-cut pixel, a whole-ring window, every pixel within the cut
    assert K.dphi_odd_params(2.0e7, 1.0e8, 1e-7, 4096, -1.0, 8192)["nct"] == 0
    assert K.dphi_odd_params(0.0, 1.0e8, 1e-7, 4096, 4095.0, 8192)["nct"] == 0
    assert K.dphi_odd_params(0.0, 1.0e6, 1e-7, 4096, 100.0, 8192)["nct"] == 0


def test_odd_params_bad_arguments_are_rejected(K):
    with pytest.raises(RuntimeError):
        K.dphi_odd_params(0.0, 1.0, 0.0, 4096, 10.0, 100)
    with pytest.raises(RuntimeError):
        K.dphi_odd_params(0.0, 1.0, 1e-6, 4096, 10.0, 100, 1.0, 1)
