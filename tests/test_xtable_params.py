"""Host-side sizing of the symmetric gather's weight tables (ksc_dphi_table_params,
no device work).

For a fixed ring pair the weight depends on the pixel pair only through the exact integer
|N| (x = dphi / 2 = |N| c), and the library tabulates it in cubic cells of 2^shift
integers.  For ring pairs of the HEALPix RING grid (geometry written out here from the
public ring definitions) at the benchmark's cut and at a wide cut, the table must: cover
every in-cut |N| (ncut >> shift < ncell) with room for the edge quads' reach of three
positions (6 L in |N|) within the 4096 cells a CTA holds; use the widest power-of-two cell
that stays within 2 K_r-table intervals of the chord and within the in-cut range (no node
more than one cell past the cut, where the K_r table is extrapolated) where that fits, else
the narrowest that fits, at most 3 intervals (no table beyond); place the cut in |N|
exactly; give
whole-ring windows, pairs with no in-cut pixel and pairs entirely within the cut no table.
du/dx is sampled independently of the library's closed-form maximum.
"""
import numpy as np
import pytest

CAP = 4096


def pad(L, shift):
    """Cells an edge quad may read past the table: three positions, 6 L in |N|."""
    return ((6 * L) >> shift) + 2


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
    return A2, B2, np.pi / (2.0 * L * Lq), float(np.float32(hw)), Lq


CASES = [  # nside, theta_cut, n_int, whether some pairs fit 2-interval cells
          # (both do; the wide cut also stretches cells and leaves some pairs without one):
    (2048, np.radians(4.0), 4371, True),    # the benchmark's cut
    (512, np.radians(16.0), 6590, True),    # a wide cut: some cells stretched
]


@pytest.mark.parametrize("nside,theta_cut,n_int,fits", CASES)
def test_table_cells_cover_the_cut_within_three_intervals(K, nside, theta_cut, n_int, fits):
    rng = np.random.default_rng(11)
    n2 = float(n_int) ** 2
    seen = {"table": 0, "stretched": 0, "none": 0}
    for _ in range(300):
        i = int(rng.integers(2, nside))
        span = int(np.ceil(theta_cut / (np.pi / (2 * nside)))) + 2
        iq = int(np.clip(i + rng.integers(-span, span + 1), 1, 4 * nside - 1))
        A2, B2, c, hw, lq = pair(nside, i, iq, theta_cut, n_int)
        t = K.dphi_table_params(A2, B2, c, n_int, hw, lq)
        whole = np.float32(2.0) * np.float32(hw) + np.float32(3.0) >= np.float32(lq)
        if hw < 0 or whole or A2 >= n2 or (n2 - A2) / B2 >= 1.0:
            assert t["ncell"] == 0, (i, iq)
            continue
        xcut = np.arcsin(np.sqrt((n2 - A2) / B2))
        xs = np.linspace(0.0, xcut, 20001)
        u = np.sqrt(A2 + B2 * np.sin(xs) ** 2)
        dmax = np.max(B2 * np.sin(xs) * np.cos(xs) / np.maximum(u, 1e-300))
        L = int(round(np.pi / (2 * c * lq)))
        ncut = int(np.floor(xcut / c))
        # the widest power-of-two cell within 2 intervals, and the narrowest that fits
        s2 = 0
        while (2 ** (s2 + 1)) * c * dmax <= 2.0 * (1 - 1e-6) and 2 ** (s2 + 1) <= ncut + 1:
            s2 += 1
        sf = s2
        while (ncut >> sf) + 1 + pad(L, sf) > CAP:
            sf += 1
        if t["ncell"] == 0:
            assert sf > 0 and (2 ** sf) * c * dmax > 3.0 * (1 - 1e-3), (i, iq)
            seen["none"] += 1
            continue
        dx = t["dx"]
        shift = int(round(np.log2(dx / c)))
        assert dx == pytest.approx(c * 2.0 ** shift, rel=1e-14)  # a power-of-two cell
        assert t["ncell"] == (t["ncut"] // 2 ** shift) + 1  # every in-cut |N| has a cell
        assert t["ncell"] + pad(L, shift) <= CAP
        assert shift == 0 or dx * dmax <= 3.0 * (1 + 1e-3)  # at most 3 intervals per cell
        assert shift == 0 or 2 ** shift <= t["ncut"] + 1 or sf > s2  # no wider than the cut
        if sf == s2:
            assert shift == s2  # within 2 intervals where the cells fit
            assert dx * dmax <= 2.0 * (1 + 1e-3) or shift == 0
            seen["table"] += 1
        else:
            assert shift == sf
            seen["stretched"] += 1
        # the cut in |N|: the largest integer with |N| c <= x_cut
        N = t["ncut"]
        assert N == ncut
        assert N * c <= xcut * (1 + 1e-12) and (N + 1) * c > xcut * (1 - 1e-12)
    assert seen["table"] + seen["stretched"] > 0
    assert (seen["table"] > 0) == fits


def test_no_table_for_degenerate_pairs(K):
    # no in-cut pixel, a whole-ring window, every pixel within the cut
    assert K.dphi_table_params(2.0e7, 1.0e8, 1e-7, 4096, -1.0, 8192)["ncell"] == 0
    assert K.dphi_table_params(0.0, 1.0e8, 1e-7, 4096, 4095.0, 8192)["ncell"] == 0
    assert K.dphi_table_params(0.0, 1.0e6, 1e-7, 4096, 100.0, 8192)["ncell"] == 0


def test_coarser_table_gets_narrower_cells(K):
    A2, B2, c, hw, lq = pair(2048, 1000, 1120, np.radians(4.0), 4371)  # rings ~1.9 deg apart
    full = K.dphi_table_params(A2, B2, c, 4371, hw, lq, 1.0)
    half = K.dphi_table_params(A2, B2, c, 4371, hw, lq, 0.5)
    assert full["ncell"] > 0 and half["ncell"] > 0
    assert half["dx"] < full["dx"]


def test_bad_arguments_are_rejected(K):
    with pytest.raises(RuntimeError):
        K.dphi_table_params(0.0, 1.0, 0.0, 4096, 10.0, 100)
    with pytest.raises(RuntimeError):
        K.dphi_table_params(0.0, 1.0, 1e-6, 0, 10.0, 100)
